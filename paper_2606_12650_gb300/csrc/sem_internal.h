// sem_internal.h -- types and launchers shared by the libsem translation units.
//
// Not part of the public ABI (include/sem.h is).  Everything here is plain
// C++/CUDA for sm_103a; no torch types.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "sem.h"

namespace sem {

constexpr int kMaxQ = 10;          // N <= 9  ->  N+1 <= 10 points per direction
// Grid sums of many blocks in two levels (publish_grouped): groups of
// kSumGroup consecutive blocks.  A problem's partials buffer holds `cap`
// block partials, then cap / kSumGroup group sums (doubles), then
// cap / kSumGroup group tickets (uint32, zero between launches); cap is at
// least kMinPartials and at least the problem's element count (the largest
// grid any of its launches uses: the operator at one element per block), a
// multiple of kSumGroup, and is stored as a uint64 in the 16 bytes before
// the buffer, where device code reads it.
constexpr int kSumGroup = 32;
constexpr int64_t kMinPartials = 1 << 17;
inline int64_t partials_cap(int64_t E) {
    const int64_t e = (E + kSumGroup - 1) / kSumGroup * kSumGroup;
    return e > kMinPartials ? e : kMinPartials;
}
// bytes of the allocation (header included)
inline size_t partials_bytes(int64_t cap) {
    return 16 + sizeof(double) * size_t(cap + cap / kSumGroup) + sizeof(uint32_t) * size_t(cap / kSumGroup);
}
__device__ __forceinline__ int64_t partials_capacity(const double *partials) {
    return int64_t(__ldg(reinterpret_cast<const unsigned long long *>(partials) - 2));
}
__host__ __device__ inline uint32_t *group_tickets(double *partials, int64_t cap) {
    return reinterpret_cast<uint32_t *>(partials + cap + cap / kSumGroup);
}

// Small per-problem constants passed to kernels by value (constant bank).
struct OpConsts {
    double D[kMaxQ * kMaxQ];       // D[i*nq + l] = l_l'(xi_i)
    double xi[kMaxQ];
    double w[kMaxQ];
};

// Device-resident CG state: scalars of the recurrences, the iteration
// counter, the stop flag and the tickets of the last-block reductions.
struct CgState {
    double rho;        // <r_k, r_k>
    double rho0;       // <r_0, r_0>
    double alpha;
    double beta;
    double pap;        // <p, A p>
    double tol;        // stop when sqrt(rho/rho0) <= tol (tol <= 0: never)
    double dot_out;    // result slot of the "dot" kernel
    double rr;         // PCG: <r_k, r_k> (the stop test uses sqrt(rr / bb))
    double bb;         // PCG: <b, b>
    double *hist;      // optional: hist[k] = sqrt(rho_k)
    int32_t iter;
    int32_t maxit;
    int32_t done;
    int32_t pad0;
    uint32_t ticket_ax;
    uint32_t ticket_up;
    uint32_t ticket_dot;
    uint32_t pad1;
};

// Status word written by kernels whose bounded waits give up.
enum DeviceStatus : int32_t {
    kStatusOk = 0,
    kStatusMbarTimeout = 1,
};

struct Problem {
    int nx = 0, ny = 0, nz = 0, N = 0, nq = 0;
    int64_t E = 0, np = 0, nL = 0, nG = 0;
    OpConsts oc{};
    double *verts = nullptr;       // [(nx+1)(ny+1)(nz+1)][3] device copy of the vertices

    // geometry (FP64): G interleaved per node [nL][6] = (rr, rs, rt, ss, st, tt)
    double *G = nullptr;
    double *B = nullptr;           // [nL] mass weights W |J|
    double *c = nullptr;           // [nL] 1 / multiplicity

    bool maps_ready = false;       // the four arrays below exist (built on first use)
    // direct-stiffness sum: global ids with >= 2 copies, copies ascending
    int32_t *sh_ptr = nullptr, *sh_idx = nullptr;
    int64_t n_sh = 0, n_sh_copies = 0;
    // Dirichlet mask: local indices on the cube boundary
    int32_t *msk_idx = nullptr;  // local indices on the cube boundary
    int64_t n_mask = 0;

    // CG work vectors and state
    double *x = nullptr, *r = nullptr, *p = nullptr, *w = nullptr;
    double *dinv = nullptr;        // Jacobi: 1 / diag(A) (0 on masked nodes), on first PCG use
    cudaGraphExec_t graph_pcg = nullptr;
    double *partials = nullptr;    // after a 16-byte header holding partials_cap (see above)
    int64_t partials_cap = 0;
    CgState *st = nullptr;
    CgState *st_host = nullptr;    // pinned mirror for polling (pad0: the mesh check's flag at set-up)
    int32_t *bad_dev = nullptr;    // deferred set-up: the geometry kernel's flag until read
    cudaGraphExec_t graph = nullptr;
    int graph_iters = 0;
    cudaStream_t graph_stream = nullptr;

    uint64_t graph_epoch = 0;      // operator-variant epoch the graphs above were captured at

    // mixed precision (allocated on first use): geometric factors rounded to
    // FP32 or BF16 ([nL][6]), FP32 inner-CG vectors and the inner CG state
    void *G32 = nullptr;           // float
    void *G16 = nullptr;           // __nv_bfloat16
    // double-word FP64 operator (allocated on first use): [nL][6] (h, l) FP32 pairs
    float *Gdw = nullptr;
    float *d32 = nullptr, *r32 = nullptr, *p32 = nullptr, *w32 = nullptr;
    CgState *st_in = nullptr;
    CgState *st_in_host = nullptr;
    cudaGraphExec_t graph32[2] = {nullptr, nullptr};  // per geometric-factor precision
    int graph32_iters = 0;
    cudaStream_t graph32_stream = nullptr;
};

// storage precision of the geometric factors in mixed-precision inner solves
enum GPrecision : int { kGF32 = 0, kGBF16 = 1 };

// ---- operator variants and the per-order tuner (sem_tune.cu) ---------------
// Variants of the local operator: the column kernel of sem_ax_kernel.cuh
// (one thread per (i, j) column, fixed elements per block), the line kernel
// of sem_ax_lines.cuh (whole lines per thread, even-odd split, elements per
// block chosen at launch), and the persistent TMA-pipelined column kernel of
// sem_ax32p.cuh (FP32 only), and the line kernel with the geometric factors
// loaded into registers before the slab wait (FP32 with BF16 factors only) or
// staged in shared memory with the slab (FP32), and the line kernel of the
// FP64 operator in double-word FP32 arithmetic (sem_ax_dw.cuh, FP64 only).
enum AxVariant : int {
    kAxColumns = 0,
    kAxLines = 1,
    kAxPersistent = 2,
    kAxLinesPrefetch = 3,
    kAxLinesStaged = 4,
    kAxLinesDW = 5,
    kAxVariants = 6
};
// What is tuned: the FP64 operator, and the FP32 operator with FP32 or BF16
// geometric factors.
enum TuneKind : int { kTuneF64 = 0, kTuneF32G32 = 1, kTuneF32G16 = 2, kTuneKinds = 3 };
struct TuneChoice {
    int variant;
    int epb;       // elements per block (line kernel); 0 = the variant's own
    double us;     // measured time of one CG-operator launch (0: not measured)
};
TuneChoice tune_get(int kind, int nq);
void tune_set(int kind, int nq, const TuneChoice &c);     // bumps the epoch
uint64_t tune_epoch();                                    // graphs captured earlier are stale
void tune_reset();                                        // back to the built-in defaults
int tune_check(int kind, int nq, const TuneChoice &c);    // SEM_OK or SEM_EARG (error set)
int tune_kind_of_gprec(int gprec);
// Times every candidate of `kind` on P's CG operator (reps launches each),
// keeps the fastest.  cand: up to cap (variant, epb, us) triples.
int tune_problem(Problem *P, int kind, int reps, double *cand, int cap, int *n_cand, TuneChoice *best);
int tune_save(const char *path);
int tune_load(const char *path);
// line-kernel launchers (sem_ax_lines64.cu, sem_ax_lines32.cu); mode 0: y = A x,
// 1: CG operator on P's vectors, 2: Jacobi-PCG operator
int launch_lines64(const Problem *P, const double *x, double *y, int mode, int epb);
// double-word FP64 operator (sem_ax_dw.cu); needs P->Gdw (dw_prepare, not during a capture)
int launch_lines_dw(const Problem *P, const double *x, double *y, int mode, int epb);
int dw_prepare(Problem *P);                   // allocate + fill P->Gdw (once)
void dw_release(Problem *P);
int prepare_f64_variant(Problem *P);          // whatever the tuned FP64 variant needs (before a capture)
// gm: where phase 2 reads the factors (0 global, 1 registers, 2 staged in shared memory)
int launch_lines32(const Problem *P, const float *x, float *y, int gprec, bool cg, int epb, int gm);
bool lines_epb_ok(int nq, int epb, size_t elem_bytes, int g_stage_bytes = 0);
void problem_drop_graphs(Problem *P);                     // sem_setup.cu

// ---- runtime services (sem_api.cu) ---------------------------------------
void *dev_alloc(size_t bytes);               // nullptr on failure (error set)
void dev_free(void *p);
// One allocation carved into many (sem_api.cu): dev_alloc inside an
// ArenaScope takes pieces of the arena, dev_free of a piece is a no-op,
// arena_release frees the arena (no piece may be in use on the GPU).
struct DevArena;
DevArena *arena_new(size_t bytes);           // nullptr on failure (error set)
void arena_release(DevArena *a);
struct ArenaScope {
    DevArena *prev;
    explicit ArenaScope(DevArena *a);
    ~ArenaScope();
};
cudaStream_t stream();
// Routes stream() of the calling thread to `s` while the scope lives.
struct StreamScope {
    cudaStream_t prev;
    explicit StreamScope(cudaStream_t s);
    ~StreamScope();
};
void *pinned_slot_alloc();                   // 256 pinned host bytes (CgState mirror); nullptr + error
void pinned_slot_free(void *p);
int sm_count();                    // SMs of the current device
int32_t *status_word();            // device status word (kernels write it)
int32_t *status_host();            // pinned host copy (filled by poll_status / cg_solve)
int poll_status();                 // sync, read and clear the status word -> SEM_OK/SEM_ETIMEDOUT
void count_launches(int64_t n);
int set_error(int code, const std::string &msg);
int cuda_check(cudaError_t err, const char *what);

// ---- setup (sem_setup.cu) --------------------------------------------------
void gll_rule_and_derivative(int N, double *xi, double *w, double *D);   // D row-major (N+1)^2
// deferred: issue the set-up on stream() without waiting; the caller waits for
// the stream, then calls problem_check_mesh (SEM_EMESH for an inverted element)
int problem_create(int nx, int ny, int nz, int N, const double *verts_dev, Problem **out, bool deferred = false);
int problem_check_mesh(const Problem *P);
int problem_maps(Problem *P);                 // gs maps, mask list, weights c (lazy)
void problem_destroy(Problem *P);
int launch_nodes(const Problem *P, const double *verts_dev, double *X);
int launch_rhs_sin(const Problem *P, const double *verts_dev_or_null, double *b);
int launch_scale(const Problem *P, const double *a, const double *f, double *out);

// ---- operators (sem_ax.cu, sem_cg.cu) --------------------------------------
int prepare_ax(const Problem *P);             // kernel attributes (before any capture)
int launch_ax(const Problem *P, const double *x, double *y);
int launch_ax_cg(const Problem *P);          // p = r + beta p; w = A_local p; <p,w>
int prepare_ax32(const Problem *P);
int convert_geometry(const Problem *P, int gprec, void *out);
int launch_ax32(const Problem *P, const float *x, float *y, int gprec);
int launch_ax32_cg(const Problem *P, int gprec);   // inner CG on r32/p32/w32 with st_in
int mixed_prepare(Problem *P, int gprec);          // allocate + convert on first use
int mixed_solve(Problem *P, const double *b, double *x, double tol, int max_outer, double inner_tol,
                int inner_maxit, int gprec, int64_t *inner_iters, int64_t *outer_iters, double *rel_res,
                double *hist_outer);
void mixed_release(Problem *P);
int launch_gs(const Problem *P, double *u);
int launch_mask(const Problem *P, double *u);
int launch_dot(const Problem *P, const double *u, const double *v);  // -> st->dot_out
int launch_sub(const Problem *P, const double *a, const double *b, double *out);  // out = a - b
int launch_cg_init(const Problem *P, const double *b, int maxit, double tol, double *hist);
int launch_cg_update(const Problem *P);
int launch_x_finish(const Problem *P);       // x += alpha p of the last iteration (deferred update)
int cg_solve(Problem *P, const double *b, double *x, double tol, int maxit, double *hist,
             int64_t *iters, double *rel_res);
int launch_ax_pcg(const Problem *P);         // p = dinv r + beta p; w = A_local p; <p,w>
int jacobi_prepare(Problem *P);              // dinv = 1 / (mask(QQ^T diag(A_local)))
int pcg_solve(Problem *P, const double *b, double *x, double tol, int maxit, double *hist,
              int64_t *iters, double *rel_res);

// ---- batches (sem_batch.cu) -------------------------------------------------
struct Batch;
Batch *batch_new(int mode, double tol, int maxit, double inner_tol, int max_outer, int K);
int batch_set(Batch *B, Problem **probs, const double *const *b, const uint8_t *start, int n);
int batch_round(Batch *B, std::vector<int> *done);
int batch_round_launch(Batch *B);                       // the round's launches, no wait
int batch_round_finish(Batch *B, std::vector<int> *done);   // wait, finished problems
int batch_results(Batch *B, int64_t *iters, double *res);
int batch_results_of(Batch *B, const std::vector<int> &which, int64_t *iters, double *res);
int batch_create(Problem **probs, int n, Batch **out);
void batch_destroy(Batch *B);
int64_t batch_total_nodes(const Batch *B);
int batch_size(const Batch *B);
int batch_solve(Batch *B, const double *b_all, double *x_all, double tol, int maxit, int mode, double inner_tol,
                int max_outer, int64_t *iters, double *res);

// ---- serving (sem_serve.cu) -------------------------------------------------
struct Server;
int serve_open(int capacity, double budget_gb, int mode, double tol, double inner_tol, int K, int maxit,
               Server **out);
int serve_submit(Server *S, int nx, int ny, int nz, int N, const double *verts, const double *b, bool assemble,
                 double arrival, int64_t *ticket);
int64_t serve_drain(Server *S, int64_t *out, int64_t cap);
int serve_step(Server *S, int64_t *n_queued, int64_t *n_active, int64_t *n_completed);
int serve_result(Server *S, int64_t ticket, double *x_out, bool x_on_device, int64_t *state, int64_t *iters,
                 double *rel_res, double *latency_ms);
int64_t serve_nodes_of(const Server *S, int64_t ticket);
double serve_now(const Server *S);
void serve_close(Server *S);

// ---- one problem split by element slabs across ranks (sem_dist.cu) ---------
struct DistProblem;
int dist_create(int nx, int ny, int nz, int N, const double *verts_dev, bool below, bool above, DistProblem **out);
void dist_destroy(DistProblem *D);
Problem *dist_problem(DistProblem *D);
int dist_gs(DistProblem *D, double *u, const sem_comm *comm);
int dist_dot(DistProblem *D, const double *u, const double *v, const sem_comm *comm, double *out);
int dist_cg_solve(DistProblem *D, const double *b, double *x, double tol, int maxit, double *hist,
                  const sem_comm *comm, int64_t *iters, double *rel_res);

// ---- device facts (sem_probe.cu) --------------------------------------------
int probe_fma_rate(int dtype, int iters, double *flops_per_s);   // dtype 0: f64, 1: f32
// failure-detection self-test: a bounded mbarrier wait that runs out (status word set)
int probe_wait_timeout(uint64_t limit_ns, double *copied_value);

}  // namespace sem
