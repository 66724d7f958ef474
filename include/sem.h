/*
 * sem.h -- C-ABI of libsem, a GB300 (sm_103a) library for the spectral-element
 * Poisson operator and its conjugate-gradient solve.
 *
 * The interface has the shape of the runtime calls that the paper's pragmas
 * lower to (Section IV, Fig. "Syntax of the nomp directives", and Section V):
 * initialise the runtime, map host arrays to and from the device, run a named
 * kernel, synchronise, finalise.  There is no source-to-source compiler and no
 * JIT here: every named kernel is hand-written CUDA, specialised at compile
 * time on the polynomial order N (the role the paper gives to the "jit"
 * clause, Section VIII-B).
 *
 * Conventions shared by every call
 *   - Every function returns an int status: SEM_OK (0) or a negative SEM_E*
 *     code.  sem_last_error() returns a message for the last failure of the
 *     calling thread's most recent call.
 *   - The library is single-context: one device, one stream.  Calls are not
 *     thread-safe; serialise them.
 *   - Device memory is obtained through the allocator installed with
 *     sem_set_allocator (cudaMalloc/cudaFree by default).  The library never
 *     holds host memory of the caller beyond a call, except the host base
 *     pointers that key the device mirrors of sem_update.
 *   - Vectors on local nodes use the layout l = i + n*(j + n*(k + n*e)),
 *     n = N+1, i (the r direction) fastest, e = ex + nx*(ey + ny*ez).
 *   - Device arrays passed to kernels must be 16-byte aligned.
 */
#ifndef SEM_H
#define SEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define SEM_OK          0
#define SEM_EINIT      -1  /* not initialised, initialised twice, or finalised */
#define SEM_EARG       -2  /* malformed argument (count, kind, value, alignment) */
#define SEM_ENOMAP     -3  /* host array has no device mirror */
#define SEM_ERANGE     -4  /* range outside the mirror, or size above a limit */
#define SEM_ENOMEM     -5  /* device allocation failed or HBM budget exceeded */
#define SEM_EKERNEL    -6  /* unknown kernel name */
#define SEM_ETIMEDOUT  -7  /* a bounded device wait gave up (device status word) */
#define SEM_ECUDA      -8  /* CUDA runtime error (message has the CUDA text) */
#define SEM_EMESH      -9  /* invalid mesh: non-positive Jacobian */
#define SEM_EHANDLE   -10  /* unknown problem handle */
#define SEM_ECOMM     -11  /* a sem_comm callback (exchange, allreduce) reported failure */

/* ---- sem_update operations (Section IV, Table "update operations") ------- */
#define SEM_ALLOC 0  /* allocate the device mirror of host[start, end), no copy  */
#define SEM_TO    1  /* copy host[start, end) to the device (allocating if needed) */
#define SEM_FROM  2  /* copy device[start, end) back to host[start, end)          */
#define SEM_FREE  3  /* release the device mirror                                 */

/* ---- sem_run argument kinds --------------------------------------------- */
#define SEM_ARG_INT        0  /* v.i : integer value                               */
#define SEM_ARG_DOUBLE     1  /* v.d : double value                                */
#define SEM_ARG_MAPPED     2  /* v.ptr : host address inside a sem_update mirror;  */
                              /*        resolved to the device address            */
#define SEM_ARG_DEVICE     3  /* v.ptr : device address (caller-owned memory)      */
#define SEM_ARG_OUT_DOUBLE 4  /* v.ptr : host double*, written before sem_run      */
                              /*        returns (sem_run then syncs its stream)   */
#define SEM_ARG_OUT_INT    5  /* v.ptr : host int64_t*, as above                   */
#define SEM_ARG_NONE       6  /* absent optional array                             */
#define SEM_ARG_HOST       7  /* v.ptr : host array read or written during the     */
                              /*        call only (small per-problem lists)       */

typedef struct sem_arg {
    int32_t kind;
    int32_t reserved;
    union {
        int64_t i;
        double d;
        void *ptr;
    } v;
} sem_arg;

/* Communication between the ranks of one problem split across processes
 * ("dist_*" kernels; Nekbone runs its CG under MPI with the elements divided
 * among ranks, Section VIII-A; the paper names multi-node runs as future
 * work, Section IX).  libsem calls these on the calling thread with HOST
 * buffers it owns (pinned); each returns 0 on success, anything else makes
 * the calling sem_run return SEM_ECOMM.
 *   allreduce_sum(ctx, vals, n): vals[0..n) <- their sum over all ranks, the
 *       same bits on every rank.
 *   exchange(ctx, send_lo, recv_lo, send_hi, recv_hi, n): send n values to
 *       the rank below (send_lo) / above (send_hi) and receive theirs into
 *       recv_lo / recv_hi; a NULL pair means there is no such neighbour.
 * The struct is passed to sem_run as a SEM_ARG_HOST pointer. */
typedef struct sem_comm {
    int (*allreduce_sum)(void *ctx, double *vals, int n);
    int (*exchange)(void *ctx, const double *send_lo, double *recv_lo, const double *send_hi, double *recv_hi,
                    int64_t n);
    void *ctx;
} sem_comm;

/* Device allocator hooks: alloc returns a device pointer (NULL on failure,
 * 256-byte aligned or better); free releases it.  ctx is passed through. */
typedef void *(*sem_alloc_fn)(size_t bytes, void *ctx);
typedef void (*sem_free_fn)(void *ptr, void *ctx);

/* Initialise the runtime (Section IV: "init" takes C-style command-line
 * arguments with runtime configuration).  Recognised arguments:
 *   --device=K        CUDA device ordinal (default 0)
 *   --verbose=V       0 silent (default), 1 setup messages on stderr
 *   --hbm-budget=GB   cap on device bytes the library allocates (default: none)
 *   --autotune-table=PATH  operator table written by "autotune_save"; a file
 *                     that cannot be read or has a bad entry fails sem_init
 *                     with SEM_EARG (the table starts from built-in defaults)
 * Unknown arguments are ignored.  A second sem_init without sem_finalize
 * returns SEM_EINIT.  Queries the device (name, SM count, shared memory per
 * block, the analogue of the paper's "context" table, Section V-B). */
int sem_init(int argc, const char **argv);

/* Map host arrays to and from the device (Section IV, "update" directive and
 * its alloc/to/from/free table).  The mirror is keyed by the host base
 * address `host` and covers elements [start, end) of size elem_size.
 *   SEM_ALLOC  creates the mirror (SEM_EARG if one exists for `host`).
 *   SEM_TO     copies host[start, end) into the mirror, creating it first if
 *              `host` has none; an existing mirror must contain the range.
 *   SEM_FROM   copies the range back; SEM_ENOMAP without a mirror, SEM_ERANGE
 *              if the range lies outside it.
 *   SEM_FREE   releases the mirror (SEM_ENOMAP without one).
 * Copies are ordered on the library stream and asynchronous with respect to
 * the host when the host memory is pinned; results of SEM_FROM are visible
 * after sem_sync (or any sem_run that syncs).  The caller keeps ownership of
 * the host memory; the library owns the mirror until SEM_FREE or
 * sem_finalize.  SEM_ENOMEM if the allocation fails or exceeds the budget. */
int sem_update(void *host, size_t start, size_t end, size_t elem_size, int op);

/* Run a named kernel (Section IV, "for" directive -> jit + run; the "name"
 * clause names kernels).  Arrays are SEM_ARG_MAPPED or SEM_ARG_DEVICE; the
 * list below gives arguments in order ([..] = optional, SEM_ARG_NONE or
 * omitted).  Local vectors have nL = E (N+1)^3 doubles.  Kernels are launched
 * on the library stream; a call with an OUT argument syncs before returning.
 *
 *   "mesh"      nx, ny, nz, N, verts[(nx+1)(ny+1)(nz+1)*3], OUT handle
 *               Build a problem on an nx*ny*nz box of order N (1 <= N <= 9):
 *               GLL rule, derivative matrix, trilinear geometry (6 factors
 *               and mass weight per node, FP64), direct-stiffness map,
 *               Dirichlet mask and multiplicity weights.  SEM_EMESH if a
 *               Jacobian is not positive.  Vertex v = a+(nx+1)(b+(ny+1)c).
 *   "mesh_free" handle
 *   "info"      handle, OUT nL, OUT nG, OUT n_shared_ids, OUT n_masked
 *   "ax"        handle, x, y            y = A_local x (per element, no sum)
 *   "gs"        handle, u               u = QQ^T u in place; copies summed in
 *                                       ascending local index (deterministic)
 *   "mask"      handle, u               zero the Dirichlet-boundary copies
 *   "axg"       handle, x, y            y = mask(QQ^T(A_local x))
 *   "dot"       handle, u, v, OUT d     sum_l c_l u_l v_l, c = 1/multiplicity
 *   "geom"      handle, G[nL*6], B[nL]  copy out factors (rr,rs,rt,ss,st,tt)
 *   "nodes"     handle, X[nL*3]         nodal coordinates
 *   "gs_map"    handle, ptr[n_shared_ids+1] int32, idx[ptr[end]] int32
 *               copies of each shared global id (ids in the library's
 *               internal order), copies ascending
 *   "rhs"       handle, f, b            b = mask(QQ^T(B f))
 *   "rhs_sin"   handle, b               f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z)
 *   "cg_solve"  handle, b, x, tol, maxit, OUT iters, OUT rel_res, [hist]
 *               Unpreconditioned CG from x = 0 (Section VIII-A) until
 *               sqrt(rho_k/rho_0) <= tol or maxit iterations (tol <= 0: exactly
 *               maxit).  rho = <r,r>_c.  hist (maxit+1 doubles, optional)
 *               receives sqrt(rho_k).  rel_res = sqrt(rho/rho_0) at exit.
 *   "true_res"  handle, b, x, OUT d     ||b - A x||_c / ||b||_c (FP64)
 *   "pcg_solve" handle, b, x, tol, maxit, OUT iters, OUT rel_res, [hist]
 *               Jacobi-preconditioned CG (the original Nekbone method,
 *               Section VIII-A): M = diag of the assembled, masked operator;
 *               stops when ||r||_c/||b||_c <= tol; hist[k] = ||r_k||_c.
 *   "jacobi"    handle, dinv[nL]        the preconditioner 1/diag(A) (0 on
 *                                       masked nodes), FP64
 *   "ax32"      handle, x, y, gprec     y = A_local x in FP32 (x, y: nL floats);
 *                                       geometric factors rounded to nearest
 *                                       even from FP64 to FP32 (gprec 0) or
 *                                       BF16 (gprec 1), converted once per problem
 *   "cg_ax32"   handle, gprec           one launch of the inner (FP32) CG operator
 *                                       kernel on the problem's FP32 vectors, stop
 *                                       flag cleared; for timing after cg_mixed
 *   "cg_mixed"  handle, b, x, tol, max_outer, inner_tol, inner_maxit, gprec,
 *               OUT inner_iters, OUT outer_iters, OUT rel_res, [hist_outer]
 *               Mixed-precision iterative refinement: from x = 0 the FP64
 *               residual r = b - A x is recomputed after each inner CG solve
 *               of A d = r run in FP32 (FP32 vectors and arithmetic, G in FP32
 *               or BF16; dot products summed per thread and per block in FP32
 *               and across blocks in FP64; alpha and beta in FP64) until its residual
 *               fell by max(inner_tol, 0.5 tol/||r||) (relative), and x += d
 *               in FP64; stops when ||b - A x||_c/||b||_c <= tol or after
 *               max_outer corrections.  rel_res is that true residual;
 *               hist_outer (max_outer+1 doubles) its value before each step.
 *   "cg_ax"     handle                  one launch of the CG iteration's fused
 *                                       operator kernel on the problem's own CG
 *                                       vectors (p = r + beta p, w = A_local p,
 *                                       <p, w>), with the stop flag cleared; for
 *                                       timing after a cg_solve (changes p)
 *   "wait_probe" limit_ns (1e3 .. 1e8), OUT copied
 *               Self-test of failure detection: a one-block kernel copies 64
 *               bytes with the TMA engine (waited for on its own mbarrier),
 *               then runs the operator kernels' bounded mbarrier wait on a
 *               barrier whose byte count is never supplied; the wait gives up
 *               after ~limit_ns and sets the device status word.  copied
 *               receives the last copied value (7.5) when the copy landed and
 *               the wait ran out (-1 otherwise).  The next sem_sync or solve
 *               returns SEM_ETIMEDOUT (the message names the wait) and clears
 *               the word; nothing is left in flight and later calls work.
 *   "peak_fma"  dtype (0 f64, 1 f32), iters, OUT flops_per_s
 *               measured FMA issue rate of the FP64 or FP32 pipe (device fact
 *               for the ALU roofline; not part of the method)
 *   Operator tuner.  The local operator exists in several variants, all
 *   computing the same map: 0 "columns" (one thread per (i, j) column of an
 *   element, FP64), 1 "lines" (whole r, s and t lines per thread with the
 *   even-odd split of D; elements per block epb chosen at launch), 2
 *   "persistent" (TMA-pipelined columns, FP32 only), 3 "lines" with the
 *   geometric factors loaded into registers ahead of use (BF16 factors only),
 *   4 "lines" with the factors copied into shared memory with the slab
 *   (FP32), 5 "lines" of the FP64 operator evaluated in double-word FP32
 *   arithmetic (pairs of FP32 numbers, ~48 significant bits; FP64 inputs,
 *   outputs and CG recurrences; FP64 only; its factors, a second 48-byte
 *   per node copy of G, are made on first use).  The variant in use is
 *   kept per kind (0 FP64, 1 FP32 with FP32 G, 2 FP32 with BF16 G) and per N;
 *   the paper's runtime specialises kernels on N and its scripts pick the
 *   thread layout (Section VIII-B); here the choice is made by timing.
 *   Changing it makes every captured CG graph be captured again.
 *   "autotune"  handle, kind, reps, cand (HOST double[3 cap] or NONE), cap,
 *               OUT n_cand
 *               Runs each candidate of `kind` at the problem's N as the CG
 *               operator (reps timed launches after 2 warm-ups, on the
 *               problem's own CG vectors, which it overwrites) and keeps the
 *               fastest.  cand receives (variant, epb, microseconds per
 *               launch) per candidate, n_cand their number (<= 24).
 *   "autotune_get" kind, N, OUT variant, OUT epb, OUT us
 *   "autotune_set" kind, N, variant, epb      SEM_EARG if the variant does
 *               not exist for the kind or epb does not fit a block
 *   "autotune_save" path (HOST NUL-terminated)  writes the table as text:
 *               lines "kind N variant epb us", '#' comments
 *   "autotune_load" path (HOST NUL-terminated)  reads such a file (all
 *               entries checked before any is used; SEM_EARG on a bad line)
 *   "batch"     n, handles (HOST int64[n]), OUT batch
 *               Group n problems (made with "mesh", any sizes and orders) for
 *               batched solves.  Their local vectors are concatenated in the
 *               given order (problem k at offset nL_0 + ... + nL_{k-1}).
 *   "batch_info" batch, OUT n, OUT nL_total
 *   "batch_solve" batch, b_all, x_all, tol, maxit, mode, inner_tol, max_outer,
 *               OUT total_iters, OUT max_rel_res, [iters HOST int64[n]],
 *               [rel_res HOST double[n]]
 *               Solve every problem of the batch at once: per order present,
 *               each CG phase is one persistent launch over that order's
 *               problems (dynamic work list), the orders' iterations parallel
 *               chains of one CUDA graph.  mode 0: FP64 CG to tol;
 *               mode 1 / 2: mixed-precision refinement (as "cg_mixed") with G
 *               in BF16 / FP32.  A problem's iterates do not depend on the
 *               other problems in the batch.  iters: CG iterations (mode 0) or
 *               inner iterations (modes 1, 2); rel_res: recursive (mode 0) or
 *               true (modes 1, 2) relative residual at exit.
 *   "batch_free" batch
 *   "serve_open" capacity, budget_gb, mode, tol, inner_tol, K, maxit, OUT server
 *               A solve server with continuous batching: at most `capacity`
 *               solves active at once, their device memory within budget_gb;
 *               mode as in batch_solve; K CG iterations per round.
 *   "serve_submit" server, nx, ny, nz, N, verts (HOST double[(nx+1)(ny+1)(nz+1)*3]),
 *               b (HOST double[nL]), assemble, arrival_s, OUT ticket
 *               Queue a request (copied; no device work).  assemble = 0: b is
 *               the right-hand side; 1: b is a nodal source f and the server
 *               forms mask(QQ^T f) on admission.  arrival_s is the arrival
 *               time on the server clock ("serve_now"), from which the latency
 *               is measured.
 *   "serve_step" server, OUT n_queued, OUT n_active, OUT n_completed
 *               Wait for the round the previous step launched and retire the
 *               solves that finished in it (result kept on the device until
 *               fetched); let the requests admitted meanwhile join; launch
 *               the next round of every active solve (requests that joined
 *               start, running ones continue) and admit queued requests in
 *               arrival order within the limits while it runs.  Returns with
 *               that round running, so the caller's submissions and fetches
 *               overlap it; a solve is reported complete by the step after
 *               the round in which it finished.
 *   "serve_result" server, ticket, [x: HOST or device double[nL]], OUT state,
 *               OUT iters, OUT rel_res, OUT latency_ms
 *               state 0 queued, 1 active, 2 done, 3 failed; when done, x
 *               receives the solution and the request is released; when
 *               failed (its problem could not be built, e.g. SEM_EMESH for an
 *               inverted element), iters holds the error code, rel_res is NaN,
 *               x is untouched and the request is released.  A failed request
 *               is drained like a finished one and never stops the others.
 *               A finished result's device memory counts against the HBM
 *               budget until it is fetched.
 *   "serve_now" server, OUT seconds       the server clock
 *   "serve_drain" server, tickets (HOST int64[cap]), cap, OUT n
 *               tickets completed since the last drain (at most cap)
 *   "serve_close" server
 *   One problem split across ranks (processes) by whole element layers
 *   along z (Nekbone's element decomposition under MPI, Section VIII-A):
 *   "dist_mesh" nx, ny, nz, N, verts (device double[(nx+1)(ny+1)(nz+1)*3]),
 *               neighbours, OUT handle
 *               This rank's slab: an nx x ny x nz box of elements whose
 *               vertex planes are those of the global mesh; neighbours bit 0:
 *               a rank holds the layers below (the z0 face is an interface,
 *               not Dirichlet), bit 1: above (z1 face).  The other faces are
 *               Dirichlet.  Weights use the global multiplicities.
 *   "dist_info" handle, OUT nL
 *   "dist_ax"   handle, x, y (device double[nL])   y = A_local x on the slab
 *   "dist_gs"   handle, u (device double[nL]), comm (HOST sem_comm)
 *               u <- mask(QQ^T u) of the whole problem: the slab's sum, one
 *               exchange of the interface-plane partial sums with each
 *               neighbour (lower rank's partial added first, so both hold the
 *               same bits), the global Dirichlet mask
 *   "dist_dot"  handle, u, v, comm, OUT double   the global weighted dot
 *   "dist_cg_solve" handle, b, x (device double[nL]), tol, maxit, comm,
 *               hist (HOST double[maxit+1] or NONE), OUT iters, OUT rel_res
 *               CG of the whole problem, each rank on its slab: the
 *               operator kernel of cg_solve, the distributed sum above, two
 *               scalar allreduces per iteration (<p, A p>, <r, r>); b and x
 *               hold this slab's local nodes; hist[k] = sqrt(<r_k, r_k>)
 *   "dist_free" handle
 * Unknown names return SEM_EKERNEL; wrong argument counts or kinds SEM_EARG. */
int sem_run(const char *kernel, int nargs, const sem_arg *args);

/* Host barrier on the library stream (Section IV, "sync").  Returns
 * SEM_ETIMEDOUT if a kernel reported a bounded wait that gave up, SEM_ECUDA
 * on an asynchronous CUDA error. */
int sem_sync(void);

/* Release every mirror, problem, graph and the stream (Section IV,
 * "finalize").  Later calls other than sem_init return SEM_EINIT. */
int sem_finalize(void);

/* Message for the most recent failing call (static storage, never NULL). */
const char *sem_last_error(void);

/* Install device allocator hooks (before or after sem_init; affects later
 * allocations).  Passing NULL for both restores cudaMalloc/cudaFree. */
int sem_set_allocator(sem_alloc_fn alloc_fn, sem_free_fn free_fn, void *ctx);

/* Use `stream` (a cudaStream_t) for all later work.  NULL restores the
 * library's own non-blocking stream.  Requires sem_init. */
int sem_set_stream(void *stream);

/* Number of kernels the library has launched since sem_init (each kernel in
 * a replayed CUDA graph counts once per replay). */
int64_t sem_launch_count(void);

/* Weighted dot product that allocates nothing on the device.  The paper has
 * no counterpart; this is a service for callers that cannot allocate device
 * memory: code running while a CUDA graph is captured in a mode that forbids
 * allocation, real-time loops that must not enter an allocator after
 * start-up, and programs whose device memory belongs to another framework's
 * allocator with no hook libsem could use.  The regular "dot" kernel needs a
 * partials buffer that libsem allocates; this variant keeps its scratch (the
 * per-block partial sums and a ticket counter) in a static device array of
 * 64 KB that every GPU loading libsem holds until the process exits.
 *   c, u, v  device arrays of n doubles (c may be NULL: all weights 1)
 *   n        number of entries, 0 <= n <= 16,777,216 (SEM_ERANGE above:
 *            the static array holds one partial per 2048 entries)
 *   out      device double receiving sum_l c_l u_l v_l
 *   stream   cudaStream_t to run on (NULL: the legacy default stream)
 * Arrays must be 8-byte aligned (SEM_EARG otherwise).  Needs no sem_init and
 * does not synchronise: *out is valid once `stream` has reached the end of
 * the call's work.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress, with that device current), which may
 * load the library's device code; make that first call before any stream
 * capture.  All calls share the array and it keeps the last call's contents;
 * the ticket counter is cleared at the start of each call.  Calls whose work
 * overlaps on the GPU (e.g. on two unordered streams) race on the array. */
int sem_dot_noalloc(const double *c, const double *u, const double *v, int64_t n, double *out,
                    void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SEM_H */
