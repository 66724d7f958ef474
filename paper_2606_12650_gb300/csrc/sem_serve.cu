// sem_serve.cu -- a solve server with continuous batching.
//
// Requests (a box mesh and a right-hand side) are queued on the host as they
// arrive.  Each step of the server (1) adds the requests admitted during the
// previous step to the active set and, if the set changed, hands the new
// membership to the batch engine, where joining problems start and running
// ones keep their state; (2) launches one round of the batch engine (K CG
// iterations of every active solve in persistent launches, plus refinement
// for mixed precision) without waiting for it; (3) while the round runs,
// admits queued requests in arrival order, within the server's slot and HBM
// limits, on a stream of its own -- admission builds each problem on the
// device (geometry, mixed-precision factors, right-hand side), so its host
// work, allocations and copies overlap the round instead of idling the GPU;
// (4) waits for the round and retires the solves that finished: the solution
// is copied to a compact device buffer, kept there until the client fetches
// it, and the problem's memory is freed.
// Latency is measured from the request's arrival time to the end of the round
// in which it finished, on the server's steady clock.  A request's result
// does not depend on which other requests shared its rounds.  A request whose
// problem cannot be built (an inverted element: SEM_EMESH) fails alone: it
// leaves the queue with state 3 and its error code, and the others go on.
#include <cuda_runtime.h>

#include <chrono>
#include <algorithm>
#include <deque>
#include <limits>
#include <map>
#include <vector>

#include "sem_box.cuh"
#include "sem_internal.h"

namespace sem {

struct ServeReq {
    int64_t ticket = 0;
    int nx = 0, ny = 0, nz = 0, N = 0;
    int64_t nL = 0;
    std::vector<double> verts, b;     // host copies until admission
    double arrival = 0.0;             // seconds on the server clock
    bool assemble = false;            // b holds a nodal source f: form mask(QQ^T f) on admission
    Problem *P = nullptr;
    DevArena *arena = nullptr;        // the request's device buffers, one allocation
    double *b_dev = nullptr;
    double *x_dev = nullptr;          // result, device-resident until fetched
    size_t bytes = 0;                 // device bytes held while active (and its result until fetched)
    bool fresh = false;               // admitted, not yet started by the batch engine
    int err = 0;                      // state 3: the error code of its failed admission
    int state = 0;                    // 0 queued, 1 active, 2 done, 3 failed
    double t_done = 0.0;
    int64_t iters = 0;
    double res = 0.0;
};

struct Server {
    Batch *B = nullptr;
    int mode = 0;
    int capacity = 0;
    size_t budget = 0;
    size_t in_use = 0;
    std::deque<ServeReq *> queue;
    std::vector<ServeReq *> active;
    std::vector<ServeReq *> pending;  // admitted during the running round; join at the next step
    std::vector<double *> pending_tmp;  // admission temporaries, freed once the admission stream is idle
    cudaStream_t adm = nullptr;       // admission work (overlaps the rounds on the library stream)
    std::map<int64_t, ServeReq *> reqs;
    std::vector<int64_t> finished;    // tickets completed since the last drain
    int64_t next_ticket = 1;
    int64_t completed = 0;
    bool changed = false;
    bool in_flight = false;           // a round launched by the last step is running
    std::chrono::steady_clock::time_point t0;
};

double serve_now(const Server *S) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - S->t0).count();
}

// Device bytes a request holds from admission until its result is fetched,
// from the node count: FP64 geometry (48), mass (8), CG vectors (32),
// right-hand side (8) and the retired result (8) per node, plus for FP64 the
// double-word copy of the factors (48; counted whichever operator body the
// tuner picked), for mixed precision BF16/FP32 factors (12 or 24) and FP32
// inner vectors (16); and per problem its reduction partials, two CG states
// and the vertex copy, plus 64 KB of allocation granularity.
static size_t request_bytes(int mode, int nx, int ny, int nz, int64_t nL) {
    size_t per = 48 + 8 + 32 + 8 + 8;
    if (mode == 0) per += 48;   // the double-word copy of G (FP64 batches' double-word body)
    if (mode == 1) per += 12 + 16;
    if (mode == 2) per += 24 + 16;
    const int64_t n_verts = int64_t(nx + 1) * (ny + 1) * (nz + 1);
    return size_t(nL) * per + partials_bytes(partials_cap(int64_t(nx) * ny * nz)) + 2 * sizeof(CgState) +
           size_t(n_verts) * 3 * sizeof(double) + (size_t(1) << 16);
}
static size_t request_bytes(int mode, const ServeReq *q) { return request_bytes(mode, q->nx, q->ny, q->nz, q->nL); }

int serve_open(int capacity, double budget_gb, int mode, double tol, double inner_tol, int K, int maxit,
               Server **out) {
    *out = nullptr;
    if (capacity < 1 || capacity > (1 << 16)) return set_error(SEM_EARG, "serve_open: capacity must be in [1, 65536]");
    if (mode < 0 || mode > 2) return set_error(SEM_EARG, "serve_open: mode must be 0, 1 or 2");
    if (K < 1 || K > 4096) return set_error(SEM_EARG, "serve_open: K must be in [1, 4096]");
    if (!(budget_gb > 0.0)) return set_error(SEM_EARG, "serve_open: the HBM budget must be positive");
    // the admission stream has the highest priority: its small kernels take
    // SMs as soon as the persistent kernels of a round free any
    int least = 0, greatest = 0;
    cudaStream_t adm = nullptr;
    int rc = cuda_check(cudaDeviceGetStreamPriorityRange(&least, &greatest), "serve_open: priorities");
    if (rc == SEM_OK)
        rc = cuda_check(cudaStreamCreateWithPriority(&adm, cudaStreamNonBlocking, greatest), "serve_open: stream");
    if (rc != SEM_OK) return rc;
    Server *S = new Server();
    S->adm = adm;
    S->B = batch_new(mode, tol, maxit, inner_tol, 50, K);
    S->mode = mode;
    S->capacity = capacity;
    S->budget = size_t(budget_gb * 1e9);
    S->t0 = std::chrono::steady_clock::now();
    *out = S;
    return SEM_OK;
}

int serve_submit(Server *S, int nx, int ny, int nz, int N, const double *verts, const double *b, bool assemble,
                 double arrival, int64_t *ticket) {
    if (nx < 1 || ny < 1 || nz < 1 || nx > 4096 || ny > 4096 || nz > 4096)
        return set_error(SEM_EARG, "serve_submit: nx, ny, nz must be in [1, 4096]");
    if (N < 1 || N > kMaxQ - 1) return set_error(SEM_EARG, "serve_submit: N must be in [1, 9]");
    const int64_t nL = int64_t(nx) * ny * nz * (N + 1) * (N + 1) * (N + 1);
    if (nL >= (int64_t(1) << 31) - 1) return set_error(SEM_ERANGE, "serve_submit: problem too large");
    if (request_bytes(S->mode, nx, ny, nz, nL) > S->budget)
        return set_error(SEM_ENOMEM, "serve_submit: the request alone exceeds the server's HBM budget");
    ServeReq *q = new ServeReq();
    q->ticket = S->next_ticket++;
    q->nx = nx; q->ny = ny; q->nz = nz; q->N = N;
    q->nL = nL;
    const size_t nv = size_t(nx + 1) * (ny + 1) * (nz + 1) * 3;
    q->verts.assign(verts, verts + nv);
    q->b.assign(b, b + nL);
    q->arrival = arrival;
    q->assemble = assemble;
    S->queue.push_back(q);
    S->reqs[q->ticket] = q;
    *ticket = q->ticket;
    return SEM_OK;
}

template <int NQ>
static int assemble_nq(const Problem *P, const double *f, double *b) {
    assemble_box_kernel<NQ><<<unsigned((P->nL + 255) / 256), 256, 0, stream()>>>(f, b, int(P->nL), P->nx, P->ny,
                                                                               P->nz);
    count_launches(1);
    return cuda_check(cudaGetLastError(), "assemble_box_kernel");
}

static int assemble_rhs(const Problem *P, const double *f, double *b) {
    switch (P->nq) {
        case 2: return assemble_nq<2>(P, f, b);
        case 3: return assemble_nq<3>(P, f, b);
        case 4: return assemble_nq<4>(P, f, b);
        case 5: return assemble_nq<5>(P, f, b);
        case 6: return assemble_nq<6>(P, f, b);
        case 7: return assemble_nq<7>(P, f, b);
        case 8: return assemble_nq<8>(P, f, b);
        case 9: return assemble_nq<9>(P, f, b);
        case 10: return assemble_nq<10>(P, f, b);
        default: return set_error(SEM_EARG, "serve: unsupported order");
    }
}

static void release_active(ServeReq *q) {
    if (q->P) problem_destroy(q->P);
    if (q->b_dev) dev_free(q->b_dev);
    arena_release(q->arena);
    q->P = nullptr;
    q->b_dev = nullptr;
    q->arena = nullptr;
}

static int admit(Server *S, ServeReq *q) {
    // one allocation for every buffer of the request (problem, factors,
    // vectors, right-hand side, set-up temporaries), carved by dev_alloc
    const size_t tmp = sizeof(double) * (q->verts.size() + (q->assemble ? size_t(q->nL) : 0)) + 4096;
    q->arena = arena_new(request_bytes(S->mode, q) + tmp);
    if (!q->arena) return SEM_ENOMEM;
    ArenaScope carve(q->arena);
    double *vdev = static_cast<double *>(dev_alloc(sizeof(double) * q->verts.size()));
    if (!vdev) {
        arena_release(q->arena);
        q->arena = nullptr;
        return SEM_ENOMEM;
    }
    int rc = cuda_check(cudaMemcpyAsync(vdev, q->verts.data(), sizeof(double) * q->verts.size(),
                                        cudaMemcpyHostToDevice, stream()), "serve: vertices");
    // deferred set-up: nothing here waits for the admission stream; the mesh
    // check and the temporaries' release follow its synchronisation
    if (rc == SEM_OK) rc = problem_create(q->nx, q->ny, q->nz, q->N, vdev, &q->P, true);
    if (rc == SEM_OK && S->mode != 0) rc = mixed_prepare(q->P, S->mode == 1 ? kGBF16 : kGF32);
    if (rc == SEM_OK) {
        q->b_dev = static_cast<double *>(dev_alloc(sizeof(double) * q->nL));
        if (!q->b_dev) rc = SEM_ENOMEM;
    }
    double *f_dev = nullptr;
    if (rc == SEM_OK && q->assemble) {
        f_dev = static_cast<double *>(dev_alloc(sizeof(double) * q->nL));
        if (!f_dev) rc = SEM_ENOMEM;
    }
    if (rc == SEM_OK)
        rc = cuda_check(cudaMemcpyAsync(q->assemble ? f_dev : q->b_dev, q->b.data(), sizeof(double) * q->nL,
                                        cudaMemcpyHostToDevice, stream()), "serve: right-hand side");
    if (rc == SEM_OK && q->assemble) rc = assemble_rhs(q->P, f_dev, q->b_dev);
    if (rc != SEM_OK) {
        // nothing of the request may still be in flight when its arena goes
        cudaStreamSynchronize(stream());
        release_active(q);
        return rc;
    }
    // no wait here: the set-up temporaries are released, and the request
    // joins the batch, after the admission stream is synchronised (next step)
    S->pending_tmp.push_back(vdev);
    if (f_dev) S->pending_tmp.push_back(f_dev);
    // the host copies above come from q->b / q->verts: pageable memory that
    // cudaMemcpyAsync has consumed by the time it returns
    std::vector<double>().swap(q->verts);
    std::vector<double>().swap(q->b);
    q->state = 1;
    q->fresh = true;
    q->bytes = request_bytes(S->mode, q);
    S->in_use += q->bytes;
    return SEM_OK;
}

// Admission in arrival order, within the slot and HBM limits, on the
// server's admission stream; admitted requests wait in `pending`.  Returns
// the first error that is not the request's own.
static int admit_queued(Server *S) {
    StreamScope scope(S->adm);
    while (!S->queue.empty() && int(S->active.size() + S->pending.size()) < S->capacity) {
        ServeReq *q = S->queue.front();
        if (S->in_use + request_bytes(S->mode, q) > S->budget) break;
        const int rc = admit(S, q);
        if (rc == SEM_ENOMEM && !(S->active.empty() && S->pending.empty())) break;   // retry once memory frees up
        if (rc == SEM_EMESH || rc == SEM_EARG || rc == SEM_ENOMEM) {
            // the request itself cannot be served: it fails alone
            S->queue.pop_front();
            std::vector<double>().swap(q->verts);
            std::vector<double>().swap(q->b);
            q->state = 3;
            q->err = rc;
            q->t_done = serve_now(S);
            ++S->completed;
            S->finished.push_back(q->ticket);
            continue;
        }
        if (rc != SEM_OK) return rc;
        S->queue.pop_front();
        S->pending.push_back(q);
    }
    return SEM_OK;
}

// Retire the members that finished in the round just completed: results to
// compact device buffers, problem memory released.
static int retire(Server *S, const std::vector<int> &done) {
    if (done.empty()) return SEM_OK;
    const double t = serve_now(S);
    // results of the finished members only
    std::vector<int64_t> its(done.size());
    std::vector<double> res(done.size());
    int rc = batch_results_of(S->B, done, its.data(), res.data());
    if (rc != SEM_OK) return rc;
    std::vector<uint8_t> gone(S->active.size(), 0);
    for (size_t j = 0; j < done.size(); ++j) {
        const int k = done[j];
        ServeReq *q = S->active[k];
        q->x_dev = static_cast<double *>(dev_alloc(sizeof(double) * q->nL));
        if (!q->x_dev) return SEM_ENOMEM;
        rc = cuda_check(cudaMemcpyAsync(q->x_dev, q->P->x, sizeof(double) * q->nL, cudaMemcpyDeviceToDevice,
                                        stream()), "serve: result");
        if (rc != SEM_OK) return rc;
        q->iters = its[j];
        q->res = res[j];
        q->t_done = t;
        gone[k] = 1;
    }
    rc = cuda_check(cudaStreamSynchronize(stream()), "serve: sync");
    if (rc != SEM_OK) return rc;
    std::vector<ServeReq *> keep;
    for (size_t k = 0; k < S->active.size(); ++k) {
        ServeReq *q = S->active[k];
        if (gone[k]) {
            release_active(q);   // q->bytes stay counted until the result is fetched
            q->state = 2;
            ++S->completed;
            S->finished.push_back(q->ticket);
        } else {
            keep.push_back(q);
        }
    }
    S->active.swap(keep);
    S->changed = true;
    return SEM_OK;
}

// One step.  The step returns with the next round running, so that the
// caller's own work (submitting, fetching results) overlaps it:
// (1) wait for the round the previous step launched and retire the solves
//     that finished in it;
// (2) requests admitted meanwhile join (with nothing running, admission runs
//     here first);
// (3) the membership goes to the batch engine;
// (4) the next round is launched, and queued requests are admitted on the
//     admission stream while it runs.
int serve_step(Server *S, int64_t *n_queued, int64_t *n_active, int64_t *n_completed) {
    int rc = SEM_OK;
    if (S->in_flight) {
        std::vector<int> done;
        S->in_flight = false;
        rc = batch_round_finish(S->B, &done);
        if (rc == SEM_OK) rc = retire(S, done);
        if (rc != SEM_OK) return rc;
    }
    if (S->active.empty() && S->pending.empty()) {
        rc = admit_queued(S);
        if (rc != SEM_OK) return rc;
    }
    if (!S->pending.empty() || !S->pending_tmp.empty()) {
        rc = cuda_check(cudaStreamSynchronize(S->adm), "serve: admission sync");
        if (rc != SEM_OK) return rc;
        for (double *t : S->pending_tmp) dev_free(t);
        S->pending_tmp.clear();
        for (ServeReq *q : S->pending) {
            const int mrc = problem_check_mesh(q->P);
            if (mrc != SEM_OK) {   // an inverted element: this request fails alone
                release_active(q);
                S->in_use -= q->bytes;
                q->state = 3;
                q->err = mrc;
                q->t_done = serve_now(S);
                ++S->completed;
                S->finished.push_back(q->ticket);
                continue;
            }
            S->active.push_back(q);
        }
        S->pending.clear();
        S->changed = true;
    }
    // hand the membership to the batch engine; requests admitted since the
    // last successful hand-over start, the others keep their state
    if (S->changed) {
        std::vector<Problem *> ps;
        std::vector<const double *> bs;
        std::vector<uint8_t> start;
        for (ServeReq *q : S->active) {
            ps.push_back(q->P);
            bs.push_back(q->b_dev);
            start.push_back(q->fresh ? 1 : 0);
        }
        rc = batch_set(S->B, ps.data(), bs.data(), start.data(), int(ps.size()));
        if (rc != SEM_OK) return rc;
        for (ServeReq *q : S->active) q->fresh = false;
        S->changed = false;
    }
    if (!S->active.empty()) {
        rc = batch_round_launch(S->B);
        if (rc != SEM_OK) return rc;
        S->in_flight = true;
    }
    rc = admit_queued(S);
    if (rc != SEM_OK) return rc;
    *n_queued = int64_t(S->queue.size());
    *n_active = int64_t(S->active.size() + S->pending.size());
    *n_completed = S->completed;
    return SEM_OK;
}

// state: 0 queued, 1 active, 2 done (x written, request released), 3 failed
// (iters = its error code, rel_res = NaN; request released).
int serve_result(Server *S, int64_t ticket, double *x_out, bool x_on_device, int64_t *state, int64_t *iters,
                 double *rel_res, double *latency_ms) {
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return set_error(SEM_EHANDLE, "serve_result: unknown ticket");
    ServeReq *q = it->second;
    *state = q->state;
    if (q->state == 3) {
        *iters = q->err;
        *rel_res = std::numeric_limits<double>::quiet_NaN();
        *latency_ms = 1e3 * (q->t_done - q->arrival);
        S->reqs.erase(it);
        delete q;
        return SEM_OK;
    }
    if (q->state != 2) return SEM_OK;
    if (x_out) {
        const int rc = cuda_check(cudaMemcpyAsync(x_out, q->x_dev, sizeof(double) * q->nL,
                                                  x_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                                  stream()), "serve_result: copy");
        if (rc != SEM_OK) return rc;
        const int rs = cuda_check(cudaStreamSynchronize(stream()), "serve_result: sync");
        if (rs != SEM_OK) return rs;
    }
    *iters = q->iters;
    *rel_res = q->res;
    *latency_ms = 1e3 * (q->t_done - q->arrival);
    dev_free(q->x_dev);
    S->in_use -= q->bytes;
    S->reqs.erase(it);
    delete q;
    return SEM_OK;
}

// Tickets completed since the last drain (up to cap of them).
int64_t serve_drain(Server *S, int64_t *out, int64_t cap) {
    const int64_t n = std::min<int64_t>(cap, int64_t(S->finished.size()));
    for (int64_t k = 0; k < n; ++k) out[k] = S->finished[size_t(k)];
    S->finished.erase(S->finished.begin(), S->finished.begin() + n);
    return n;
}

int64_t serve_nodes_of(const Server *S, int64_t ticket) {
    auto it = S->reqs.find(ticket);
    return it == S->reqs.end() ? -1 : it->second->nL;
}

void serve_close(Server *S) {
    if (!S) return;
    cudaStreamSynchronize(stream());
    if (S->adm) {
        cudaStreamSynchronize(S->adm);
        for (double *t : S->pending_tmp) dev_free(t);
        cudaStreamDestroy(S->adm);
    }
    for (auto &kv : S->reqs) {
        ServeReq *q = kv.second;
        release_active(q);
        if (q->x_dev) dev_free(q->x_dev);
        delete q;
    }
    batch_destroy(S->B);
    delete S;
}

}  // namespace sem
