// sem_api.cu -- the C-ABI of libsem: runtime context, device allocator
// hooks, host-array mirrors, argument marshalling and the named-kernel
// dispatch.  The call shapes follow the runtime interface the paper's
// pragmas lower to (init / update / run / sync / finalize, Sections IV-V).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "sem.h"
#include "sem_internal.h"

namespace sem {
namespace {

struct Mirror {
    uintptr_t host_base;   // key: host base pointer
    size_t start, end, elem;
    void *dev;             // device copy of host[start, end)
};

struct Context {
    bool up = false;
    int device = 0;
    int verbose = 0;
    size_t budget = 0;                 // 0: unlimited
    size_t in_use = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t cur_stream = nullptr;
    sem_alloc_fn alloc_fn = nullptr;
    sem_free_fn free_fn = nullptr;
    void *alloc_ctx = nullptr;
    std::map<void *, size_t> sizes;    // device pointer -> bytes
    std::map<uintptr_t, Mirror> mirrors;
    std::map<int64_t, Problem *> problems;
    std::map<int64_t, Batch *> batches;
    std::map<int64_t, Server *> servers;
    std::map<int64_t, DistProblem *> dists;
    int64_t next_handle = 1;
    int32_t *status_dev = nullptr;
    int32_t *status_pinned = nullptr;
    cudaDeviceProp prop{};
};

Context g;
std::atomic<int64_t> g_launches{0};
thread_local char g_err[1024] = "no error";

}  // namespace

int set_error(int code, const std::string &msg) {
    snprintf(g_err, sizeof g_err, "%s", msg.c_str());
    return code;
}

int cuda_check(cudaError_t err, const char *what) {
    if (err == cudaSuccess) return SEM_OK;
    char buf[512];
    snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorString(err), cudaGetErrorName(err));
    if (err == cudaErrorMemoryAllocation) return set_error(SEM_ENOMEM, buf);
    return set_error(SEM_ECUDA, buf);
}

// Device arenas: one allocation from which a group of buffers that live and
// die together is carved (a served request's problem: ~20 buffers, where each
// allocation through the allocator hook costs a call into the host runtime
// that owns the memory).  Inside an ArenaScope, dev_alloc carves 256-byte
// aligned pieces from the arena and falls back to a real allocation when it
// is full; dev_free of a carved piece does nothing -- arena_release frees the
// arena as a whole.
struct DevArena {
    unsigned char *base = nullptr;
    size_t cap = 0, used = 0;
    std::vector<void *> carved;
};
namespace {
thread_local DevArena *g_arena = nullptr;
std::map<void *, DevArena *> g_carved;
}  // namespace

DevArena *arena_new(size_t bytes) {
    void *p = dev_alloc(bytes);
    if (!p) return nullptr;
    DevArena *a = new DevArena();
    a->base = static_cast<unsigned char *>(p);
    a->cap = bytes;
    return a;
}

void arena_release(DevArena *a) {
    if (!a) return;
    for (void *p : a->carved) g_carved.erase(p);
    dev_free(a->base);
    delete a;
}

ArenaScope::ArenaScope(DevArena *a) : prev(g_arena) { g_arena = a; }
ArenaScope::~ArenaScope() { g_arena = prev; }

void *dev_alloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (g_arena) {
        const size_t need = (bytes + 255) / 256 * 256;
        if (g_arena->used + need <= g_arena->cap) {
            void *p = g_arena->base + g_arena->used;
            g_arena->used += need;
            g_arena->carved.push_back(p);
            g_carved[p] = g_arena;
            return p;
        }
    }
    if (g.budget && g.in_use + bytes > g.budget) {
        char buf[200];
        snprintf(buf, sizeof buf, "device allocation of %zu bytes exceeds the HBM budget (%zu of %zu in use)",
                 bytes, g.in_use, g.budget);
        set_error(SEM_ENOMEM, buf);
        return nullptr;
    }
    void *p = nullptr;
    if (g.alloc_fn) {
        p = g.alloc_fn(bytes, g.alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (!p) {
        char buf[128];
        snprintf(buf, sizeof buf, "device allocation of %zu bytes failed", bytes);
        set_error(SEM_ENOMEM, buf);
        return nullptr;
    }
    if (reinterpret_cast<uintptr_t>(p) & 255u) {
        set_error(SEM_ENOMEM, "allocator returned memory that is not 256-byte aligned");
        if (g.free_fn) g.free_fn(p, g.alloc_ctx); else cudaFree(p);
        return nullptr;
    }
    g.sizes[p] = bytes;
    g.in_use += bytes;
    return p;
}

void dev_free(void *p) {
    if (!p) return;
    if (g_carved.count(p)) return;   // released with its arena
    auto it = g.sizes.find(p);
    if (it != g.sizes.end()) {
        g.in_use -= it->second;
        g.sizes.erase(it);
    }
    if (g.free_fn) g.free_fn(p, g.alloc_ctx); else cudaFree(p);
}

// Pinned host slots for the small device-state mirrors that solves read back
// once per graph replay (one CgState each).  Taken from chunks of pinned
// memory kept for the life of the context: a solve server creates and frees
// problems continually, and cudaMallocHost / cudaFreeHost per problem cost
// milliseconds (the free waits for the device).
namespace {
constexpr size_t kPinnedSlot = 256;           // bytes per slot (>= sizeof(CgState), aligned)
constexpr size_t kPinnedChunkSlots = 1024;
std::vector<void *> g_pinned_chunks;
std::vector<void *> g_pinned_free;
}  // namespace

void *pinned_slot_alloc() {
    static_assert(sizeof(CgState) <= kPinnedSlot, "pinned slot too small");
    if (g_pinned_free.empty()) {
        void *chunk = nullptr;
        if (cudaMallocHost(&chunk, kPinnedSlot * kPinnedChunkSlots) != cudaSuccess) {
            cudaGetLastError();
            set_error(SEM_ENOMEM, "pinned host allocation failed");
            return nullptr;
        }
        g_pinned_chunks.push_back(chunk);
        for (size_t k = kPinnedChunkSlots; k-- > 0;)
            g_pinned_free.push_back(static_cast<unsigned char *>(chunk) + k * kPinnedSlot);
    }
    void *p = g_pinned_free.back();
    g_pinned_free.pop_back();
    return p;
}

void pinned_slot_free(void *p) {
    if (p) g_pinned_free.push_back(p);
}

static void pinned_release_all() {
    for (void *c : g_pinned_chunks) cudaFreeHost(c);
    g_pinned_chunks.clear();
    g_pinned_free.clear();
}

// Work a thread issues inside a StreamScope goes to that scope's stream (the
// server admits requests on its own stream while a batch round runs on the
// library stream).
thread_local cudaStream_t g_stream_override = nullptr;
cudaStream_t stream() { return g_stream_override ? g_stream_override : g.cur_stream; }
StreamScope::StreamScope(cudaStream_t s) : prev(g_stream_override) { g_stream_override = s; }
StreamScope::~StreamScope() { g_stream_override = prev; }
int sm_count() { return g.prop.multiProcessorCount > 0 ? g.prop.multiProcessorCount : 1; }
int32_t *status_word() { return g.status_dev; }
int32_t *status_host() { return g.status_pinned; }
void count_launches(int64_t n) { g_launches += n; }

int poll_status() {
    int rc = cuda_check(cudaMemcpyAsync(g.status_pinned, g.status_dev, sizeof(int32_t),
                                        cudaMemcpyDeviceToHost, g.cur_stream), "status read");
    if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(g.cur_stream), "status sync");
    if (rc != SEM_OK) return rc;
    if (*g.status_pinned != kStatusOk) {
        const int32_t code = *g.status_pinned;
        *g.status_pinned = 0;
        cudaMemsetAsync(g.status_dev, 0, sizeof(int32_t), g.cur_stream);
        cudaStreamSynchronize(g.cur_stream);
        char buf[192];
        snprintf(buf, sizeof buf,
                 "a bounded device wait gave up (status %d: %s)", code,
                 code == kStatusMbarTimeout ? "an mbarrier wait for a TMA copy into shared memory ran past its limit"
                                            : "unknown wait");
        return set_error(SEM_ETIMEDOUT, buf);
    }
    return SEM_OK;
}

namespace {

// ---------------------------------------------------------------- mirrors
Mirror *find_mirror_containing(uintptr_t addr, size_t bytes) {
    // mirrors are keyed by host base; the window is [base + start*elem, base + end*elem)
    for (auto &kv : g.mirrors) {
        Mirror &m = kv.second;
        const uintptr_t lo = m.host_base + m.start * m.elem, hi = m.host_base + m.end * m.elem;
        if (addr >= lo && addr + bytes <= hi) return &m;
    }
    return nullptr;
}

// ---------------------------------------------------------------- arguments
struct ArgReader {
    const char *kernel;
    int nargs;
    const sem_arg *args;
    int err = SEM_OK;

    bool need(int n) {
        if (nargs < n) {
            fail(SEM_EARG, "expects at least " + std::to_string(n) + " arguments");
            return false;
        }
        return true;
    }
    int fail(int code, const std::string &msg) {
        if (err == SEM_OK) err = set_error(code, std::string(kernel) + ": " + msg);
        return err;
    }
    int64_t i(int k, const char *name) {
        if (k >= nargs || args[k].kind != SEM_ARG_INT) {
            fail(SEM_EARG, std::string("argument ") + std::to_string(k) + " (" + name + ") must be SEM_ARG_INT");
            return 0;
        }
        return args[k].v.i;
    }
    double d(int k, const char *name) {
        if (k >= nargs || (args[k].kind != SEM_ARG_DOUBLE && args[k].kind != SEM_ARG_INT)) {
            fail(SEM_EARG, std::string("argument ") + std::to_string(k) + " (" + name + ") must be SEM_ARG_DOUBLE");
            return 0;
        }
        return args[k].kind == SEM_ARG_DOUBLE ? args[k].v.d : double(args[k].v.i);
    }
    // device address of an array argument holding `bytes` bytes
    void *arr(int k, size_t bytes, const char *name, bool optional = false) {
        if (k >= nargs || args[k].kind == SEM_ARG_NONE) {
            if (!optional)
                fail(SEM_EARG, std::string("array argument ") + std::to_string(k) + " (" + name + ") missing");
            return nullptr;
        }
        const sem_arg &a = args[k];
        void *dev = nullptr;
        if (a.kind == SEM_ARG_DEVICE) {
            dev = a.v.ptr;
        } else if (a.kind == SEM_ARG_MAPPED) {
            const uintptr_t h = reinterpret_cast<uintptr_t>(a.v.ptr);
            Mirror *m = find_mirror_containing(h, bytes);
            if (!m) {
                // distinguish "no mirror at all" from "range too small"
                for (auto &kv : g.mirrors) {
                    Mirror &mm = kv.second;
                    const uintptr_t lo = mm.host_base + mm.start * mm.elem, hi = mm.host_base + mm.end * mm.elem;
                    if (h >= lo && h < hi) {
                        fail(SEM_ERANGE, std::string(name) + ": mirror is smaller than the array the kernel needs");
                        return nullptr;
                    }
                }
                fail(SEM_ENOMAP, std::string(name) + ": host array has no device mirror");
                return nullptr;
            }
            dev = static_cast<unsigned char *>(m->dev) + (h - (m->host_base + m->start * m->elem));
        } else {
            fail(SEM_EARG, std::string("argument ") + std::to_string(k) + " (" + name + ") must be an array");
            return nullptr;
        }
        if (!dev || (reinterpret_cast<uintptr_t>(dev) & 15u)) {
            fail(SEM_EARG, std::string(name) + ": device array must be non-null and 16-byte aligned");
            return nullptr;
        }
        return dev;
    }
    void *host(int k, size_t bytes, const char *name, bool optional = false) {
        if (k >= nargs || args[k].kind == SEM_ARG_NONE) {
            if (!optional) fail(SEM_EARG, std::string("host array ") + name + " missing");
            return nullptr;
        }
        if (args[k].kind != SEM_ARG_HOST || (!args[k].v.ptr && bytes)) {
            fail(SEM_EARG, std::string("argument ") + std::to_string(k) + " (" + name + ") must be SEM_ARG_HOST");
            return nullptr;
        }
        return args[k].v.ptr;
    }
    void *out(int k, int kind, const char *name) {
        if (k >= nargs || args[k].kind != kind || !args[k].v.ptr) {
            fail(SEM_EARG, std::string("argument ") + std::to_string(k) + " (" + name + ") must be an OUT pointer");
            return nullptr;
        }
        return args[k].v.ptr;
    }
};

Problem *get_problem(ArgReader &R, int k, bool need_maps = true) {
    const int64_t h = R.i(k, "handle");
    if (R.err) return nullptr;
    auto it = g.problems.find(h);
    if (it == g.problems.end()) {
        R.fail(SEM_EHANDLE, "unknown problem handle " + std::to_string(h));
        return nullptr;
    }
    if (need_maps) {
        const int rc = problem_maps(it->second);
        if (rc != SEM_OK) {
            R.err = rc;
            return nullptr;
        }
    }
    return it->second;
}

int sync_stream(const char *what) { return cuda_check(cudaStreamSynchronize(g.cur_stream), what); }

// ---------------------------------------------------------------- named kernels
int run_mesh(ArgReader &R) {
    if (!R.need(6)) return R.err;
    const int64_t nx = R.i(0, "nx"), ny = R.i(1, "ny"), nz = R.i(2, "nz"), N = R.i(3, "N");
    if (R.err) return R.err;
    if (nx < 1 || ny < 1 || nz < 1 || nx > (1 << 20) || ny > (1 << 20) || nz > (1 << 20))
        return R.fail(SEM_EARG, "nx, ny, nz must be in [1, 2^20]");
    const size_t nv = size_t(nx + 1) * size_t(ny + 1) * size_t(nz + 1);
    const double *verts = static_cast<const double *>(R.arr(4, nv * 3 * sizeof(double), "verts"));
    int64_t *out = static_cast<int64_t *>(R.out(5, SEM_ARG_OUT_INT, "handle"));
    if (R.err) return R.err;
    Problem *P = nullptr;
    const int rc = problem_create(int(nx), int(ny), int(nz), int(N), verts, &P);
    if (rc != SEM_OK) return rc;
    const int64_t h = g.next_handle++;
    g.problems[h] = P;
    *out = h;
    if (g.verbose)
        fprintf(stderr, "[sem] mesh %lld: %dx%dx%d N=%d nL=%lld nG=%lld shared=%lld masked=%lld\n",
                (long long)h, P->nx, P->ny, P->nz, P->N, (long long)P->nL, (long long)P->nG,
                (long long)P->n_sh, (long long)P->n_mask);
    return SEM_OK;
}

int run_mesh_free(ArgReader &R) {
    if (!R.need(1)) return R.err;
    const int64_t h = R.i(0, "handle");
    if (R.err) return R.err;
    auto it = g.problems.find(h);
    if (it == g.problems.end()) return R.fail(SEM_EHANDLE, "unknown problem handle");
    if (!g.batches.empty()) return R.fail(SEM_EARG, "free the batches first (they hold their problems)");
    sync_stream("mesh_free");
    problem_destroy(it->second);
    g.problems.erase(it);
    return SEM_OK;
}

int run_info(ArgReader &R) {
    if (!R.need(5)) return R.err;
    Problem *P = get_problem(R, 0);
    int64_t *o1 = static_cast<int64_t *>(R.out(1, SEM_ARG_OUT_INT, "nL"));
    int64_t *o2 = static_cast<int64_t *>(R.out(2, SEM_ARG_OUT_INT, "nG"));
    int64_t *o3 = static_cast<int64_t *>(R.out(3, SEM_ARG_OUT_INT, "n_shared_ids"));
    int64_t *o4 = static_cast<int64_t *>(R.out(4, SEM_ARG_OUT_INT, "n_masked"));
    if (R.err) return R.err;
    *o1 = P->nL;
    *o2 = P->nG;
    *o3 = P->n_sh;
    *o4 = P->n_mask;
    return SEM_OK;
}

int run_ax(ArgReader &R, bool assembled) {
    if (!R.need(3)) return R.err;
    Problem *P = get_problem(R, 0);
    if (R.err) return R.err;
    const size_t vb = size_t(P->nL) * sizeof(double);
    const double *x = static_cast<const double *>(R.arr(1, vb, "x"));
    double *y = static_cast<double *>(R.arr(2, vb, "y"));
    if (R.err) return R.err;
    if (x == y) return R.fail(SEM_EARG, "x and y must not alias");
    int rc = launch_ax(P, x, y);
    if (rc == SEM_OK && assembled) rc = launch_gs(P, y);
    if (rc == SEM_OK && assembled) rc = launch_mask(P, y);
    return rc;
}

int run_inplace(ArgReader &R, int which) {
    if (!R.need(2)) return R.err;
    Problem *P = get_problem(R, 0);
    if (R.err) return R.err;
    double *u = static_cast<double *>(R.arr(1, size_t(P->nL) * sizeof(double), "u"));
    if (R.err) return R.err;
    return which == 0 ? launch_gs(P, u) : launch_mask(P, u);
}

int run_dot(ArgReader &R) {
    if (!R.need(4)) return R.err;
    Problem *P = get_problem(R, 0);
    if (R.err) return R.err;
    const size_t vb = size_t(P->nL) * sizeof(double);
    const double *u = static_cast<const double *>(R.arr(1, vb, "u"));
    const double *v = static_cast<const double *>(R.arr(2, vb, "v"));
    double *out = static_cast<double *>(R.out(3, SEM_ARG_OUT_DOUBLE, "result"));
    if (R.err) return R.err;
    int rc = launch_dot(P, u, v);
    if (rc != SEM_OK) return rc;
    double val = 0.0;
    rc = cuda_check(cudaMemcpyAsync(&P->st_host->dot_out, &P->st->dot_out, sizeof(double),
                                    cudaMemcpyDeviceToHost, g.cur_stream), "dot: read");
    if (rc == SEM_OK) rc = sync_stream("dot: sync");
    if (rc == SEM_OK) val = P->st_host->dot_out;
    *out = val;
    return rc;
}

int run_geom(ArgReader &R) {
    if (!R.need(3)) return R.err;
    Problem *P = get_problem(R, 0, false);
    if (R.err) return R.err;
    double *G = static_cast<double *>(R.arr(1, size_t(P->nL) * 6 * sizeof(double), "G"));
    double *B = static_cast<double *>(R.arr(2, size_t(P->nL) * sizeof(double), "B"));
    if (R.err) return R.err;
    int rc = cuda_check(cudaMemcpyAsync(G, P->G, size_t(P->nL) * 6 * sizeof(double), cudaMemcpyDeviceToDevice,
                                        g.cur_stream), "geom: copy G");
    if (rc == SEM_OK)
        rc = cuda_check(cudaMemcpyAsync(B, P->B, size_t(P->nL) * sizeof(double), cudaMemcpyDeviceToDevice,
                                        g.cur_stream), "geom: copy B");
    return rc;
}

int run_nodes(ArgReader &R) {
    if (!R.need(2)) return R.err;
    Problem *P = get_problem(R, 0, false);
    if (R.err) return R.err;
    double *X = static_cast<double *>(R.arr(1, size_t(P->nL) * 3 * sizeof(double), "X"));
    if (R.err) return R.err;
    return launch_nodes(P, nullptr, X);
}

int run_gs_map(ArgReader &R) {
    if (!R.need(3)) return R.err;
    Problem *P = get_problem(R, 0);
    if (R.err) return R.err;
    int32_t *ptr = static_cast<int32_t *>(R.arr(1, size_t(P->n_sh + 1) * sizeof(int32_t), "ptr"));
    int32_t *idx = static_cast<int32_t *>(R.arr(2, size_t(std::max<int64_t>(P->n_sh_copies, 1)) * sizeof(int32_t), "idx"));
    if (R.err) return R.err;
    int rc = cuda_check(cudaMemcpyAsync(ptr, P->sh_ptr, size_t(P->n_sh + 1) * sizeof(int32_t),
                                        cudaMemcpyDeviceToDevice, g.cur_stream), "gs_map: ptr");
    if (rc == SEM_OK && P->n_sh_copies)
        rc = cuda_check(cudaMemcpyAsync(idx, P->sh_idx, size_t(P->n_sh_copies) * sizeof(int32_t),
                                        cudaMemcpyDeviceToDevice, g.cur_stream), "gs_map: idx");
    return rc;
}

int run_rhs(ArgReader &R, bool sin_source) {
    Problem *P = nullptr;
    if (sin_source) {
        if (!R.need(2)) return R.err;
        P = get_problem(R, 0);
        if (R.err) return R.err;
        double *b = static_cast<double *>(R.arr(1, size_t(P->nL) * sizeof(double), "b"));
        if (R.err) return R.err;
        return launch_rhs_sin(P, nullptr, b);
    }
    if (!R.need(3)) return R.err;
    P = get_problem(R, 0);
    if (R.err) return R.err;
    const size_t vb = size_t(P->nL) * sizeof(double);
    const double *f = static_cast<const double *>(R.arr(1, vb, "f"));
    double *b = static_cast<double *>(R.arr(2, vb, "b"));
    if (R.err) return R.err;
    int rc = launch_scale(P, P->B, f, b);
    if (rc == SEM_OK) rc = launch_gs(P, b);
    if (rc == SEM_OK) rc = launch_mask(P, b);
    return rc;
}

int run_cg_solve(ArgReader &R) {
    if (!R.need(7)) return R.err;
    Problem *P = get_problem(R, 0);
    if (R.err) return R.err;
    const size_t vb = size_t(P->nL) * sizeof(double);
    const double *b = static_cast<const double *>(R.arr(1, vb, "b"));
    double *x = static_cast<double *>(R.arr(2, vb, "x"));
    const double tol = R.d(3, "tol");
    const int64_t maxit = R.i(4, "maxit");
    int64_t *oit = static_cast<int64_t *>(R.out(5, SEM_ARG_OUT_INT, "iters"));
    double *ores = static_cast<double *>(R.out(6, SEM_ARG_OUT_DOUBLE, "rel_res"));
    if (R.err) return R.err;
    if (maxit < 0 || maxit > (1 << 30)) return R.fail(SEM_EARG, "maxit must be in [0, 2^30]");
    double *hist = static_cast<double *>(R.arr(7, size_t(maxit + 1) * sizeof(double), "hist", true));
    if (R.err) return R.err;
    if (b == x) return R.fail(SEM_EARG, "b and x must not alias");
    return cg_solve(P, b, x, tol, int(maxit), hist, oit, ores);
}

int run_ax32(ArgReader &R) {
    if (!R.need(4)) return R.err;
    Problem *P = get_problem(R, 0, false);
    if (R.err) return R.err;
    const size_t vb = size_t(P->nL) * sizeof(float);
    const float *x = static_cast<const float *>(R.arr(1, vb, "x"));
    float *y = static_cast<float *>(R.arr(2, vb, "y"));
    const int64_t gprec = R.i(3, "gprec");
    if (R.err) return R.err;
    if (x == y) return R.fail(SEM_EARG, "x and y must not alias");
    const int rc = mixed_prepare(P, int(gprec));
    return rc != SEM_OK ? rc : launch_ax32(P, x, y, int(gprec));
}

int run_cg_ax32(ArgReader &R) {
    if (!R.need(2)) return R.err;
    Problem *P = get_problem(R, 0, false);
    const int64_t gprec = R.i(1, "gprec");
    if (R.err) return R.err;
    int rc = mixed_prepare(P, int(gprec));
    if (rc == SEM_OK)
        rc = cuda_check(cudaMemsetAsync(&P->st_in->done, 0, sizeof(int32_t), g.cur_stream), "cg_ax32: flag");
    return rc != SEM_OK ? rc : launch_ax32_cg(P, int(gprec));
}

// autotune(handle, kind, reps, cand HOST double[3 cap] | NONE, cap, OUT n_cand)
int run_autotune(ArgReader &R) {
    if (!R.need(6)) return R.err;
    Problem *P = get_problem(R, 0, false);
    const int64_t kind = R.i(1, "kind"), reps = R.i(2, "reps"), cap = R.i(4, "cap");
    if (R.err) return R.err;
    if (cap < 0 || cap > 64) return R.fail(SEM_EARG, "cap must be in [0, 64]");
    double *cand = static_cast<double *>(R.host(3, size_t(cap) * 3 * sizeof(double), "cand", true));
    int64_t *n_out = static_cast<int64_t *>(R.out(5, SEM_ARG_OUT_INT, "n_cand"));
    if (R.err) return R.err;
    int n = 0;
    TuneChoice best{};
    const int rc = tune_problem(P, int(kind), int(reps), cand, int(cap), &n, &best);
    if (rc == SEM_OK) *n_out = n;
    return rc;
}

// autotune_get(kind, N, OUT variant, OUT epb, OUT us)
int run_autotune_get(ArgReader &R) {
    if (!R.need(5)) return R.err;
    const int64_t kind = R.i(0, "kind"), N = R.i(1, "N");
    int64_t *ov = static_cast<int64_t *>(R.out(2, SEM_ARG_OUT_INT, "variant"));
    int64_t *oe = static_cast<int64_t *>(R.out(3, SEM_ARG_OUT_INT, "epb"));
    double *ou = static_cast<double *>(R.out(4, SEM_ARG_OUT_DOUBLE, "us"));
    if (R.err) return R.err;
    if (kind < 0 || kind >= kTuneKinds) return R.fail(SEM_EARG, "kind must be 0, 1 or 2");
    if (N < 1 || N > kMaxQ - 1) return R.fail(SEM_EARG, "N must be in [1, 9]");
    const TuneChoice c = tune_get(int(kind), int(N) + 1);
    *ov = c.variant;
    *oe = c.epb;
    *ou = c.us;
    return SEM_OK;
}

// autotune_set(kind, N, variant, epb)
int run_autotune_set(ArgReader &R) {
    if (!R.need(4)) return R.err;
    const int64_t kind = R.i(0, "kind"), N = R.i(1, "N"), variant = R.i(2, "variant"), epb = R.i(3, "epb");
    if (R.err) return R.err;
    const TuneChoice c{int(variant), int(epb), 0.0};
    const int rc = tune_check(int(kind), int(N) + 1, c);
    if (rc != SEM_OK) return rc;
    sync_stream("autotune_set");
    tune_set(int(kind), int(N) + 1, c);
    return SEM_OK;
}

// autotune_save(path HOST) / autotune_load(path HOST): NUL-terminated path
int run_autotune_file(ArgReader &R, bool save) {
    if (!R.need(1)) return R.err;
    const char *path = static_cast<const char *>(R.host(0, 1, "path"));
    if (R.err) return R.err;
    if (save) return tune_save(path);
    sync_stream("autotune_load");
    return tune_load(path);
}

int run_cg_mixed(ArgReader &R) {
    if (!R.need(11)) return R.err;
    Problem *P = get_problem(R, 0);
    if (R.err) return R.err;
    const size_t vb = size_t(P->nL) * sizeof(double);
    const double *b = static_cast<const double *>(R.arr(1, vb, "b"));
    double *x = static_cast<double *>(R.arr(2, vb, "x"));
    const double tol = R.d(3, "tol");
    const int64_t max_outer = R.i(4, "max_outer");
    const double inner_tol = R.d(5, "inner_tol");
    const int64_t inner_maxit = R.i(6, "inner_maxit");
    const int64_t gprec = R.i(7, "gprec");
    int64_t *o_in = static_cast<int64_t *>(R.out(8, SEM_ARG_OUT_INT, "inner_iters"));
    int64_t *o_out = static_cast<int64_t *>(R.out(9, SEM_ARG_OUT_INT, "outer_iters"));
    double *o_res = static_cast<double *>(R.out(10, SEM_ARG_OUT_DOUBLE, "rel_res"));
    if (R.err) return R.err;
    if (max_outer < 0 || max_outer > 1000 || inner_maxit < 1 || inner_maxit > (1 << 30))
        return R.fail(SEM_EARG, "max_outer must be in [0, 1000] and inner_maxit in [1, 2^30]");
    double *hist = static_cast<double *>(R.arr(11, size_t(max_outer + 1) * sizeof(double), "hist_outer", true));
    if (R.err) return R.err;
    if (b == x) return R.fail(SEM_EARG, "b and x must not alias");
    return mixed_solve(P, b, x, tol, int(max_outer), inner_tol, int(inner_maxit), int(gprec), o_in, o_out, o_res,
                       hist);
}

Batch *get_batch(ArgReader &R, int k) {
    const int64_t h = R.i(k, "batch");
    if (R.err) return nullptr;
    auto it = g.batches.find(h);
    if (it == g.batches.end()) {
        R.fail(SEM_EHANDLE, "unknown batch handle " + std::to_string(h));
        return nullptr;
    }
    return it->second;
}

int run_batch(ArgReader &R) {
    if (!R.need(3)) return R.err;
    const int64_t n = R.i(0, "n");
    if (R.err) return R.err;
    if (n < 1 || n > (1 << 20)) return R.fail(SEM_EARG, "n must be in [1, 2^20]");
    const int64_t *hs = static_cast<const int64_t *>(R.host(1, size_t(n) * 8, "handles"));
    int64_t *out = static_cast<int64_t *>(R.out(2, SEM_ARG_OUT_INT, "batch"));
    if (R.err) return R.err;
    std::vector<Problem *> ps;
    for (int64_t k = 0; k < n; ++k) {
        auto it = g.problems.find(hs[k]);
        if (it == g.problems.end()) return R.fail(SEM_EHANDLE, "unknown problem handle " + std::to_string(hs[k]));
        for (Problem *q : ps)
            if (q == it->second) return R.fail(SEM_EARG, "a problem appears twice in the batch");
        ps.push_back(it->second);
    }
    Batch *B = nullptr;
    const int rc = batch_create(ps.data(), int(n), &B);
    if (rc != SEM_OK) return rc;
    const int64_t h = g.next_handle++;
    g.batches[h] = B;
    *out = h;
    return SEM_OK;
}

int run_batch_info(ArgReader &R) {
    if (!R.need(3)) return R.err;
    Batch *B = get_batch(R, 0);
    int64_t *o1 = static_cast<int64_t *>(R.out(1, SEM_ARG_OUT_INT, "n"));
    int64_t *o2 = static_cast<int64_t *>(R.out(2, SEM_ARG_OUT_INT, "nL_total"));
    if (R.err) return R.err;
    *o1 = batch_size(B);
    *o2 = batch_total_nodes(B);
    return SEM_OK;
}

int run_batch_solve(ArgReader &R) {
    if (!R.need(10)) return R.err;
    Batch *B = get_batch(R, 0);
    if (R.err) return R.err;
    const size_t vb = size_t(batch_total_nodes(B)) * sizeof(double);
    const double *b = static_cast<const double *>(R.arr(1, vb, "b_all"));
    double *x = static_cast<double *>(R.arr(2, vb, "x_all"));
    const double tol = R.d(3, "tol");
    const int64_t maxit = R.i(4, "maxit");
    const int64_t mode = R.i(5, "mode");
    const double inner_tol = R.d(6, "inner_tol");
    const int64_t max_outer = R.i(7, "max_outer");
    int64_t *o_it = static_cast<int64_t *>(R.out(8, SEM_ARG_OUT_INT, "total_iters"));
    double *o_res = static_cast<double *>(R.out(9, SEM_ARG_OUT_DOUBLE, "max_rel_res"));
    const int n = batch_size(B);
    int64_t *its = static_cast<int64_t *>(R.host(10, size_t(n) * 8, "iters", true));
    double *res = static_cast<double *>(R.host(11, size_t(n) * 8, "rel_res", true));
    if (R.err) return R.err;
    if (maxit < 1 || maxit > (1 << 30) || max_outer < 0 || max_outer > 1000)
        return R.fail(SEM_EARG, "maxit must be in [1, 2^30] and max_outer in [0, 1000]");
    if (b == x) return R.fail(SEM_EARG, "b_all and x_all must not alias");
    std::vector<int64_t> it(n);
    std::vector<double> rr(n);
    const int rc = batch_solve(B, b, x, tol, int(maxit), int(mode), inner_tol, int(max_outer), it.data(), rr.data());
    if (rc != SEM_OK) return rc;
    int64_t tot = 0;
    double mx = 0.0;
    for (int k = 0; k < n; ++k) {
        tot += it[k];
        mx = std::max(mx, rr[k]);
        if (its) its[k] = it[k];
        if (res) res[k] = rr[k];
    }
    *o_it = tot;
    *o_res = mx;
    return SEM_OK;
}

int run_batch_free(ArgReader &R) {
    if (!R.need(1)) return R.err;
    const int64_t h = R.i(0, "batch");
    if (R.err) return R.err;
    auto it = g.batches.find(h);
    if (it == g.batches.end()) return R.fail(SEM_EHANDLE, "unknown batch handle");
    sync_stream("batch_free");
    batch_destroy(it->second);
    g.batches.erase(it);
    return SEM_OK;
}

Server *get_server(ArgReader &R, int k) {
    const int64_t h = R.i(k, "server");
    if (R.err) return nullptr;
    auto it = g.servers.find(h);
    if (it == g.servers.end()) {
        R.fail(SEM_EHANDLE, "unknown server handle " + std::to_string(h));
        return nullptr;
    }
    return it->second;
}

int run_serve_open(ArgReader &R) {
    if (!R.need(8)) return R.err;
    const int64_t cap = R.i(0, "capacity");
    const double budget = R.d(1, "budget_gb");
    const int64_t mode = R.i(2, "mode");
    const double tol = R.d(3, "tol");
    const double inner_tol = R.d(4, "inner_tol");
    const int64_t K = R.i(5, "K");
    const int64_t maxit = R.i(6, "maxit");
    int64_t *out = static_cast<int64_t *>(R.out(7, SEM_ARG_OUT_INT, "server"));
    if (R.err) return R.err;
    if (maxit < 1 || maxit > (1 << 30)) return R.fail(SEM_EARG, "maxit must be in [1, 2^30]");
    Server *S = nullptr;
    const int rc = serve_open(int(cap), budget, int(mode), tol, inner_tol, int(K), int(maxit), &S);
    if (rc != SEM_OK) return rc;
    const int64_t h = g.next_handle++;
    g.servers[h] = S;
    *out = h;
    return SEM_OK;
}

int run_serve_submit(ArgReader &R) {
    if (!R.need(10)) return R.err;
    Server *S = get_server(R, 0);
    const int64_t nx = R.i(1, "nx"), ny = R.i(2, "ny"), nz = R.i(3, "nz"), N = R.i(4, "N");
    if (R.err) return R.err;
    if (nx < 1 || ny < 1 || nz < 1 || nx > 4096 || ny > 4096 || nz > 4096 || N < 1 || N > 9)
        return R.fail(SEM_EARG, "nx, ny, nz must be in [1, 4096] and N in [1, 9]");
    const size_t nv = size_t(nx + 1) * size_t(ny + 1) * size_t(nz + 1) * 3;
    const size_t nL = size_t(nx) * ny * nz * (N + 1) * (N + 1) * (N + 1);
    const double *verts = static_cast<const double *>(R.host(5, nv * 8, "verts"));
    const double *b = static_cast<const double *>(R.host(6, nL * 8, "b"));
    const int64_t assemble = R.i(7, "assemble");
    const double arrival = R.d(8, "arrival_s");
    int64_t *ticket = static_cast<int64_t *>(R.out(9, SEM_ARG_OUT_INT, "ticket"));
    if (R.err) return R.err;
    return serve_submit(S, int(nx), int(ny), int(nz), int(N), verts, b, assemble != 0, arrival, ticket);
}

int run_serve_drain(ArgReader &R) {
    if (!R.need(4)) return R.err;
    Server *S = get_server(R, 0);
    const int64_t cap = R.i(2, "cap");
    if (R.err) return R.err;
    if (cap < 0) return R.fail(SEM_EARG, "cap must be >= 0");
    int64_t *out = static_cast<int64_t *>(R.host(1, size_t(cap) * 8, "tickets"));
    int64_t *n = static_cast<int64_t *>(R.out(3, SEM_ARG_OUT_INT, "n"));
    if (R.err) return R.err;
    *n = serve_drain(S, out, cap);
    return SEM_OK;
}

int run_serve_step(ArgReader &R) {
    if (!R.need(4)) return R.err;
    Server *S = get_server(R, 0);
    int64_t *o1 = static_cast<int64_t *>(R.out(1, SEM_ARG_OUT_INT, "queued"));
    int64_t *o2 = static_cast<int64_t *>(R.out(2, SEM_ARG_OUT_INT, "active"));
    int64_t *o3 = static_cast<int64_t *>(R.out(3, SEM_ARG_OUT_INT, "completed"));
    if (R.err) return R.err;
    return serve_step(S, o1, o2, o3);
}

int run_serve_result(ArgReader &R) {
    if (!R.need(7)) return R.err;
    Server *S = get_server(R, 0);
    const int64_t ticket = R.i(1, "ticket");
    if (R.err) return R.err;
    double *x = nullptr;
    bool on_dev = false;
    if (R.nargs > 2 && R.args[2].kind != SEM_ARG_NONE) {
        const int64_t nL = serve_nodes_of(S, ticket);
        if (nL < 0) return R.fail(SEM_EHANDLE, "unknown ticket");
        if (R.args[2].kind == SEM_ARG_HOST) {
            x = static_cast<double *>(R.host(2, size_t(nL) * 8, "x"));
        } else {
            x = static_cast<double *>(R.arr(2, size_t(nL) * 8, "x"));
            on_dev = true;
        }
    }
    int64_t *st = static_cast<int64_t *>(R.out(3, SEM_ARG_OUT_INT, "state"));
    int64_t *its = static_cast<int64_t *>(R.out(4, SEM_ARG_OUT_INT, "iters"));
    double *res = static_cast<double *>(R.out(5, SEM_ARG_OUT_DOUBLE, "rel_res"));
    double *lat = static_cast<double *>(R.out(6, SEM_ARG_OUT_DOUBLE, "latency_ms"));
    if (R.err) return R.err;
    *its = 0;
    *res = 0.0;
    *lat = 0.0;
    return serve_result(S, ticket, x, on_dev, st, its, res, lat);
}

int run_serve_now(ArgReader &R) {
    if (!R.need(2)) return R.err;
    Server *S = get_server(R, 0);
    double *o = static_cast<double *>(R.out(1, SEM_ARG_OUT_DOUBLE, "seconds"));
    if (R.err) return R.err;
    *o = serve_now(S);
    return SEM_OK;
}

int run_serve_close(ArgReader &R) {
    if (!R.need(1)) return R.err;
    const int64_t h = R.i(0, "server");
    if (R.err) return R.err;
    auto it = g.servers.find(h);
    if (it == g.servers.end()) return R.fail(SEM_EHANDLE, "unknown server handle");
    serve_close(it->second);
    g.servers.erase(it);
    return SEM_OK;
}

int run_cg_ax(ArgReader &R) {
    if (!R.need(1)) return R.err;
    Problem *P = get_problem(R, 0, false);
    if (R.err) return R.err;
    // clear the stop flag a finished solve leaves behind, so the kernel does its work
    const int rc = cuda_check(cudaMemsetAsync(&P->st->done, 0, sizeof(int32_t), g.cur_stream), "cg_ax: flag");
    return rc != SEM_OK ? rc : launch_ax_cg(P);
}

// ---- one problem split across ranks (sem_dist.cu)
DistProblem *get_dist(ArgReader &R, int k) {
    const int64_t h = R.i(k, "handle");
    if (R.err) return nullptr;
    auto it = g.dists.find(h);
    if (it == g.dists.end()) {
        R.fail(SEM_EHANDLE, "unknown split-problem handle " + std::to_string(h));
        return nullptr;
    }
    return it->second;
}

const sem_comm *get_comm(ArgReader &R, int k) {
    return static_cast<const sem_comm *>(R.host(k, sizeof(sem_comm), "comm"));
}

int run_dist_mesh(ArgReader &R) {
    if (!R.need(7)) return R.err;
    const int64_t nx = R.i(0, "nx"), ny = R.i(1, "ny"), nz = R.i(2, "nz"), N = R.i(3, "N");
    if (R.err) return R.err;
    if (nx < 1 || ny < 1 || nz < 1 || nx > (1 << 20) || ny > (1 << 20) || nz > (1 << 20))
        return R.fail(SEM_EARG, "nx, ny, nz must be in [1, 2^20]");
    const size_t nv = size_t(nx + 1) * size_t(ny + 1) * size_t(nz + 1);
    const double *verts = static_cast<const double *>(R.arr(4, nv * 3 * sizeof(double), "verts"));
    const int64_t nb = R.i(5, "neighbours");
    int64_t *out = static_cast<int64_t *>(R.out(6, SEM_ARG_OUT_INT, "handle"));
    if (R.err) return R.err;
    if (nb < 0 || nb > 3) return R.fail(SEM_EARG, "neighbours must be in [0, 3]");
    DistProblem *D = nullptr;
    const int rc = dist_create(int(nx), int(ny), int(nz), int(N), verts, (nb & 1) != 0, (nb & 2) != 0, &D);
    if (rc != SEM_OK) return rc;
    const int64_t h = g.next_handle++;
    g.dists[h] = D;
    *out = h;
    return SEM_OK;
}

int run_dist_info(ArgReader &R) {
    if (!R.need(2)) return R.err;
    DistProblem *D = get_dist(R, 0);
    int64_t *o = static_cast<int64_t *>(R.out(1, SEM_ARG_OUT_INT, "nL"));
    if (R.err) return R.err;
    *o = dist_problem(D)->nL;
    return SEM_OK;
}

int run_dist_ax(ArgReader &R) {
    if (!R.need(3)) return R.err;
    DistProblem *D = get_dist(R, 0);
    if (R.err) return R.err;
    Problem *P = dist_problem(D);
    const size_t vb = size_t(P->nL) * sizeof(double);
    const double *x = static_cast<const double *>(R.arr(1, vb, "x"));
    double *y = static_cast<double *>(R.arr(2, vb, "y"));
    if (R.err) return R.err;
    if (x == y) return R.fail(SEM_EARG, "x and y must not alias");
    return launch_ax(P, x, y);
}

int run_dist_gs(ArgReader &R) {
    if (!R.need(3)) return R.err;
    DistProblem *D = get_dist(R, 0);
    if (R.err) return R.err;
    double *u = static_cast<double *>(R.arr(1, size_t(dist_problem(D)->nL) * sizeof(double), "u"));
    const sem_comm *comm = get_comm(R, 2);
    if (R.err) return R.err;
    const int rc = dist_gs(D, u, comm);
    return rc != SEM_OK ? rc : sync_stream("dist_gs");
}

int run_dist_dot(ArgReader &R) {
    if (!R.need(5)) return R.err;
    DistProblem *D = get_dist(R, 0);
    if (R.err) return R.err;
    const size_t vb = size_t(dist_problem(D)->nL) * sizeof(double);
    const double *u = static_cast<const double *>(R.arr(1, vb, "u"));
    const double *v = static_cast<const double *>(R.arr(2, vb, "v"));
    const sem_comm *comm = get_comm(R, 3);
    double *o = static_cast<double *>(R.out(4, SEM_ARG_OUT_DOUBLE, "result"));
    if (R.err) return R.err;
    return dist_dot(D, u, v, comm, o);
}

int run_dist_cg_solve(ArgReader &R) {
    if (!R.need(9)) return R.err;
    DistProblem *D = get_dist(R, 0);
    if (R.err) return R.err;
    const size_t vb = size_t(dist_problem(D)->nL) * sizeof(double);
    const double *b = static_cast<const double *>(R.arr(1, vb, "b"));
    double *x = static_cast<double *>(R.arr(2, vb, "x"));
    const double tol = R.d(3, "tol");
    const int64_t maxit = R.i(4, "maxit");
    const sem_comm *comm = get_comm(R, 5);
    if (R.err) return R.err;
    if (maxit < 0 || maxit > (1 << 30)) return R.fail(SEM_EARG, "maxit must be in [0, 2^30]");
    double *hist = static_cast<double *>(R.host(6, size_t(maxit + 1) * sizeof(double), "hist", true));
    int64_t *oit = static_cast<int64_t *>(R.out(7, SEM_ARG_OUT_INT, "iters"));
    double *ores = static_cast<double *>(R.out(8, SEM_ARG_OUT_DOUBLE, "rel_res"));
    if (R.err) return R.err;
    if (b == x) return R.fail(SEM_EARG, "b and x must not alias");
    return dist_cg_solve(D, b, x, tol, int(maxit), hist, comm, oit, ores);
}

int run_dist_free(ArgReader &R) {
    if (!R.need(1)) return R.err;
    const int64_t h = R.i(0, "handle");
    if (R.err) return R.err;
    auto it = g.dists.find(h);
    if (it == g.dists.end()) return R.fail(SEM_EHANDLE, "unknown split-problem handle");
    dist_destroy(it->second);
    g.dists.erase(it);
    return SEM_OK;
}

int run_wait_probe(ArgReader &R) {
    if (!R.need(2)) return R.err;
    const int64_t limit = R.i(0, "limit_ns");
    double *out = static_cast<double *>(R.out(1, SEM_ARG_OUT_DOUBLE, "copied"));
    if (R.err) return R.err;
    if (limit < 0) return R.fail(SEM_EARG, "limit_ns must be positive");
    return probe_wait_timeout(uint64_t(limit), out);
}

int run_peak_fma(ArgReader &R) {
    if (!R.need(3)) return R.err;
    const int64_t dtype = R.i(0, "dtype"), iters = R.i(1, "iters");
    double *out = static_cast<double *>(R.out(2, SEM_ARG_OUT_DOUBLE, "flops_per_s"));
    if (R.err) return R.err;
    if (dtype != 0 && dtype != 1) return R.fail(SEM_EARG, "dtype must be 0 (f64) or 1 (f32)");
    return probe_fma_rate(int(dtype), int(iters), out);
}

int run_pcg_solve(ArgReader &R) {
    if (!R.need(7)) return R.err;
    Problem *P = get_problem(R, 0);
    if (R.err) return R.err;
    const size_t vb = size_t(P->nL) * sizeof(double);
    const double *b = static_cast<const double *>(R.arr(1, vb, "b"));
    double *x = static_cast<double *>(R.arr(2, vb, "x"));
    const double tol = R.d(3, "tol");
    const int64_t maxit = R.i(4, "maxit");
    int64_t *oit = static_cast<int64_t *>(R.out(5, SEM_ARG_OUT_INT, "iters"));
    double *ores = static_cast<double *>(R.out(6, SEM_ARG_OUT_DOUBLE, "rel_res"));
    if (R.err) return R.err;
    if (maxit < 0 || maxit > (1 << 30)) return R.fail(SEM_EARG, "maxit must be in [0, 2^30]");
    double *hist = static_cast<double *>(R.arr(7, size_t(maxit + 1) * sizeof(double), "hist", true));
    if (R.err) return R.err;
    if (b == x) return R.fail(SEM_EARG, "b and x must not alias");
    return pcg_solve(P, b, x, tol, int(maxit), hist, oit, ores);
}

int run_jacobi(ArgReader &R) {
    if (!R.need(2)) return R.err;
    Problem *P = get_problem(R, 0);
    if (R.err) return R.err;
    double *out = static_cast<double *>(R.arr(1, size_t(P->nL) * sizeof(double), "dinv"));
    if (R.err) return R.err;
    const int rc = jacobi_prepare(P);
    if (rc != SEM_OK) return rc;
    return cuda_check(cudaMemcpyAsync(out, P->dinv, size_t(P->nL) * sizeof(double), cudaMemcpyDeviceToDevice,
                                      g.cur_stream), "jacobi: copy");
}

int run_true_res(ArgReader &R) {
    if (!R.need(4)) return R.err;
    Problem *P = get_problem(R, 0);
    if (R.err) return R.err;
    const size_t vb = size_t(P->nL) * sizeof(double);
    const double *b = static_cast<const double *>(R.arr(1, vb, "b"));
    const double *x = static_cast<const double *>(R.arr(2, vb, "x"));
    double *out = static_cast<double *>(R.out(3, SEM_ARG_OUT_DOUBLE, "result"));
    if (R.err) return R.err;
    // w = A x (assembled, masked); r = b - w, both in the problem's work vectors
    double *w = P->w, *r = P->r;
    if (x == w || x == r || b == w || b == r) return R.fail(SEM_EARG, "arguments alias work vectors");
    int rc = launch_ax(P, x, w);
    if (rc == SEM_OK) rc = launch_gs(P, w);
    if (rc == SEM_OK) rc = launch_mask(P, w);
    if (rc == SEM_OK) rc = launch_sub(P, b, w, r);
    double rr = 0.0, bb = 0.0;
    for (int pass = 0; pass < 2 && rc == SEM_OK; ++pass) {
        rc = launch_dot(P, pass == 0 ? r : b, pass == 0 ? r : b);
        if (rc == SEM_OK)
            rc = cuda_check(cudaMemcpyAsync(&P->st_host->dot_out, &P->st->dot_out, sizeof(double),
                                            cudaMemcpyDeviceToHost, g.cur_stream), "true_res: read");
        if (rc == SEM_OK) rc = sync_stream("true_res: sync");
        if (rc == SEM_OK) (pass == 0 ? rr : bb) = P->st_host->dot_out;
    }
    if (rc != SEM_OK) return rc;
    *out = bb > 0.0 ? std::sqrt(rr / bb) : std::sqrt(rr);
    return SEM_OK;
}

}  // namespace
}  // namespace sem

using namespace sem;

extern "C" {

int sem_init(int argc, const char **argv) {
    if (g.up) return set_error(SEM_EINIT, "sem_init: already initialised");
    int device = 0, verbose = 0;
    double budget_gb = 0.0;
    const char *table = nullptr;
    for (int a = 0; a < argc; ++a) {
        if (!argv || !argv[a]) continue;
        const char *s = argv[a];
        if (!strncmp(s, "--device=", 9)) device = atoi(s + 9);
        else if (!strncmp(s, "--verbose=", 10)) verbose = atoi(s + 10);
        else if (!strncmp(s, "--hbm-budget=", 13)) budget_gb = atof(s + 13);
        else if (!strncmp(s, "--autotune-table=", 17)) table = s + 17;
    }
    tune_reset();
    if (table) {
        const int trc = tune_load(table);
        if (trc != SEM_OK) return trc;
    }
    int rc = cuda_check(cudaSetDevice(device), "sem_init: cudaSetDevice");
    if (rc != SEM_OK) return rc;
    rc = cuda_check(cudaGetDeviceProperties(&g.prop, device), "sem_init: device query");
    if (rc != SEM_OK) return rc;
    rc = cuda_check(cudaStreamCreateWithFlags(&g.own_stream, cudaStreamNonBlocking), "sem_init: stream");
    if (rc != SEM_OK) return rc;
    g.cur_stream = g.own_stream;
    g.device = device;
    g.verbose = verbose;
    g.budget = budget_gb > 0 ? size_t(budget_gb * 1e9) : 0;
    g.in_use = 0;
    g.up = true;
    g.status_dev = static_cast<int32_t *>(dev_alloc(sizeof(int32_t) * 4));
    if (!g.status_dev) {
        g.up = false;
        return SEM_ENOMEM;
    }
    rc = cuda_check(cudaMallocHost(&g.status_pinned, sizeof(int32_t) * 4), "sem_init: pinned status");
    if (rc == SEM_OK) rc = cuda_check(cudaMemsetAsync(g.status_dev, 0, sizeof(int32_t) * 4, g.cur_stream), "sem_init");
    if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(g.cur_stream), "sem_init: sync");
    if (rc != SEM_OK) {
        g.up = false;
        return rc;
    }
    g_launches = 0;
    if (verbose)
        fprintf(stderr, "[sem] device %d: %s, %d SMs, cc %d.%d, %zu KB smem/block (opt-in)\n", device,
                g.prop.name, g.prop.multiProcessorCount, g.prop.major, g.prop.minor,
                size_t(g.prop.sharedMemPerBlockOptin) / 1024);
    return SEM_OK;
}

int sem_update(void *host, size_t start, size_t end, size_t elem_size, int op) {
    if (!g.up) return set_error(SEM_EINIT, "sem_update: not initialised");
    if (!host || elem_size == 0 || end < start) return set_error(SEM_EARG, "sem_update: bad host pointer or range");
    const uintptr_t key = reinterpret_cast<uintptr_t>(host);
    auto it = g.mirrors.find(key);
    switch (op) {
        case SEM_ALLOC:
        case SEM_TO: {
            if (it == g.mirrors.end()) {
                if (end == start) return set_error(SEM_EARG, "sem_update: empty range");
                Mirror m{key, start, end, elem_size, nullptr};
                m.dev = dev_alloc((end - start) * elem_size);
                if (!m.dev) return SEM_ENOMEM;
                it = g.mirrors.emplace(key, m).first;
            } else if (op == SEM_ALLOC) {
                return set_error(SEM_EARG, "sem_update(alloc): host array already has a mirror");
            }
            if (op == SEM_TO) {
                Mirror &m = it->second;
                if (elem_size != m.elem || start < m.start || end > m.end)
                    return set_error(SEM_ERANGE, "sem_update(to): range outside the mirror");
                if (end > start)
                    return cuda_check(cudaMemcpyAsync(static_cast<unsigned char *>(m.dev) + (start - m.start) * m.elem,
                                                      static_cast<unsigned char *>(host) + start * m.elem,
                                                      (end - start) * m.elem, cudaMemcpyHostToDevice, g.cur_stream),
                                      "sem_update(to)");
            }
            return SEM_OK;
        }
        case SEM_FROM: {
            if (it == g.mirrors.end()) return set_error(SEM_ENOMAP, "sem_update(from): host array has no mirror");
            Mirror &m = it->second;
            if (elem_size != m.elem || start < m.start || end > m.end)
                return set_error(SEM_ERANGE, "sem_update(from): range outside the mirror");
            if (end > start)
                return cuda_check(cudaMemcpyAsync(static_cast<unsigned char *>(host) + start * m.elem,
                                                  static_cast<unsigned char *>(m.dev) + (start - m.start) * m.elem,
                                                  (end - start) * m.elem, cudaMemcpyDeviceToHost, g.cur_stream),
                                  "sem_update(from)");
            return SEM_OK;
        }
        case SEM_FREE: {
            if (it == g.mirrors.end()) return set_error(SEM_ENOMAP, "sem_update(free): host array has no mirror");
            cudaStreamSynchronize(g.cur_stream);
            dev_free(it->second.dev);
            g.mirrors.erase(it);
            return SEM_OK;
        }
        default:
            return set_error(SEM_EARG, "sem_update: unknown operation");
    }
}

int sem_run(const char *kernel, int nargs, const sem_arg *args) {
    if (!g.up) return set_error(SEM_EINIT, "sem_run: not initialised");
    if (!kernel) return set_error(SEM_EARG, "sem_run: kernel name is NULL");
    if (nargs < 0 || (nargs > 0 && !args)) return set_error(SEM_EARG, "sem_run: bad argument list");
    ArgReader R{kernel, nargs, args};
    const std::string k(kernel);
    int rc;
    if (k == "mesh") rc = run_mesh(R);
    else if (k == "mesh_free") rc = run_mesh_free(R);
    else if (k == "info") rc = run_info(R);
    else if (k == "ax") rc = run_ax(R, false);
    else if (k == "axg") rc = run_ax(R, true);
    else if (k == "gs") rc = run_inplace(R, 0);
    else if (k == "mask") rc = run_inplace(R, 1);
    else if (k == "dot") rc = run_dot(R);
    else if (k == "geom") rc = run_geom(R);
    else if (k == "nodes") rc = run_nodes(R);
    else if (k == "gs_map") rc = run_gs_map(R);
    else if (k == "rhs") rc = run_rhs(R, false);
    else if (k == "rhs_sin") rc = run_rhs(R, true);
    else if (k == "cg_solve") rc = run_cg_solve(R);
    else if (k == "true_res") rc = run_true_res(R);
    else if (k == "pcg_solve") rc = run_pcg_solve(R);
    else if (k == "jacobi") rc = run_jacobi(R);
    else if (k == "cg_ax") rc = run_cg_ax(R);
    else if (k == "ax32") rc = run_ax32(R);
    else if (k == "cg_ax32") rc = run_cg_ax32(R);
    else if (k == "cg_mixed") rc = run_cg_mixed(R);
    else if (k == "batch") rc = run_batch(R);
    else if (k == "batch_info") rc = run_batch_info(R);
    else if (k == "batch_solve") rc = run_batch_solve(R);
    else if (k == "batch_free") rc = run_batch_free(R);
    else if (k == "serve_open") rc = run_serve_open(R);
    else if (k == "serve_submit") rc = run_serve_submit(R);
    else if (k == "serve_step") rc = run_serve_step(R);
    else if (k == "serve_result") rc = run_serve_result(R);
    else if (k == "serve_now") rc = run_serve_now(R);
    else if (k == "serve_drain") rc = run_serve_drain(R);
    else if (k == "serve_close") rc = run_serve_close(R);
    else if (k == "peak_fma") rc = run_peak_fma(R);
    else if (k == "wait_probe") rc = run_wait_probe(R);
    else if (k == "dist_mesh") rc = run_dist_mesh(R);
    else if (k == "dist_info") rc = run_dist_info(R);
    else if (k == "dist_ax") rc = run_dist_ax(R);
    else if (k == "dist_gs") rc = run_dist_gs(R);
    else if (k == "dist_dot") rc = run_dist_dot(R);
    else if (k == "dist_cg_solve") rc = run_dist_cg_solve(R);
    else if (k == "dist_free") rc = run_dist_free(R);
    else if (k == "autotune") rc = run_autotune(R);
    else if (k == "autotune_get") rc = run_autotune_get(R);
    else if (k == "autotune_set") rc = run_autotune_set(R);
    else if (k == "autotune_save") rc = run_autotune_file(R, true);
    else if (k == "autotune_load") rc = run_autotune_file(R, false);
    else return set_error(SEM_EKERNEL, "sem_run: unknown kernel '" + k + "'");
    return rc;
}

int sem_sync(void) {
    if (!g.up) return set_error(SEM_EINIT, "sem_sync: not initialised");
    int rc = cuda_check(cudaStreamSynchronize(g.cur_stream), "sem_sync");
    if (rc != SEM_OK) return rc;
    return poll_status();
}

int sem_finalize(void) {
    if (!g.up) return set_error(SEM_EINIT, "sem_finalize: not initialised");
    cudaStreamSynchronize(g.cur_stream);
    for (auto &kv : g.servers) serve_close(kv.second);
    g.servers.clear();
    for (auto &kv : g.batches) batch_destroy(kv.second);
    g.batches.clear();
    for (auto &kv : g.problems) problem_destroy(kv.second);
    g.problems.clear();
    for (auto &kv : g.dists) dist_destroy(kv.second);
    g.dists.clear();
    for (auto &kv : g.mirrors) dev_free(kv.second.dev);
    g.mirrors.clear();
    dev_free(g.status_dev);
    g.status_dev = nullptr;
    if (g.status_pinned) cudaFreeHost(g.status_pinned);
    pinned_release_all();
    g.status_pinned = nullptr;
    if (g.own_stream) cudaStreamDestroy(g.own_stream);
    g.own_stream = nullptr;
    g.cur_stream = nullptr;
    g.sizes.clear();
    g.in_use = 0;
    g.up = false;
    return SEM_OK;
}

const char *sem_last_error(void) { return g_err; }

int sem_set_allocator(sem_alloc_fn alloc_fn, sem_free_fn free_fn, void *ctx) {
    if ((alloc_fn == nullptr) != (free_fn == nullptr))
        return set_error(SEM_EARG, "sem_set_allocator: give both hooks or neither");
    if (!g.sizes.empty()) return set_error(SEM_EARG, "sem_set_allocator: device memory is still allocated");
    g.alloc_fn = alloc_fn;
    g.free_fn = free_fn;
    g.alloc_ctx = ctx;
    return SEM_OK;
}

int sem_set_stream(void *s) {
    if (!g.up) return set_error(SEM_EINIT, "sem_set_stream: not initialised");
    cudaStreamSynchronize(g.cur_stream);
    g.cur_stream = s ? static_cast<cudaStream_t>(s) : g.own_stream;
    return SEM_OK;
}

int64_t sem_launch_count(void) { return g_launches.load(); }

}  // extern "C"
