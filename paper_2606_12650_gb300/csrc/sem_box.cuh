// sem_box.cuh -- copies of a global node on the structured box mesh.
//
// On an nx x ny x nz box of order N, local node (e; i, j, k) of element
// (ex, ey, ez) shares its global node with the elements across every element
// face it lies on: along r when i = 0 (element ex-1, at i = N) or i = N
// (element ex+1, at i = 0), and likewise along s and t.  Nodes on the cube
// boundary are Dirichlet (masked).  Moving to the neighbour across the r face
// changes the local index by sx * (NP - N) (sx = -1 at i = 0, +1 at i = N,
// NP = (N+1)^3); across s by sy * (nx NP - N (N+1)); across t by
// sz * (nx ny NP - N (N+1)^2).  Local indices order copies by element first,
// and element indices are lexicographic in (ez, ey, ex); so visiting the t
// choice, then s, then r, each with the lower element first, lists the copies
// in ascending local index -- the order of the sorted-segment gather-scatter,
// which makes every copy's sum bit-identical.
#pragma once

#include <algorithm>
#include <cstdint>
#include <type_traits>

namespace sem {

struct BoxNode {
    int sx, sy, sz;     // -1 low face, +1 high face, 0 interior (per direction)
    int ox, oy, oz;     // signed local-index offsets to the neighbour copies
    bool masked;        // on the cube boundary
    bool owner;         // first copy of its global node
};

// Division by a divisor d >= 1 fixed for a launch, for dividends n < 2^31:
// with l = ceil(log2 d) and m = ceil(2^(31+l) / d) < 2^32, floor(n / d) =
// floor(n m / 2^(31+l)) (Granlund and Montgomery, "Division by invariant
// integers using multiplication", 1994, Thm 4.2 with N = 31).  One wide
// multiply and a shift instead of the ~20-instruction integer division.
struct DivU {
    uint32_t m;
    uint32_t s;
};

inline DivU make_divu(uint32_t d) {
    uint32_t l = 0;
    while ((uint64_t(1) << l) < d) ++l;
    const uint64_t m = ((uint64_t(1) << (31 + l)) + d - 1) / d;
    return DivU{uint32_t(m), 31 + l};
}

__device__ __forceinline__ uint32_t divu(uint32_t n, DivU D) { return uint32_t((uint64_t(n) * D.m) >> D.s); }

// Box sizes with their fast divisors (element index -> (ex, ey, ez)).
struct BoxDims {
    int nx, ny, nz;
    DivU dx, dy;
};

inline BoxDims box_dims(int nx, int ny, int nz) { return BoxDims{nx, ny, nz, make_divu(uint32_t(nx)), make_divu(uint32_t(ny))}; }

template <int NQ>
__device__ __forceinline__ BoxNode box_node(int l, int nx, int ny, int nz) {
    constexpr int N = NQ - 1, NQ2 = NQ * NQ, NP = NQ2 * NQ;
    const unsigned e = unsigned(l) / unsigned(NP);
    const int q = l - int(e) * NP;
    const int i = q % NQ, j = (q / NQ) % NQ, k = q / NQ2;
    const unsigned t = e / unsigned(nx);
    const int ex = int(e - t * unsigned(nx));
    const unsigned tz = t / unsigned(ny);
    const int ey = int(t - tz * unsigned(ny)), ez = int(tz);
    BoxNode b;
    b.sx = i == 0 ? -1 : (i == N ? 1 : 0);
    b.sy = j == 0 ? -1 : (j == N ? 1 : 0);
    b.sz = k == 0 ? -1 : (k == N ? 1 : 0);
    b.ox = b.sx * (NP - N);
    b.oy = b.sy * (nx * NP - N * NQ);
    b.oz = b.sz * (nx * ny * NP - N * NQ2);
    b.masked = (b.sx < 0 && ex == 0) || (b.sx > 0 && ex == nx - 1) ||
               (b.sy < 0 && ey == 0) || (b.sy > 0 && ey == ny - 1) ||
               (b.sz < 0 && ez == 0) || (b.sz > 0 && ez == nz - 1);
    b.owner = b.sx >= 0 && b.sy >= 0 && b.sz >= 0;
    return b;
}

}  // namespace sem

#include "sem_device.cuh"
#include "sem_dw.cuh"

namespace sem {

// Accumulators of <r, r>: FP64 or FP32 fma, or (FP64 CG update) double-word
// FP32, which takes the reduction off GB300's 1/64-rate FP64 pipe; the
// recurrences (copy sums, r -= alpha w) stay FP64.
struct DwAcc {
    dwf v;
};
__device__ __forceinline__ void acc_square(double &a, double r) { a = fma(r, r, a); }
__device__ __forceinline__ void acc_square(float &a, float r) { a = fmaf(r, r, a); }
__device__ __forceinline__ void acc_square(DwAcc &a, double r) { a.v = dw_add_square(a.v, r); }
// Jacobi PCG: acc + d r^2 (= r . (d r) with z = d r), FP64 or double-word
__device__ __forceinline__ void acc_weighted_square(double &a, double d, double r) { a = fma(r, d * r, a); }
__device__ __forceinline__ void acc_weighted_square(DwAcc &a, double d, double r) {
    a.v = dw_add_weighted_square(a.v, d, r);
}
__device__ __forceinline__ void acc_merge(double &a, double b) { a += b; }
__device__ __forceinline__ void acc_merge(float &a, float b) { a += b; }
__device__ __forceinline__ void acc_merge(DwAcc &a, const DwAcc &b) { a.v = dw_add(a.v, b.v); }
__device__ __forceinline__ double acc_value(double a) { return a; }
__device__ __forceinline__ double acc_value(float a) { return double(a); }
__device__ __forceinline__ double acc_value(const DwAcc &a) { return dw_to_double(a.v); }
template <typename Acc>
__device__ __forceinline__ Acc acc_zero() { return Acc(0); }
template <>
__device__ __forceinline__ DwAcc acc_zero<DwAcc>() { return DwAcc{{0.0f, 0.0f}}; }

// Vector width for the update: V consecutive nodes of one row share the
// element, j and k; V divides N+1 and V * sizeof(T) <= 16 bytes.
template <int NQ, typename T>
struct UpdVec {
    static constexpr int by16 = 16 / int(sizeof(T));
    static constexpr int value = (NQ % by16 == 0) ? by16 : ((NQ % 2 == 0 && by16 >= 2) ? 2 : 1);
};

template <typename T, int V>
struct VecT;
template <> struct VecT<float, 4> { using type = float4; };
template <> struct VecT<float, 2> { using type = float2; };
template <> struct VecT<float, 1> { using type = float; };
template <> struct VecT<double, 2> { using type = double2; };
template <> struct VecT<double, 1> { using type = double; };

template <typename T, int V>
__device__ __forceinline__ void vload(const T *p, T (&v)[V]) {
    const typename VecT<T, V>::type q = *reinterpret_cast<const typename VecT<T, V>::type *>(p);
    const T *a = reinterpret_cast<const T *>(&q);
#pragma unroll
    for (int c = 0; c < V; ++c) v[c] = a[c];
}

template <typename T, int V>
__device__ __forceinline__ void vload_nc(const T *p, T (&v)[V]) {
    const typename VecT<T, V>::type q = __ldg(reinterpret_cast<const typename VecT<T, V>::type *>(p));
    const T *a = reinterpret_cast<const T *>(&q);
#pragma unroll
    for (int c = 0; c < V; ++c) v[c] = a[c];
}

template <typename T, int V>
__device__ __forceinline__ void vstore(T *p, const T (&v)[V]) {
    typename VecT<T, V>::type q;
    T *a = reinterpret_cast<T *>(&q);
#pragma unroll
    for (int c = 0; c < V; ++c) a[c] = v[c];
    *reinterpret_cast<typename VecT<T, V>::type *>(p) = q;
}

// Fused direct-stiffness sum + CG update for the V consecutive nodes
// l0 .. l0+V-1 (one row piece of one element).  A node's copies are the
// combinations of {own, neighbour} element along each direction in which it
// lies on an interior element face; enumerating the (t, s) choices with the
// lower element first, and within each the r-face neighbour of node 0 (lower
// element) before the own value and that of node N (upper element) after it,
// lists the copies in ascending local index -- the order of the sorted-
// segment gather-scatter, so every copy of a node gets the same bits.  The
// nodes then update themselves: r -= alpha (QQ^T w), and x += alpha p unless
// DX (the x update is deferred to the next operator kernel, which holds p in
// shared memory anyway).  Masked nodes are left as they are (zero).  <r, r>
// (PRE: <r, M^-1 r> and <r, r> into *acc_rr) is accumulated into acc at each
// node's first copy.
template <int NQ, int V, typename T, typename Acc, bool PRE = false, bool DX = false>
__device__ __forceinline__ void update_vec(T *__restrict__ x, T *__restrict__ r, const T *__restrict__ p,
                                          const T *__restrict__ w, int l0, const BoxDims &bd, T alpha,
                                          Acc &acc, const T *__restrict__ dinv = nullptr,
                                          Acc *acc_rr = nullptr) {
    constexpr int N = NQ - 1, NQ2 = NQ * NQ, NP = NQ2 * NQ;
    const int nx = bd.nx, ny = bd.ny, nz = bd.nz;
    const unsigned e = unsigned(l0) / unsigned(NP);
    const int q = l0 - int(e) * NP;
    const int i0 = q % NQ, j = (q / NQ) % NQ, k = q / NQ2;
    const unsigned t = divu(e, bd.dx);
    const int ex = int(e - t * unsigned(nx));
    const unsigned tz = divu(t, bd.dy);
    const int ey = int(t - tz * unsigned(ny)), ez = int(tz);
    const int sy = j == 0 ? -1 : (j == N ? 1 : 0);
    const int sz = k == 0 ? -1 : (k == N ? 1 : 0);
    if ((sy < 0 && ey == 0) || (sy > 0 && ey == ny - 1) || (sz < 0 && ez == 0) || (sz > 0 && ez == nz - 1))
        return;                                           // on the cube boundary
    const int oy = sy * (nx * NP - N * NQ);
    const int oz = sz * (nx * ny * NP - N * NQ2);
    const bool has_lo = i0 == 0 && ex > 0;                // node i = 0 has a lower r neighbour
    const bool has_hi = i0 + V - 1 == N && ex < nx - 1;   // node i = N has a higher r neighbour
    const bool mask_lo = i0 == 0 && ex == 0;
    const bool mask_hi = i0 + V - 1 == N && ex == nx - 1;
    // the node's own values first: their loads then overlap those of w and
    // its neighbour copies below instead of waiting for the sum
    T xv[V], pv[V], rv[V], dv[V];
    if (!DX) {
        vload<T, V>(x + l0, xv);
        vload<T, V>(p + l0, pv);
    }
    vload<T, V>(r + l0, rv);
    if (PRE) vload<T, V>(dinv + l0, dv);
    T sv[V];
    if (sy == 0 && sz == 0) {
        // Row inside the element in s and t: copies only across the r faces.
        // Rows are handed out so that a warp holds rows of one class, so this
        // branch is taken or skipped by whole warps.
        T wv[V];
        vload_nc<T, V>(w + l0, wv);
        const T lo = has_lo ? __ldg(w + l0 - (NP - N)) : T(0);
        const T hi = has_hi ? __ldg(w + l0 + (V - 1) + (NP - N)) : T(0);
#pragma unroll
        for (int v = 0; v < V; ++v) sv[v] = wv[v];
        if (V < NQ) {
            // no piece holds both node 0 and node N: one addition serves
            // either (lo + own_0) or (own_N + hi)
            const T a = has_lo ? lo : wv[V - 1];
            const T b = has_lo ? wv[0] : hi;
            const T sum = a + b;
            if (has_lo) sv[0] = sum;
            if (has_hi) sv[V - 1] = sum;
        } else {
            if (has_lo) sv[0] = lo + wv[0];
            if (has_hi) sv[V - 1] = sv[V - 1] + hi;
        }
    } else {
        const int z0 = sz < 0 ? oz : 0, z1 = sz > 0 ? oz : 0;
        const int y0 = sy < 0 ? oy : 0, y1 = sy > 0 ? oy : 0;
        T wv[4][V], lo[4], hi[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int cz = c >> 1, cy = c & 1;
            const bool valid = (cz == 0 || sz) && (cy == 0 || sy);
            const int off = l0 + (cz ? z1 : z0) + (cy ? y1 : y0);
            if (valid) {
                vload_nc<T, V>(w + off, wv[c]);
                lo[c] = has_lo ? __ldg(w + off - (NP - N)) : T(0);              // element ex-1, node i = N
                hi[c] = has_hi ? __ldg(w + off + (V - 1) + (NP - N)) : T(0);   // element ex+1, node i = 0
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) wv[c][v] = T(0);
                lo[c] = hi[c] = T(0);
            }
        }
        if constexpr (V == NQ || sizeof(T) == 4) {
            // one piece is the whole row (node 0 and node N may both have an
            // r-face neighbour), or FP32, where additions are cheap and the
            // step is bound by memory: each node's additions, the neighbour
            // ones predicated on the lane
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const bool first_lo = (v == 0) && has_lo;
                const bool last_hi = (v == V - 1) && has_hi;
                T s = first_lo ? lo[0] + wv[0][v] : wv[0][v];
                if (last_hi) s = s + hi[0];
#pragma unroll
                for (int c = 1; c < 4; ++c) {
                    const int cz = c >> 1, cy = c & 1;
                    const bool valid = (cz == 0 || sz) && (cy == 0 || sy);
                    if (!valid) continue;
                    if (first_lo) s = s + lo[c];
                    s = s + wv[c][v];
                    if (last_hi) s = s + hi[c];
                }
                sv[v] = s;
            }
        } else {
            // FP64: the same chain of additions in every lane of a warp (no
            // additions predicated off, which would still take FP64 issue
            // slots at 1/64 rate): a piece shorter than the row holds at most one
            // node with an r-face neighbour (node 0 with one below, or node N
            // with one above).  That node sums, per copy class c in order, the
            // pair (lower element's copy, upper element's copy) -- (lo, own) or
            // (own, hi); a piece without such a node runs the chain on its last
            // node with zeros for the neighbour (x + 0 == x).  The other nodes
            // sum their own copies.  The operands and their order are those of
            // the ascending local index, so every copy of a node still gets the
            // same bits.
            T spec = T(0), oe = T(0), mid[V];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int cz = c >> 1, cy = c & 1;
                const bool valid = (cz == 0 || sz) && (cy == 0 || sy);   // c = 0 always
                if (!valid) continue;
                const T x = has_lo ? lo[c] : hi[c];              // 0 without a neighbour
                const T ws = has_lo ? wv[c][0] : wv[c][V - 1];
                const T a = has_lo ? x : ws, b = has_lo ? ws : x;
                spec = c == 0 ? a + b : (spec + a) + b;
                if (V >= 2) {
                    const T we = has_lo ? wv[c][V - 1] : wv[c][0];
                    oe = c == 0 ? we : oe + we;
                }
#pragma unroll
                for (int v = 1; v < V - 1; ++v) mid[v] = c == 0 ? wv[c][v] : mid[v] + wv[c][v];
            }
            if (V == 1) {
                sv[0] = spec;
            } else {
                sv[0] = has_lo ? spec : oe;
                sv[V - 1] = has_lo ? oe : spec;
#pragma unroll
                for (int v = 1; v < V - 1; ++v) sv[v] = mid[v];
            }
        }
    }
    const bool owner_row = sy >= 0 && sz >= 0;
    Acc rr = acc_zero<Acc>();
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const bool masked = (v == 0 && mask_lo) || (v == V - 1 && mask_hi);
        if (!masked) {
            if (!DX) xv[v] = fma(alpha, pv[v], xv[v]);
            rv[v] = fma(-alpha, sv[v], rv[v]);
            if (owner_row && !((v == 0) && has_lo)) {
                if constexpr (PRE) {
                    // <r, M^-1 r> for beta and <r, r> for the stop test
                    acc_weighted_square(acc, dv[v], rv[v]);
                    acc_square(rr, rv[v]);
                } else {
                    acc_square(acc, rv[v]);
                }
            }
        }
    }
    if (!DX) vstore<T, V>(x + l0, xv);
    vstore<T, V>(r + l0, rv);
    if constexpr (PRE) acc_merge(*acc_rr, rr);
}

// Row-class mapping of update vectors to threads: a warp takes the same row
// (j, k) of EG consecutive elements, LR = (N+1)/V lanes per row, so every
// lane of a warp is in the same face class in s and t (the gather branches
// of update_vec are warp-uniform).  Returns the first local node of the
// lane's vector, or -1 for an idle lane.
template <int NQ, int V>
struct RowMap {
    static constexpr int NQ2 = NQ * NQ, NP = NQ2 * NQ;
    static constexpr int LR = NQ / V;
    static constexpr int EG = 32 / LR;
    static __device__ __forceinline__ int l0(int task, int lane, int E) {
        const int eg = task / NQ2;
        const int row = task - eg * NQ2;
        const int g = lane / LR, v = lane - g * LR;
        const int e = eg * EG + g;
        if (g >= EG || e >= E) return -1;
        return e * NP + row * NQ + v * V;
    }
    static __host__ __device__ int tasks(int E) { return (E + EG - 1) / EG * NQ2; }
};

// b = mask(QQ^T f) on the box (copies summed in ascending local index).
template <int NQ>
__global__ void assemble_box_kernel(const double *__restrict__ f, double *__restrict__ b, int nL, int nx, int ny,
                                    int nz) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nL) return;
    const BoxNode bn = box_node<NQ>(l, nx, ny, nz);
    if (bn.masked) {
        b[l] = 0.0;
        return;
    }
    const int z0 = bn.sz < 0 ? bn.oz : 0, z1 = bn.sz > 0 ? bn.oz : 0;
    const int y0 = bn.sy < 0 ? bn.oy : 0, y1 = bn.sy > 0 ? bn.oy : 0;
    const int x0 = bn.sx < 0 ? bn.ox : 0, x1 = bn.sx > 0 ? bn.ox : 0;
    double s = 0.0;
    bool first = true;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int cz = c >> 2, cy = (c >> 1) & 1, cx = c & 1;
        if (!((cz == 0 || bn.sz) && (cy == 0 || bn.sy) && (cx == 0 || bn.sx))) continue;
        const double v = f[l + (cz ? z1 : z0) + (cy ? y1 : y0) + (cx ? x1 : x0)];
        s = first ? v : s + v;
        first = false;
    }
    b[l] = s;
}

// One CG update step over all local nodes (grid-stride), with the <r, r>
// reduction: per-thread partials and block sums in Acc, the grid sum in FP64
// over groups of blocks, and the block that completes it closes the
// iteration (beta, counter, stop flag).  Bounded to 48
// registers so that 5 blocks of 256 threads stay resident per SM: the FP32
// step is latency-bound (E = 32^3, N = 7: inner iteration -3 %).
template <int NQ, typename T, typename Acc>
__global__ void __launch_bounds__(256, 5) cg_update_nodes_kernel(T *__restrict__ x, T *__restrict__ r,
                                                              const T *__restrict__ p, const T *__restrict__ w,
                                                              int nL, BoxDims bd, double *partials, CgState *st) {
    __shared__ double scratch[256];
    if (st->done) return;
    const T alpha = T(st->alpha);
    Acc acc = acc_zero<Acc>();
    constexpr int V = UpdVec<NQ, T>::value;
    const int nv = nL / V;   // nL is a multiple of (N+1), hence of V
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nv; u += gridDim.x * blockDim.x)
        update_vec<NQ, V, T, Acc>(x, r, p, w, u * V, bd, alpha, acc);
    // all blocks of the resident wave reach this point together: block sums
    // in Acc when it is FP32, one warp's FP64 sum otherwise, grid sum in groups
    double bs;
    if constexpr (std::is_same<Acc, float>::value)
        bs = double(block_sum_f32(acc, reinterpret_cast<float *>(scratch)));
    else
        bs = block_sum_wide(acc_value(acc), scratch);
    if (publish_grouped(bs, partials, &st->ticket_up)) {
        const double rho_new = finish_grouped(partials, &st->ticket_up);
        if (threadIdx.x == 0) cg_close_iteration(st, rho_new);
    }
}

// The same step with the row-class mapping (RowMap): used where the
// arithmetic pipe, not HBM, bounds the update (FP64 on GB300).
template <int NQ, typename T, typename Acc>
__global__ void __launch_bounds__(256) cg_update_class_kernel(T *__restrict__ x, T *__restrict__ r,
                                                              const T *__restrict__ p, const T *__restrict__ w,
                                                              int nL, BoxDims bd, double *partials, CgState *st) {
    __shared__ double scratch[256];
    if (st->done) return;
    constexpr int V = UpdVec<NQ, T>::value;
    using RM = RowMap<NQ, V>;
    const T alpha = T(st->alpha);
    const int E = nL / RM::NP;
    const int ntask = RM::tasks(E);
    const int lane = threadIdx.x & 31;
    const int nwarps = int(gridDim.x * blockDim.x) >> 5;
    Acc acc = acc_zero<Acc>();
    for (int task = int(blockIdx.x * blockDim.x + threadIdx.x) >> 5; task < ntask; task += nwarps) {
        const int l0 = RM::l0(task, lane, E);
        if (l0 >= 0) update_vec<NQ, V, T, Acc, false, true>(x, r, p, w, l0, bd, alpha, acc);
    }
    // one warp's FP64 sum per block (13 instead of 40 warp-wide FP64 adds),
    // grid sum in groups
    const double bs = block_sum_wide(acc_value(acc), scratch);
    if (publish_grouped(bs, partials, &st->ticket_up)) {
        const double rho_new = finish_grouped(partials, &st->ticket_up);
        if (threadIdx.x == 0) cg_close_iteration(st, rho_new);
    }
}

// Blocks of an update launch, grid-stride beyond.  Measured on GB300 at
// E = 32^3, N = 7: the FP32 update is fastest with one resident wave
// (inner CG iteration 216 -> 190 us); the FP64 update with 8 blocks per SM
// (230 us; one wave of 5 per SM: 293 us; one vector per thread, 32768
// blocks: 340 us -- each block's FP64 reduction costs more than the latency
// it hides).
template <typename K>
static int64_t resident_blocks(K kern, int threads) {
    static int per_sm = 0;
    if (!per_sm) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0) != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            per_sm = 4;
        }
    }
    return int64_t(per_sm) * sm_count();
}

template <int NQ, typename T, typename Acc>
static int launch_update_rows_nq(const Problem *P, T *x, T *r, const T *p, const T *w, CgState *st) {
    constexpr int V = UpdVec<NQ, T>::value;
    if constexpr (sizeof(T) == 8) {
        using RM = RowMap<NQ, V>;
        int64_t blocks = (int64_t(RM::tasks(int(P->E))) * 32 + 255) / 256;
        blocks = std::min<int64_t>(blocks, int64_t(sm_count()) * 8);
        cg_update_class_kernel<NQ, T, Acc><<<unsigned(blocks), 256, 0, stream()>>>(
            x, r, p, w, int(P->nL), box_dims(P->nx, P->ny, P->nz), P->partials, st);
        count_launches(1);
        return cuda_check(cudaGetLastError(), "cg_update_class_kernel");
    }
    int64_t blocks = (P->nL / V + 255) / 256;
    blocks = std::min(blocks, resident_blocks(cg_update_nodes_kernel<NQ, T, Acc>, 256));
    cg_update_nodes_kernel<NQ, T, Acc><<<unsigned(blocks), 256, 0, stream()>>>(
        x, r, p, w, int(P->nL), box_dims(P->nx, P->ny, P->nz), P->partials, st);
    count_launches(1);
    return cuda_check(cudaGetLastError(), "cg_update_nodes_kernel");
}

template <typename T, typename Acc>
static int launch_update_rows(const Problem *P, T *x, T *r, const T *p, const T *w, CgState *st) {
    switch (P->nq) {
        case 2: return launch_update_rows_nq<2, T, Acc>(P, x, r, p, w, st);
        case 3: return launch_update_rows_nq<3, T, Acc>(P, x, r, p, w, st);
        case 4: return launch_update_rows_nq<4, T, Acc>(P, x, r, p, w, st);
        case 5: return launch_update_rows_nq<5, T, Acc>(P, x, r, p, w, st);
        case 6: return launch_update_rows_nq<6, T, Acc>(P, x, r, p, w, st);
        case 7: return launch_update_rows_nq<7, T, Acc>(P, x, r, p, w, st);
        case 8: return launch_update_rows_nq<8, T, Acc>(P, x, r, p, w, st);
        case 9: return launch_update_rows_nq<9, T, Acc>(P, x, r, p, w, st);
        case 10: return launch_update_rows_nq<10, T, Acc>(P, x, r, p, w, st);
        default: return set_error(SEM_EARG, "cg: unsupported order");
    }
}

}  // namespace sem
