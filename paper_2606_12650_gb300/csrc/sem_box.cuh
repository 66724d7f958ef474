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

#include <cstdint>

namespace sem {

struct BoxNode {
    int sx, sy, sz;     // -1 low face, +1 high face, 0 interior (per direction)
    int ox, oy, oz;     // signed local-index offsets to the neighbour copies
    bool masked;        // on the cube boundary
    bool owner;         // first copy of its global node
};

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

// Sum of v over the copies of node l, in ascending local index.
template <typename T, typename Acc>
__device__ __forceinline__ Acc box_sum(const T *__restrict__ v, int l, const BoxNode &b) {
    const int nzo = b.sz ? 2 : 1, nyo = b.sy ? 2 : 1, nxo = b.sx ? 2 : 1;
    Acc s = Acc(0);
    bool first = true;
    for (int cz = 0; cz < nzo; ++cz) {
        const int dz = (nzo == 2 && ((b.sz < 0) == (cz == 0))) ? b.oz : 0;
        for (int cy = 0; cy < nyo; ++cy) {
            const int dy = (nyo == 2 && ((b.sy < 0) == (cy == 0))) ? b.oy : 0;
            for (int cx = 0; cx < nxo; ++cx) {
                const int dx = (nxo == 2 && ((b.sx < 0) == (cx == 0))) ? b.ox : 0;
                const Acc val = Acc(__ldg(v + l + dz + dy + dx));
                s = first ? val : s + val;
                first = false;
            }
        }
    }
    return s;
}

}  // namespace sem

namespace sem {

// Fused direct-stiffness sum + CG update over element rows.  A row is the
// NQ nodes (i = 0..N) of one (j, k) line of one element: contiguous in
// memory, so a warp's rows form one contiguous run.  For a row, the copies of
// its nodes across the s and t faces are whole rows of the neighbouring
// elements (loaded as rows); only the two end nodes also have copies across
// the r faces (single values).  Every copy of a node sums the same list in
// ascending local index, so all copies get the same bits; each copy updates
// only itself:  x += alpha p,  r -= alpha (QQ^T w).  Masked nodes are left
// unchanged (they stay zero).  Returns this thread's partial of <r, r> over
// the rows it owns (each global node counted at its first copy).
template <int NQ, typename T, typename Acc>
__device__ __forceinline__ Acc update_row(T *__restrict__ x, T *__restrict__ r, const T *__restrict__ p,
                                         const T *__restrict__ w, int row, int nx, int ny, int nz, T alpha) {
    constexpr int N = NQ - 1, NQ2 = NQ * NQ, NP = NQ2 * NQ;
    const unsigned e = unsigned(row) / unsigned(NQ2);
    const int jk = row - int(e) * NQ2;
    const int j = jk % NQ, k = jk / NQ;
    const unsigned t = e / unsigned(nx);
    const int ex = int(e - t * unsigned(nx));
    const unsigned tz = t / unsigned(ny);
    const int ey = int(t - tz * unsigned(ny)), ez = int(tz);
    const int sy = j == 0 ? -1 : (j == N ? 1 : 0);
    const int sz = k == 0 ? -1 : (k == N ? 1 : 0);
    if ((sy < 0 && ey == 0) || (sy > 0 && ey == ny - 1) || (sz < 0 && ez == 0) || (sz > 0 && ez == nz - 1))
        return Acc(0);                                   // the whole row is on the cube boundary
    const int base = row * NQ;
    const int oy = sy * (nx * NP - N * NQ);
    const int oz = sz * (nx * ny * NP - N * NQ2);
    const bool xlo = ex > 0, xhi = ex < nx - 1;          // r-face neighbours exist
    const int nzo = sz ? 2 : 1, nyo = sy ? 2 : 1;
    // Copies across the t and s faces are whole rows; visit the (t, s)
    // choices in ascending element order (t major, lower element first) and
    // accumulate every node's sum in place.
    Acc ws[NQ];
#pragma unroll
    for (int i = 0; i < NQ; ++i) ws[i] = Acc(0);
    bool first = true;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int cz = c >> 1, cy = c & 1;
        if (cz >= nzo || cy >= nyo) continue;
        const int dz = (nzo == 2 && ((sz < 0) == (cz == 0))) ? oz : 0;
        const int dy = (nyo == 2 && ((sy < 0) == (cy == 0))) ? oy : 0;
        const T *wc = w + base + dz + dy;
        const Acc lo = xlo ? Acc(__ldg(wc - (NP - N))) : Acc(0);   // element ex-1, node i = N
        const Acc hi = xhi ? Acc(__ldg(wc + NP)) : Acc(0);         // element ex+1, node i = 0
#pragma unroll
        for (int i = 0; i < NQ; ++i) {
            const Acc v = Acc(__ldg(wc + i));
            Acc s = ws[i];
            if (i == 0 && xlo) s = first ? lo : s + lo;
            s = (first && !(i == 0 && xlo)) ? v : s + v;
            if (i == N && xhi) s = s + hi;
            ws[i] = s;
        }
        first = false;
    }
    const bool owner_row = sy >= 0 && sz >= 0;
    Acc acc = Acc(0);
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        const bool masked = (i == 0 && !xlo) || (i == N && !xhi);
        if (masked) continue;
        const T xn = fma(alpha, p[base + i], x[base + i]);
        const T rn = fma(-alpha, T(ws[i]), r[base + i]);
        x[base + i] = xn;
        r[base + i] = rn;
        const bool owner = owner_row && !(i == 0 && xlo);
        if (owner) acc = fma(Acc(rn), Acc(rn), acc);
    }
    return acc;
}

}  // namespace sem

#include "sem_device.cuh"

namespace sem {

// One CG update step over all element rows (grid-stride), with the <r, r>
// reduction: per-thread partials in Acc, block and grid sums in FP64, and the
// last block closes the iteration (beta, counter, stop flag).
template <int NQ, typename T, typename Acc>
__global__ void __launch_bounds__(256) cg_update_rows_kernel(T *__restrict__ x, T *__restrict__ r,
                                                             const T *__restrict__ p, const T *__restrict__ w,
                                                             int nrows, int nx, int ny, int nz, double *partials,
                                                             CgState *st) {
    __shared__ double red[32];
    if (st->done) return;
    const T alpha = T(st->alpha);
    Acc acc = Acc(0);
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < nrows; row += gridDim.x * blockDim.x)
        acc += update_row<NQ, T, Acc>(x, r, p, w, row, nx, ny, nz, alpha);
    const double bs = block_sum(double(acc), red);
    if (publish_partial(bs, partials, &st->ticket_up)) {
        const double rho_new = finish_partials(partials, int(gridDim.x), &st->ticket_up, red);
        if (threadIdx.x == 0) cg_close_iteration(st, rho_new);
    }
}

template <int NQ, typename T, typename Acc>
static int launch_update_rows_nq(const Problem *P, T *x, T *r, const T *p, const T *w, CgState *st) {
    const int64_t nrows = P->E * NQ * NQ;
    int64_t blocks = (nrows + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;   // grid-stride: ~7 rows per thread at E = 32768, N = 7
    cg_update_rows_kernel<NQ, T, Acc><<<unsigned(blocks), 256, 0, stream()>>>(x, r, p, w, int(nrows), P->nx, P->ny,
                                                                              P->nz, P->partials, st);
    count_launches(1);
    return cuda_check(cudaGetLastError(), "cg_update_rows_kernel");
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
