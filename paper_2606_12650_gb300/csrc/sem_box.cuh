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
