// sem_box.cuh -- copies of a global node on the structured box mesh.
//
// On an nx x ny x nz box of order N, local node (e; i, j, k) of element
// (ex, ey, ez) shares its global node with the elements across every element
// face it lies on: along r when i = 0 (element ex-1, at i = N) or i = N
// (element ex+1, at i = 0), and likewise along s and t.  Nodes on the cube
// boundary are Dirichlet (masked).  The copies are listed in ascending local
// index, which is the (ez, ey, ex) lexicographic order of their elements, so a
// left-to-right sum over the list adds in the same order as the sorted-segment
// gather-scatter and gives the same bits at every copy.
#pragma once

#include <cstdint>

namespace sem {

struct BoxCopies {
    int64_t l[8];   // local indices of the copies, ascending
    int n;          // number of copies (0 for a masked node)
    bool owner;     // the node itself is the first copy
};

template <int NQ>
__device__ __forceinline__ BoxCopies box_copies(int64_t node, int nx, int ny, int nz) {
    constexpr int N = NQ - 1, NQ2 = NQ * NQ, NP = NQ2 * NQ;
    const int64_t e = node / NP;
    const int q = int(node - e * NP);
    const int i = q % NQ, j = (q / NQ) % NQ, k = q / NQ2;
    const int ex = int(e % nx);
    const int64_t eyz = e / nx;
    const int ey = int(eyz % ny), ez = int(eyz / ny);
    BoxCopies out;
    out.n = 0;
    out.owner = false;
    // per direction: the elements sharing the node (ascending) and the node's
    // index inside each of them
    int ce[3][2], ci[3][2], cnt[3];
    const int idx[3] = {i, j, k}, el[3] = {ex, ey, ez}, ne[3] = {nx, ny, nz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        cnt[d] = 1;
        ce[d][0] = el[d];
        ci[d][0] = idx[d];
        if (idx[d] == 0) {
            if (el[d] == 0) return out;                 // on the cube boundary: masked
            ce[d][0] = el[d] - 1; ci[d][0] = N;
            ce[d][1] = el[d];     ci[d][1] = 0;
            cnt[d] = 2;
        } else if (idx[d] == N) {
            if (el[d] == ne[d] - 1) return out;         // masked
            ce[d][0] = el[d];     ci[d][0] = N;
            ce[d][1] = el[d] + 1; ci[d][1] = 0;
            cnt[d] = 2;
        }
    }
    out.owner = ce[0][0] == ex && ce[1][0] == ey && ce[2][0] == ez;
    for (int c = 0; c < cnt[2]; ++c)
        for (int b = 0; b < cnt[1]; ++b)
            for (int a = 0; a < cnt[0]; ++a) {
                const int64_t e2 = ce[0][a] + int64_t(nx) * (ce[1][b] + int64_t(ny) * ce[2][c]);
                out.l[out.n++] = e2 * NP + ci[0][a] + NQ * (ci[1][b] + NQ * ci[2][c]);
            }
    return out;
}

}  // namespace sem
