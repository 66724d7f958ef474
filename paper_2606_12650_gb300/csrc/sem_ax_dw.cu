// sem_ax_dw.cu -- the double-word FP64 operator (sem_ax_dw.cuh): its
// geometric factors in double-word form, its coefficients, and its launches
// (plain y = A_local x, the CG operator and the Jacobi-PCG operator, for
// every order, elements per block chosen at launch).
#include "sem_ax_dw.cuh"

namespace sem {

// Gdw[2 (6 l + c)] = rn(G), Gdw[2 (6 l + c) + 1] = rn(G - rn(G)).
__global__ void geometry_dw_kernel(const double *__restrict__ G, float *__restrict__ Gdw, int64_t n) {
    for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < n; q += int64_t(gridDim.x) * blockDim.x) {
        const double g = G[q];
        const float h = __double2float_rn(g);
        Gdw[2 * q] = h;
        Gdw[2 * q + 1] = __double2float_rn(g - double(h));
    }
}

int dw_prepare(Problem *P) {
    if (P->Gdw) return SEM_OK;
    float *g = static_cast<float *>(dev_alloc(sizeof(float) * 12 * size_t(P->nL)));
    if (!g) return SEM_ENOMEM;
    const int64_t n = 6 * P->nL;
    const unsigned blocks = unsigned(std::min<int64_t>((n + 255) / 256, int64_t(sm_count()) * 16));
    geometry_dw_kernel<<<blocks, 256, 0, stream()>>>(P->G, g, n);
    count_launches(1);
    const int rc = cuda_check(cudaGetLastError(), "geometry_dw_kernel");
    if (rc != SEM_OK) {
        dev_free(g);
        return rc;
    }
    P->Gdw = g;
    return SEM_OK;
}

void dw_release(Problem *P) {
    if (P->Gdw) dev_free(P->Gdw);
    P->Gdw = nullptr;
}

template <int NQ, bool CG, bool PRE>
static int launch_dw_nq(const Problem *Pb, const AxDwArgs &L) {
    const int nt = line_threads(NQ, L.epb);
    if (L.epb < 1 || nt == 0) return set_error(SEM_EARG, "ax dw: elements per block out of range");
    const size_t sm = LineShape::smem(NQ, L.epb, int(sizeof(double)));
    if (sm > size_t(227) * 1024) return set_error(SEM_EARG, "ax dw: shared memory per block too large");
    auto kern = ax_dw_kernel<NQ, CG, PRE>;
    // raise the dynamic shared-memory limit when a larger block is first
    // asked for (the tuner and the first solve do so before any capture)
    static size_t sm_set = 0;
    if (sm > sm_set) {
        const int rc = cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)),
                                  "ax dw: smem attribute");
        if (rc != SEM_OK) return rc;
        sm_set = sm;
    }
    const int64_t blocks = (Pb->E + L.epb - 1) / L.epb;
    if (CG && blocks > Pb->partials_cap) return set_error(SEM_ERANGE, "ax dw: more blocks than reduction slots");
    kern<<<unsigned(blocks), nt, sm, stream()>>>(L);
    count_launches(1);
    return cuda_check(cudaGetLastError(), "ax_dw_kernel");
}

template <bool CG, bool PRE>
static int launch_dw_any(const Problem *Pb, const AxDwArgs &L) {
    switch (Pb->nq) {
        case 2: return launch_dw_nq<2, CG, PRE>(Pb, L);
        case 3: return launch_dw_nq<3, CG, PRE>(Pb, L);
        case 4: return launch_dw_nq<4, CG, PRE>(Pb, L);
        case 5: return launch_dw_nq<5, CG, PRE>(Pb, L);
        case 6: return launch_dw_nq<6, CG, PRE>(Pb, L);
        case 7: return launch_dw_nq<7, CG, PRE>(Pb, L);
        case 8: return launch_dw_nq<8, CG, PRE>(Pb, L);
        case 9: return launch_dw_nq<9, CG, PRE>(Pb, L);
        case 10: return launch_dw_nq<10, CG, PRE>(Pb, L);
        default: return set_error(SEM_EARG, "ax dw: unsupported order");
    }
}

int launch_lines_dw(const Problem *P, const double *x, double *y, int mode, int epb) {
    if (!lines_epb_ok(P->nq, epb, sizeof(double))) return set_error(SEM_EARG, "ax dw: bad elements per block");
    if (!P->Gdw) return set_error(SEM_EARG, "ax dw: double-word factors not prepared (dw_prepare)");
    AxDwArgs L{};
    L.a = ax_args<double, double>(P, P->G, P->partials, P->st);
    L.Gdw = P->Gdw;
    double Dt[kMaxQ * kMaxQ];
    for (int i = 0; i < P->nq; ++i)
        for (int l = 0; l < P->nq; ++l) Dt[i * P->nq + l] = P->oc.D[l * P->nq + i];
    L.d = eo_coefficients_dw(P->oc.D, P->nq);
    L.dt = eo_coefficients_dw(Dt, P->nq);
    L.epb = epb;
    if (mode == 0) {
        L.a.x = x;
        L.a.y = y;
        return launch_dw_any<false, false>(P, L);
    }
    L.a.x = P->r;
    L.a.y = P->w;
    L.a.p = P->p;
    L.a.xs = P->x;   // x += alpha p of the previous iteration
    if (mode == 1) return launch_dw_any<true, false>(P, L);
    L.a.dinv = P->dinv;
    return launch_dw_any<true, true>(P, L);
}

}  // namespace sem
