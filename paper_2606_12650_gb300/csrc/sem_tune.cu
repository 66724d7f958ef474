// sem_tune.cu -- the per-order tuner of the local operator.
//
// The paper's runtime specialises kernels on values known at run time (its
// "jit" clause fixes N, Section VIII-B) and lets transformation scripts
// choose the thread layout.  Here the variants are compiled ahead of time for
// every order and the choice is made by timing: for one order and one
// precision, each candidate -- the column kernel, the persistent kernel
// (FP32), the line kernel at several element-per-block counts, and for FP64
// the line kernel in double-word FP32 arithmetic -- runs
// the CG operator `reps` times on a real problem, and the fastest is kept.
// The table can be saved to and loaded from a text file (one line per entry:
// kind, N, variant, elements per block, microseconds), so a tuned table is
// reused by later runs (`sem_init --autotune-table=PATH`).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "sem_device.cuh"
#include "sem_internal.h"

namespace sem {
namespace {

TuneChoice g_tab[kTuneKinds][kMaxQ + 1];
bool g_init = false;
uint64_t g_epoch = 1;

// Built-in table: the winners of tuning runs on GB300 with ~17 M local
// nodes per problem (E = 129^3 at N = 1 down to 26^3 at N = 9; CG operator,
// 10 launches per candidate), as {variant, elements per block} indexed by
// N + 1 (entries 0 and 1 unused); the run-time tuner replaces entries for
// the problems at hand.  FP64: the double-word line kernel at every order
// (e.g. N = 3: 281 us against 1203 us for the DFMA line kernel; N = 7: 371
// against 1579; N = 9: 576 against 2117).
struct DefaultEntry {
    int variant, epb;
};
constexpr DefaultEntry kDefault[kTuneKinds][kMaxQ + 1] = {
    // FP64
    {{0, 0}, {0, 0}, {5, 32}, {5, 14}, {5, 8}, {5, 5}, {5, 7}, {5, 5}, {5, 4}, {5, 3}, {5, 5}},
    // FP32, FP32 factors
    {{2, 0}, {2, 0}, {2, 0}, {2, 0}, {2, 0}, {1, 10}, {1, 10}, {1, 5}, {1, 3}, {1, 3}, {1, 2}},
    // FP32, BF16 factors
    {{2, 0}, {2, 0}, {2, 0}, {2, 0}, {2, 0}, {1, 10}, {4, 7}, {1, 5}, {1, 2}, {1, 1}, {1, 2}},
};

TuneChoice default_choice(int kind, int nq) {
    if (kind < 0 || kind >= kTuneKinds || nq < 0 || nq > kMaxQ) return {kAxColumns, 0, 0.0};
    return {kDefault[kind][nq].variant, kDefault[kind][nq].epb, 0.0};
}

void ensure_init() {
    if (g_init) return;
    for (int k = 0; k < kTuneKinds; ++k)
        for (int q = 0; q <= kMaxQ; ++q) g_tab[k][q] = default_choice(k, q);
    g_init = true;
}

size_t elem_bytes(int kind) { return kind == kTuneF64 ? sizeof(double) : sizeof(float); }

bool choice_ok(int kind, int nq, const TuneChoice &c) {
    if (kind < 0 || kind >= kTuneKinds || nq < 2 || nq > kMaxQ) return false;
    switch (c.variant) {
        case kAxColumns: return kind == kTuneF64;
        case kAxPersistent: return kind != kTuneF64;
        case kAxLines: return lines_epb_ok(nq, c.epb, elem_bytes(kind));
        case kAxLinesPrefetch: return kind == kTuneF32G16 && lines_epb_ok(nq, c.epb, elem_bytes(kind));
        case kAxLinesStaged:
            return kind != kTuneF64 && lines_epb_ok(nq, c.epb, elem_bytes(kind), kind == kTuneF32G32 ? 24 : 12);
        case kAxLinesDW: return kind == kTuneF64 && lines_epb_ok(nq, c.epb, sizeof(double));
        default: return false;
    }
}

// The candidates for (kind, nq): the kind's column kernel, then the line
// kernel with ~64 .. 512 threads per block (for FP64 also in double-word
// arithmetic; for FP32 with staged factors and, for BF16 factors, with the
// factors prefetched).
int candidates(int kind, int nq, TuneChoice *out, int cap) {
    int n = 0;
    out[n++] = {kind == kTuneF64 ? kAxColumns : kAxPersistent, 0, 0.0};
    const bool f64 = kind == kTuneF64;
    const int variants[3] = {kAxLines, f64 ? kAxLinesDW : kAxLinesStaged, kAxLinesPrefetch};
    const int nv = f64 ? 2 : (kind == kTuneF32G32 ? 2 : 3);
    for (int v = 0; v < nv; ++v) {
        int prev = 0;
        for (int t : {64, 128, 192, 256, 384, 512}) {
            int epb = t / (nq * nq);
            if (epb < 1) epb = 1;
            const TuneChoice c{variants[v], epb, 0.0};
            if (epb != prev && choice_ok(kind, nq, c) && n < cap) out[n++] = c;
            prev = epb;
        }
    }
    return n;
}

template <typename T>
__global__ void tune_fill_kernel(T *r, T *p, int64_t n) {
    for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < n; q += int64_t(gridDim.x) * blockDim.x) {
        r[q] = T(1 + (q & 7) * 0.125);
        p[q] = T(0);
    }
}

__global__ void tune_state_kernel(CgState *st, double *partials) {
    reset_group_tickets(partials);
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    st->alpha = 0.0;
    st->beta = 0.0;
    st->rho = 1.0;
    st->done = 0;
    st->ticket_ax = 0;
}

}  // namespace

int tune_kind_of_gprec(int gprec) { return gprec == kGF32 ? kTuneF32G32 : kTuneF32G16; }

TuneChoice tune_get(int kind, int nq) {
    ensure_init();
    if (kind < 0 || kind >= kTuneKinds || nq < 0 || nq > kMaxQ) return default_choice(kTuneF64, 2);
    return g_tab[kind][nq];
}

void tune_set(int kind, int nq, const TuneChoice &c) {
    ensure_init();
    if (kind < 0 || kind >= kTuneKinds || nq < 0 || nq > kMaxQ) return;
    g_tab[kind][nq] = c;
    ++g_epoch;
}

void tune_reset() {
    g_init = false;
    ensure_init();
    ++g_epoch;
}

uint64_t tune_epoch() { return g_epoch; }

int tune_check(int kind, int nq, const TuneChoice &c) {
    if (kind < 0 || kind >= kTuneKinds) return set_error(SEM_EARG, "autotune: kind must be 0 (FP64), 1 or 2 (FP32)");
    if (nq < 2 || nq > kMaxQ) return set_error(SEM_EARG, "autotune: N must be in [1, 9]");
    if (!choice_ok(kind, nq, c)) return set_error(SEM_EARG, "autotune: variant not available for this kind and N");
    return SEM_OK;
}

int tune_problem(Problem *P, int kind, int reps, double *cand, int cap, int *n_cand, TuneChoice *best) {
    if (kind < 0 || kind >= kTuneKinds) return set_error(SEM_EARG, "autotune: kind must be 0 (FP64), 1 or 2 (FP32)");
    if (reps < 1 || reps > 10000) return set_error(SEM_EARG, "autotune: reps must be in [1, 10000]");
    const int nq = P->nq;
    const int gprec = kind == kTuneF32G32 ? kGF32 : kGBF16;
    int rc = kind != kTuneF64 ? mixed_prepare(P, gprec) : dw_prepare(P);
    if (rc != SEM_OK) return rc;
    CgState *st = kind == kTuneF64 ? P->st : P->st_in;
    unsigned blocks = unsigned(std::min<int64_t>((P->nL + 255) / 256, int64_t(sm_count()) * 8));
    if (kind == kTuneF64)
        tune_fill_kernel<double><<<blocks, 256, 0, stream()>>>(P->r, P->p, P->nL);
    else
        tune_fill_kernel<float><<<blocks, 256, 0, stream()>>>(P->r32, P->p32, P->nL);
    tune_state_kernel<<<1, 256, 0, stream()>>>(st, P->partials);
    count_launches(2);
    rc = cuda_check(cudaGetLastError(), "autotune: set-up");
    if (rc != SEM_OK) return rc;

    TuneChoice list[24];
    const int n = candidates(kind, nq, list, 24);
    const TuneChoice saved = tune_get(kind, nq);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    rc = cuda_check(cudaEventCreate(&e0), "autotune: event");
    if (rc == SEM_OK) rc = cuda_check(cudaEventCreate(&e1), "autotune: event");
    int ibest = -1;
    auto launch = [&]() { return kind == kTuneF64 ? launch_ax_cg(P) : launch_ax32_cg(P, gprec); };
    for (int c = 0; c < n && rc == SEM_OK; ++c) {
        g_tab[kind][nq] = list[c];   // no epoch bump while timing
        for (int w = 0; w < 2 && rc == SEM_OK; ++w) rc = launch();
        if (rc == SEM_OK) rc = cuda_check(cudaEventRecord(e0, stream()), "autotune: record");
        for (int k = 0; k < reps && rc == SEM_OK; ++k) rc = launch();
        if (rc == SEM_OK) rc = cuda_check(cudaEventRecord(e1, stream()), "autotune: record");
        if (rc == SEM_OK) rc = cuda_check(cudaEventSynchronize(e1), "autotune: sync");
        float ms = 0.f;
        if (rc == SEM_OK) rc = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "autotune: elapsed");
        if (rc != SEM_OK) break;
        list[c].us = 1e3 * double(ms) / reps;
        if (ibest < 0 || list[c].us < list[ibest].us) ibest = c;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc == SEM_OK) rc = poll_status();
    if (rc != SEM_OK || ibest < 0) {
        tune_set(kind, nq, saved);
        return rc != SEM_OK ? rc : set_error(SEM_ECUDA, "autotune: no candidate ran");
    }
    tune_set(kind, nq, list[ibest]);
    if (cand)
        for (int c = 0; c < n && c < cap; ++c) {
            cand[3 * c] = list[c].variant;
            cand[3 * c + 1] = list[c].epb;
            cand[3 * c + 2] = list[c].us;
        }
    *n_cand = n;
    *best = list[ibest];
    return SEM_OK;
}

int tune_save(const char *path) {
    ensure_init();
    FILE *f = fopen(path, "w");
    if (!f) return set_error(SEM_EARG, std::string("autotune_save: cannot write ") + path);
    fprintf(f, "# libsem operator table: kind(0 fp64, 1 fp32/fp32 G, 2 fp32/bf16 G) N variant(0 columns, "
               "1 lines, 2 persistent, 3 lines with G prefetch, 4 lines with G staged, 5 lines in double-word FP32) "
               "elements_per_block us\n");
    for (int k = 0; k < kTuneKinds; ++k)
        for (int q = 2; q <= kMaxQ; ++q) {
            const TuneChoice &c = g_tab[k][q];
            fprintf(f, "%d %d %d %d %.3f\n", k, q - 1, c.variant, c.epb, c.us);
        }
    const bool ok = fclose(f) == 0;
    return ok ? SEM_OK : set_error(SEM_EARG, std::string("autotune_save: write failed for ") + path);
}

int tune_load(const char *path) {
    FILE *f = fopen(path, "r");
    if (!f) return set_error(SEM_EARG, std::string("autotune table: cannot read ") + path);
    ensure_init();
    TuneChoice tab[kTuneKinds][kMaxQ + 1];
    memcpy(tab, g_tab, sizeof tab);
    char line[256];
    int lineno = 0, rc = SEM_OK;
    while (fgets(line, sizeof line, f)) {
        ++lineno;
        const char *s = line;
        while (*s == ' ' || *s == '\t') ++s;
        if (*s == '#' || *s == '\n' || *s == '\r' || *s == 0) continue;
        int kind, N, variant, epb;
        double us = 0.0;
        const int got = sscanf(s, "%d %d %d %d %lf", &kind, &N, &variant, &epb, &us);
        const int nq = N + 1;
        const TuneChoice c{variant, epb, got >= 5 ? us : 0.0};
        if (got < 4 || !choice_ok(kind, nq, c)) {
            rc = set_error(SEM_EARG, std::string("autotune table ") + path + ": bad entry on line " +
                                         std::to_string(lineno));
            break;
        }
        tab[kind][nq] = c;
    }
    fclose(f);
    if (rc != SEM_OK) return rc;
    memcpy(g_tab, tab, sizeof tab);
    ++g_epoch;
    return SEM_OK;
}

}  // namespace sem
