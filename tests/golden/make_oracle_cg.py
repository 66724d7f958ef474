"""Write the oracle's converged CG solution of the small FP64 workload.

The workload is the 4 x 4 x 4 box (E = 64) of order N = 7, interior vertices
jittered by +-5 % (seed 1), Dirichlet boundary, right-hand side from the
manufactured u = sin(pi x) sin(pi y) sin(pi z) (b = mask(QQ^T(B f)),
f = 3 pi^2 u), solved by the oracle's unpreconditioned CG from x = 0 to
sqrt(<r,r>/<b,b>) <= 1e-12 (the CG of Nekbone without preconditioner,
Section VIII-A).  bench.py reads the stored b and x to state the error of the
GPU solves (FP64 and mixed precision) against the FP64 oracle without running
the oracle itself.  This script calls only ``oracle/`` and the seeded input
generators; tests/test_golden_files.py checks the stored file against a fresh
run.

    python tests/golden/make_oracle_cg.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "oracle_cg_E64_N7.npz")
NX, N, SEED, TOL = 4, 7, 1, 1e-12


def solve():
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2606_12650_gb300.inputs import box_vertices
    verts = box_vertices(NX, NX, NX, 0.05, seed=SEED)
    P = oracle.Problem(NX, NX, NX, N, verts)
    b = P.rhs_sin()
    x, iters, hist = P.cg(b, maxit=20000, tol=TOL)
    return {"b": b, "x": x, "iters": np.int64(iters), "rel_res": np.float64(hist[-1] / hist[0]),
            "true_rel_res": np.float64(P.true_residual(b, x)), "nx": np.int64(NX), "N": np.int64(N),
            "seed": np.int64(SEED), "tol": np.float64(TOL)}


if __name__ == "__main__":
    d = solve()
    np.savez_compressed(OUT, **d)
    print(f"wrote {OUT}: {int(d['iters'])} iterations, rel. residual {float(d['rel_res']):.3e}")
