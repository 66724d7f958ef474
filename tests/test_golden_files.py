"""Stored oracle outputs are what their committed scripts write (no GPU).

tests/golden/oracle_cg_E64_N7.npz holds the oracle's CG solution of the
small FP64 workload (bench.py states the GPU solves' error against it); a
fresh run of tests/golden/make_oracle_cg.py must reproduce it (to rounding:
libm's sin may differ between hosts).
"""
import os
import sys

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_oracle_cg_solution_matches_a_fresh_run(oracle_mod):
    sys.path.insert(0, HERE)
    import make_oracle_cg
    stored = np.load(os.path.join(HERE, "oracle_cg_E64_N7.npz"))
    fresh = make_oracle_cg.solve()
    assert int(stored["iters"]) == int(fresh["iters"])
    for key in ("b", "x"):
        a, b = stored[key], fresh[key]
        assert a.shape == b.shape
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max(), key
    assert float(stored["true_rel_res"]) <= 1.5e-12
