"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of ``oracle/sem_oracle.c`` (on the CPU,
in a temporary directory), builds it, and runs the pin suite against it with
``SEM_ORACLE_LIB`` pointing at the broken library.  The suite must fail.  A
case may name the pins (a ``-k`` expression) that must catch it on their own.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sem_oracle.c")

MUTATIONS = {
    "transposed_D_in_second_stage": ("acc += D[m * n + i] * wr", "acc += D[i * n + m] * wr"),
    "dropped_cross_term": ("wr[q] = g[0] * ur + g[1] * us + g[2] * ut;",
                           "wr[q] = g[0] * ur + g[1] * us;"),
    "cofactor_sign": ("cof[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];",
                      "cof[0][1] = J[1][0] * J[2][2] - J[1][2] * J[2][0];"),
    "wrong_lattice_index": ("gy = (long)ey * N + j", "gy = (long)ey * N + i"),
    "gll_weight_formula": ("w[j] = 2.0 / (N * (N + 1.0) * P * P);",
                           "w[j] = 2.0 / ((N + 1.0) * (N + 1.0) * P * P);"),
    "D_corner_entry": ("v = N * (N + 1.0) / 4.0;", "v = N * (N + 1.0) / 2.0;"),
    "cg_beta_inverted": ("for (long l = 0; l < nL; ++l) p[l] = r[l] + beta * p[l];",
                         "for (long l = 0; l < nL; ++l) p[l] = r[l] + (1.0 / beta) * p[l];"),
    "gs_last_copy_wins": ("else sum[g] += u[l];", "else sum[g] = u[l];"),
    "mask_misses_a_face": ("gz == 0 || gz == mz", "gz == 0"),
    "geometry_weight_missing": ("double W = w[i] * w[j] * w[k];", "double W = w[i] * w[j];"),
    "pcg_unpreconditioned_z": ("for (long l = 0; l < nL; ++l) z[l] = dinv[l] * r[l];",
                               "for (long l = 0; l < nL; ++l) z[l] = r[l];"),
    "diag_wrong_entry": ("d[(long)np * e + q] = y[q];", "d[(long)np * e + q] = y[0];"),
    "ut_wrong_stride": ("ut += D[k * n + m] * ue[i + n * (j + n * m)];",
                        "ut += D[k * n + m] * ue[i + n * (m + n * j)];"),
    # the geometry differentiated from absolute coordinates: only ~1e-13 off,
    # caught by the extended-precision pin at h = 1/32 alone
    "geometry_from_absolute_coordinates": (
        "acc += (verts[3 * v + d] - verts[3 * v0 + d]) * hr[a] * hs[b] * ht[c];",
        "acc += verts[3 * v + d] * hr[a] * hs[b] * ht[c];",
        "extended_precision"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    before, after = MUTATIONS[name][:2]
    select = ["-k", MUTATIONS[name][2]] if len(MUTATIONS[name]) > 2 else []
    src = open(SRC).read()
    assert src.count(before) == 1, f"mutation anchor for {name} not found exactly once"
    mutated = tmp_path / "sem_oracle_mut.c"
    mutated.write_text(src.replace(before, after))
    lib = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99",
                    str(mutated), "-o", str(lib), "-lm"], check=True)
    env = dict(os.environ, SEM_ORACLE_LIB=str(lib))
    proc = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           os.path.join(ROOT, "tests", "test_oracle_pins.py")] + select,
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    # a pin must fail (not merely no test run: pytest exits non-zero then too)
    assert proc.returncode == 1 and " failed" in proc.stdout, \
        f"pins did not catch mutation {name}:\n{proc.stdout[-2000:]}"
