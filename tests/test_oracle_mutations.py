"""Planted mistakes in a copy of the oracle must fail the oracle pins.

Each case edits one line of a copy of ``oracle/jk_oracle.c`` (a dropped
term, a wrong sign, a wrong index or factor), compiles it with gcc into a
temporary directory, and runs ``tests/test_oracle_pins.py`` against it via
``JK_ORACLE_LIB``. Everything runs on the CPU.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "jk_oracle.c")

MUTATIONS = {
    "hermite_E_drops_t+1_term": ("v = h * em1 + XPA * e0 + (t + 1) * ep1;", "v = h * em1 + XPA * e0;"),
    "hermite_E_wrong_centre": ("v = h * em1 + XPA * e0 + (t + 1) * ep1;",
                               "v = h * em1 + XPB * e0 + (t + 1) * ep1;"),
    "ket_sign_dropped": ("double sg = ((t2 + u2 + v2) & 1) ? -1.0 : 1.0;", "double sg = 1.0;"),
    "hermite_R_wrong_factor": ("if (t > 1) val += (t - 1) * RR(n + 1, t - 2, u, v);",
                               "if (t > 1) val += (t) * RR(n + 1, t - 2, u, v);"),
    "hermite_R_wrong_axis": ("val = Y * RR(n + 1, t, u - 1, v);", "val = X * RR(n + 1, t, u - 1, v);"),
    "boys_series_index": ("term *= 2.0 * T / (2 * mmax + 2 * k + 1);",
                          "term *= 2.0 * T / (2 * mmax + 2 * k - 1);"),
    "boys_upward_sign": ("F[m + 1] = ((2 * m + 1) * F[m] - e) / (2.0 * T);",
                         "F[m + 1] = ((2 * m + 1) * F[m] + e) / (2.0 * T);"),
    "prefactor": ("double pref = scale * sqrt(theta) * 2.0 * pow(M_PI, 2.5) / (p * q * sqrt(p + q));",
                  "double pref = scale * sqrt(theta) * 2.0 * pow(M_PI, 2.5) / (p * q * sqrt(p * q));"),
    "range_separation_theta": ("double theta = omega > 0.0 ? omega * omega / (omega * omega + rho) : 1.0;",
                               "double theta = omega > 0.0 ? omega * omega / (omega * omega + p) : 1.0;"),
    "range_separation_prefactor": ("double pref = scale * sqrt(theta) * 2.0",
                                   "double pref = scale * theta * 2.0"),
    "degeneracy_factor_dropped": ("if (p1 == p2) f *= 0.5;", ""),
    "K_update_wrong_density": ("Yk[I * nao + L] += v * Dk[Jx * nao + Kx];",
                               "Yk[I * nao + L] += v * Dk[Jx * nao + L];"),
    "J_ket_update_factor": ("Xk[Kx * nao + L] += 2.0 * v * Dk[I * nao + Jx];",
                            "Xk[Kx * nao + L] += v * Dk[I * nao + Jx];"),
    "dmax_row_offset_dropped": ("double v = fabs(D[((size_t)k * nao + off[a] + i) * nao + off[b] + j]);",
                                "double v = fabs(D[((size_t)k * nao + off[a]) * nao + off[b] + j]);"),
    "dmax_first_density_only": ("            for (int k = 0; k < ndm; ++k)\n                for (int i = 0; i < ncart(sh[a].l); ++i)",
                                "            for (int k = 0; k < 1; ++k)\n                for (int i = 0; i < ncart(sh[a].l); ++i)"),
    "bound_drops_K_block_bd": ("            dm = fmax(dm, Dm[b * nsh + d]);\n", ""),
    "schwarz_wrong_diagonal": ("double v = fabs(blk[((i * nb + j) * na + i) * nb + j]);",
                               "double v = fabs(blk[((i * nb + i) * na + j) * nb + j]);"),
}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_fails_pins(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert old in src, f"mutation anchor for {name} not found"
    mutated = tmp_path / "jk_oracle.c"
    mutated.write_text(src.replace(old, new, 1))
    lib = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-D_DEFAULT_SOURCE",
                    str(mutated), "-o", str(lib), "-lm"], check=True)
    env = dict(os.environ, JK_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        "-q", "-x", "-p", "no:cacheprovider"], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutation {name} was not caught:\n{r.stdout[-800:]}"
