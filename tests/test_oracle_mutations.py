"""The oracle's pins reject plausible mistakes.  Each case plants one bug in a
copy of oracle/iga_oracle.c (on the CPU), builds it, and runs the pin tests
against it in a subprocess: they must fail."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "iga_oracle.c")

MUTANTS = {
    # transposed inverse Jacobian in the physical gradient
    "transposed_Ginv": ("s2 += Gi[j * d + i] * gr[j];", "s2 += Gi[i * d + j] * gr[j];"),
    # off-diagonal stiffness terms dropped in sum factorization
    "dropped_cross_terms": ("for (int be = 0; be < d; ++be) {", "for (int be = al; be <= al; ++be) {"),
    # sign error in the second Cox--de Boor term
    "coxdeboor_sign": ("right = (t[i + p + 1] - xi) / d2", "right = (xi - t[i + p + 1]) / d2"),
    # wrong index in the recursion
    "coxdeboor_index": ("right = (t[i + p + 1] - xi) / d2 * ora_bspline(t, i + 1, p - 1, xi);",
                        "right = (t[i + p + 1] - xi) / d2 * ora_bspline(t, i, p - 1, xi);"),
    # derivative identity with the wrong sign
    "derivative_sign": ("  return a - b;\n}", "  return a + b;\n}"),
    # Gauss weights missing the factor 2 of the Golub--Welsch formula
    "gauss_weight": ("w[i] = 2.0 * V[0 * q + i] * V[0 * q + i];", "w[i] = V[0 * q + i] * V[0 * q + i];"),
    # span half-length missing from the mapped weights
    "weight_map": ("w[j] = half * wr[j];", "w[j] = wr[j];"),
    # dof stride by elements instead of functions
    "dof_stride": ("stride *= nf[k];", "stride *= L.K[k];"),
    # adjoint product of u with itself
    "adjoint_product": ("dot += pu * pv;", "dot += pu * pu;"),
    # y-direction weight dropped in stage 2 of Algorithm 2
    "sf_stage2_weight": ("Dbuf[((i3 * n3 + j3) * q1 + k1) * q2 + k2] * B->w[1][k2];",
                         "Dbuf[((i3 * n3 + j3) * q1 + k1) * q2 + k2];"),
    # global assembly: element matrix inserted transposed
    "assemble_transposed": ("values[l] += Ae[((size_t)e * N + a) * N + b];",
                            "values[l] += Ae[((size_t)e * N + b) * N + a];", "test_oracle_assembly.py"),
    # operator application gathers the test function's dof instead of the trial's
    "apply_gather": ("if (Ke) sK += Ke[(size_t)a * N + b] * x[dof[b]];",
                     "if (Ke) sK += Ke[(size_t)a * N + b] * x[dof[a]];", "test_oracle_assembly.py"),
    # weighted quadrature: the right end of the domain evaluated as 0
    "wq_right_end": ("  if (x >= t[m - 1]) return (i == m - p - 2) ? 1.0 : 0.0;",
                     "  if (x >= t[m - 1]) return 0.0;", "test_oracle_wq.py"),
    # weighted quadrature: Gauss weights without the half-length factor
    "wq_gram_weight": (": 0.5 * (eb - ea) * gw[g] * ora_bspline(t, i, p, xi)",
                       ": gw[g] * ora_bspline(t, i, p, xi)", "test_oracle_wq.py"),
    # weighted quadrature: the derivative rule made exact against trial values
    "wq_deriv_values": ("A[a * nq + q] = der ? wq_bspline_deriv(t, m, js[a], p, x[qlo + q])",
                        "A[a * nq + q] = der ? wq_bspline(t, m, js[a], p, x[qlo + q])",
                        "test_oracle_wq.py"),
    # weighted quadrature: B' at the right end of the domain taken from the half-open recursion (0)
    "wq_deriv_right_end": ("  if (x < t[m - 1]) return ora_bspline_deriv(t, i, p, x);",
                           "  if (x <= t[m - 1]) return ora_bspline_deriv(t, i, p, x);",
                           "test_oracle_wq.py"),
    # weighted-quadrature stiffness: the y and z derivative terms exchanged
    "wq_stiff_direction": ("const int v1 = k == 0, v2 = k == 1, v3 = k == 2;",
                           "const int v1 = k == 0, v2 = k == 2, v3 = k == 1;", "test_oracle_wq.py"),
    # weighted quadrature: test and trial weights exchanged in direction 2
    "wq_transposed": ("const double f2 = W[1][(size_t)i2 * np[1] + q2] * Bv[1][(size_t)j2 * np[1] + q2];",
                      "const double f2 = W[1][(size_t)j2 * np[1] + q2] * Bv[1][(size_t)i2 * np[1] + q2];",
                      "test_oracle_wq.py"),
    # element-matrix backward: the upstream gradient read transposed for the mass
    "grad_mass_product": ("if (GM) sm += GM[((size_t)s * N + a) * N + b] * phi[a] * phi[b];",
                          "if (GM) sm += GM[((size_t)s * N + a) * N + b] * phi[a] * phi[a];",
                          "test_oracle_assembly.py"),
    # Algorithm 1: the trial function's y index taken from the test function
    "classical_trial_index": ("int b = j1 + n1 * (j2 + n2 * j3);", "int b = j1 + n1 * (i2 + n2 * j3);"),
    # quadrature-point index: the y stride taken from the wrong direction
    "qp_stride_direction": ("kk[1] = (k / L->q[0]) % L->q[1];", "kk[1] = (k / L->q[1]) % L->q[1];",
                            "test_oracle_aniso.py"),
    # local-function index: the z stride built from n_1 twice
    "local_stride_direction": ("aa[2] = (L->d == 3) ? a / (L->n[0] * L->n[1]) : 0;",
                               "aa[2] = (L->d == 3) ? a / (L->n[0] * L->n[0]) : 0;",
                               "test_oracle_aniso.py"),
    # Algorithm 2 stage 1: the z contraction weighted with the y direction's Gauss weights
    "sf_stage1_weight_direction": ("acc += FAC(2, sa[2], i3, k3) * FAC(2, sb[2], j3, k3) * B->w[2][k3] *",
                                   "acc += FAC(2, sa[2], i3, k3) * FAC(2, sb[2], j3, k3) * B->w[1][k3] *",
                                   "test_oracle_aniso.py"),
    # element-matrix backward: every component of the trial gradient replaced by its x component
    "grad_stiff_component": ("for (int i = 0; i < d; ++i) dot += grad[(size_t)a * 3 + i] * grad[(size_t)b * 3 + i];",
                             "for (int i = 0; i < d; ++i) dot += grad[(size_t)a * 3 + i] * grad[(size_t)b * 3 + 0];",
                             "test_oracle_assembly.py"),
    # sparsity pattern misses the first function of every element
    "pattern_drop": ("for (int b = 0; b < N; ++b)\n        if (mark[dof[b]] != i)",
                     "for (int b = 1; b < N; ++b)\n        if (mark[dof[b]] != i)", "test_oracle_assembly.py"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(tmp_path, name):
    old, new = MUTANTS[name][:2]
    pins = MUTANTS[name][2] if len(MUTANTS[name]) > 2 else "test_oracle_pins.py"
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site not found: {old}"
    mutated = src.replace(old, new, 1)
    cfile = tmp_path / "iga_oracle.c"
    cfile.write_text(mutated)
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared",
                    "-I", os.path.join(ROOT, "oracle"), "-o", str(so), str(cfile), "-lm"], check=True)
    env = dict(os.environ, IGA_ORACLE_SO=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pins)],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"
    assert " failed" in r.stdout, f"mutant {name} did not fail a pin cleanly:\n{r.stdout[-2000:]}"
