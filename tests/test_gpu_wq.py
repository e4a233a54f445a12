"""GPU parity of the weighted-quadrature mass matrix (iga_wq_points,
iga_wq_mass) with the oracle, and closed forms at the benchmark size.

The plan builds the rule with its own host code (Newton Gauss rule,
triangular Cox--de Boor, Cholesky of A A^T); the oracle with its own
(Golub--Welsch, recursive Cox--de Boor, Gaussian elimination).  Values are
compared within 1e-12 of the largest entry; points within 1e-15.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2207_00280_gb300 import capi
from paper_2207_00280_gb300 import workloads as wl
from paper_2207_00280_gb300.plan import IgaPlan, Patch

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda")


def _nonuniform_knots(p, seed, n_inner=5):
    rng = np.random.default_rng(seed)
    inner = np.sort(rng.uniform(0.08, 0.92, size=n_inner))
    if p >= 2:
        inner = np.sort(np.concatenate([inner, inner[1:2]]))
    return np.concatenate([[0.0] * (p + 1), inner, [1.0] * (p + 1)])


def _cases():
    return [
        ("p1_uniform", [wl.open_uniform_knots(5, 1)] * 3, 1),
        ("p2_mixed", [wl.open_uniform_knots(4, 2), _nonuniform_knots(2, 61), wl.open_uniform_knots(3, 2)], 2),
        ("p3_uniform", [wl.open_uniform_knots(6, 3)] * 3, 3),
        ("p4_uniform", [wl.open_uniform_knots(3, 4), wl.open_uniform_knots(9, 4), wl.open_uniform_knots(2, 4)], 4),
        # a C0 line (multiplicity p: B' jumps there and is taken from the right on both
        # sides), one element in y, a double knot in z
        ("p3_c0_one_element", [np.array([0.0] * 4 + [0.3, 0.3, 0.3, 0.6] + [1.0] * 4),
                               wl.open_uniform_knots(1, 3),
                               np.array([0.0] * 4 + [0.5, 0.5] + [1.0] * 4)], 3),
    ]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_points_match_oracle(case):
    _, knots, p = case
    plan = IgaPlan(Patch(list(knots), p, p + 1), method="sumfact", precision="fp64")
    xs = plan.wq_points(0)
    for k, t in enumerate(knots):
        ref = oracle.wq_points(t, p)
        assert len(xs[k]) == len(ref)
        np.testing.assert_allclose(xs[k], ref, rtol=0, atol=1e-15)
    assert plan.wq_grid_size(0) == int(np.prod([len(x) for x in xs]))
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp64_df"])
@pytest.mark.parametrize("coef", ["one", "lognormal"])
@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_mass_matches_oracle(case, coef, precision):
    """fp64_df plans run the contraction in float-float on the FP32 pipes."""
    _, knots, p = case
    P = oracle.Patch(list(knots), p, p + 1)
    rp, ci = P.csr_pattern()
    plan = IgaPlan(Patch(list(knots), p, p + 1), method="sumfact", precision=precision)
    n = plan.wq_grid_size(0)
    c = None if coef == "one" else wl.lognormal(n, 91)
    ref = P.wq_mass(rp, ci, c=c)
    ct = torch.as_tensor(c, device=DEV) if c is not None else None
    vals = plan.wq_mass(c=ct).cpu().numpy()
    assert np.abs(vals - ref).max() <= 1e-12 * np.abs(ref).max()
    plan.close()


def test_batch_matches_oracle():
    specs = [([wl.open_uniform_knots(3, 1)] * 3, 1),
             ([wl.open_uniform_knots(4, 3), wl.open_uniform_knots(5, 3), wl.open_uniform_knots(4, 3)], 3),
             ([_nonuniform_knots(2, 62)] * 3, 2)]
    plan = IgaPlan([Patch(list(k), p, p + 1) for k, p in specs], method="sumfact", precision="fp64")
    total = plan.wq_grid_size(-1)
    c = wl.lognormal(total, 92)
    vals = plan.wq_mass(c=torch.as_tensor(c, device=DEV)).cpu().numpy()
    off, nnz = 0, 0
    for i, (knots, p) in enumerate(specs):
        P = oracle.Patch(knots, p, p + 1)
        rp, ci = P.csr_pattern()
        g = plan.wq_grid_size(i)
        ref = P.wq_mass(rp, ci, c=c[off:off + g])
        got = vals[nnz:nnz + len(ci)]
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), i
        off += g
        nnz += len(ci)
    assert off == total and nnz == len(vals)
    plan.close()


def test_full_size_row_sums_are_basis_integrals():
    """3D p=3, 32^3 elements, c = 1: the weighted-quadrature mass is the exact
    Gram matrix, whose row sums are int phi_i = prod_k (t_{i_k+p+1} - t_{i_k})/(p+1)."""
    K_el, p = 32, 3
    t = wl.open_uniform_knots(K_el, p)
    plan = IgaPlan(Patch([t] * 3, p, p + 1), method="sumfact", precision="fp64")
    rp, _ = plan.csr_pattern()
    vals = plan.wq_mass()
    seg = torch.repeat_interleave(torch.arange(plan.n_dofs, device=DEV), rp[1:] - rp[:-1])
    rows = torch.zeros(plan.n_dofs, dtype=torch.float64, device=DEV).index_add_(0, seg, vals)
    nf = len(t) - p - 1
    b = np.array([(t[i + p + 1] - t[i]) / (p + 1) for i in range(nf)])
    ref = np.einsum("k,j,i->kji", b, b, b).reshape(-1)
    assert np.abs(rows.cpu().numpy() - ref).max() <= 1e-13 * ref.max()
    plan.close()


def test_fp32_plan_rejected():
    t = wl.open_uniform_knots(3, 2)
    plan = IgaPlan(Patch([t] * 3, 2, 3), method="sumfact", precision="fp32")
    with pytest.raises(capi.IgaError) as ei:
        plan.wq_mass()
    assert ei.value.code == capi.IGA_ERR_UNSUPPORTED
    plan.close()


# --------------------------------------------------------------------------
# Weighted-quadrature diffusion stiffness (iga_wq_stiffness)
# --------------------------------------------------------------------------

def _stiff_cases():
    return [c for c in _cases() if c[2] >= 2]


@pytest.mark.parametrize("precision", ["fp64", "fp64_df"])
@pytest.mark.parametrize("coef", ["one", "lognormal"])
@pytest.mark.parametrize("case", _stiff_cases(), ids=lambda c: c[0])
def test_stiffness_matches_oracle(case, coef, precision):
    _, knots, p = case
    P = oracle.Patch(list(knots), p, p + 1)
    rp, ci = P.csr_pattern()
    plan = IgaPlan(Patch(list(knots), p, p + 1), method="sumfact", precision=precision)
    n = plan.wq_grid_size(0)
    c = None if coef == "one" else wl.lognormal(n, 94)
    ref = P.wq_stiffness(rp, ci, c=c)
    ct = torch.as_tensor(c, device=DEV) if c is not None else None
    vals = plan.wq_stiffness(c=ct).cpu().numpy()
    assert np.abs(vals - ref).max() <= 1e-12 * np.abs(ref).max()
    plan.close()


def test_stiffness_batch_matches_oracle():
    specs = [([wl.open_uniform_knots(4, 2), wl.open_uniform_knots(3, 2), wl.open_uniform_knots(5, 2)], 2),
             ([wl.open_uniform_knots(4, 3), wl.open_uniform_knots(5, 3), wl.open_uniform_knots(4, 3)], 3),
             ([_nonuniform_knots(2, 63)] * 3, 2)]
    plan = IgaPlan([Patch(list(k), p, p + 1) for k, p in specs], method="sumfact", precision="fp64")
    total = plan.wq_grid_size(-1)
    c = wl.lognormal(total, 95)
    vals = plan.wq_stiffness(c=torch.as_tensor(c, device=DEV)).cpu().numpy()
    off, nnz = 0, 0
    for i, (knots, p) in enumerate(specs):
        P = oracle.Patch(knots, p, p + 1)
        rp, ci = P.csr_pattern()
        g = plan.wq_grid_size(i)
        ref = P.wq_stiffness(rp, ci, c=c[off:off + g])
        got = vals[nnz:nnz + len(ci)]
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), i
        off += g
        nnz += len(ci)
    assert off == total and nnz == len(vals)
    plan.close()


def _bspline_integrals(t, p):
    nf = len(t) - p - 1
    return np.array([(t[i + p + 1] - t[i]) / (p + 1) for i in range(nf)])


def test_stiffness_full_size_closed_forms():
    """3D p=3, 32^3 elements.  Lognormal c: every row sums to zero (the trial
    gradients sum to zero at every point).  c = 1 (exact): K x = boundary
    flux for x the Greville abscissae of one direction (a linear field),
    (B_{i_k}(1) - B_{i_k}(0)) prod_{l != k} int B_{i_l}, in each direction."""
    K_el, p = 32, 3
    t = wl.open_uniform_knots(K_el, p)
    plan = IgaPlan(Patch([t] * 3, p, p + 1), method="sumfact", precision="fp64")
    rp, ci = plan.csr_pattern()
    n = plan.n_dofs
    seg = torch.repeat_interleave(torch.arange(n, device=DEV), rp[1:] - rp[:-1])
    c = torch.as_tensor(wl.lognormal(plan.wq_grid_size(0), 96), device=DEV)
    vals = plan.wq_stiffness(c=c)
    rows = torch.zeros(n, dtype=torch.float64, device=DEV).index_add_(0, seg, vals)
    assert float(rows.abs().max()) <= 1e-13 * float(vals.abs().max())
    vals1 = plan.wq_stiffness()
    nf = len(t) - p - 1
    gre = np.array([np.mean(t[i + 1:i + p + 1]) for i in range(nf)])
    b = _bspline_integrals(t, p)
    jump = np.zeros(nf)
    jump[0], jump[-1] = -1.0, 1.0
    idx = np.arange(n)
    comp = (idx % nf, (idx // nf) % nf, idx // (nf * nf))
    for k in range(3):
        x = torch.as_tensor(gre[comp[k]], device=DEV)
        y = torch.zeros(n, dtype=torch.float64, device=DEV).index_add_(0, seg, vals1 * x[ci.long()])
        f = [b, b, b]
        f[k] = jump
        flux = np.einsum("k,j,i->kji", f[2], f[1], f[0]).reshape(-1)
        assert np.abs(y.cpu().numpy() - flux).max() <= 1e-12 * np.abs(flux).max(), k
    plan.close()


def test_stiffness_unsupported():
    for p in (1, 5):
        t = wl.open_uniform_knots(3, p)
        plan = IgaPlan(Patch([t] * 3, p, p + 1), method="sumfact", precision="fp64")
        with pytest.raises(capi.IgaError) as ei:
            plan.wq_stiffness()
        assert ei.value.code == capi.IGA_ERR_UNSUPPORTED
        plan.close()
    t = wl.open_uniform_knots(3, 2)
    plan = IgaPlan(Patch([t] * 3, 2, 3), method="sumfact", precision="fp32")
    with pytest.raises(capi.IgaError) as ei:
        plan.wq_stiffness()
    assert ei.value.code == capi.IGA_ERR_UNSUPPORTED
    plan.close()


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_2d_mass_and_stiffness_match_oracle(p):
    """2D patches: the planner gives the missing direction one point with a
    trivial rule, so the 3D row kernels form the 2D matrices; against the
    oracle's 2D weighted quadrature (lognormal c on the 2D point grid)."""
    knots = [wl.open_uniform_knots(5, p), _nonuniform_knots(p, 64 + p)]
    P = oracle.Patch(list(knots), p, p + 1)
    rp, ci = P.csr_pattern()
    plan = IgaPlan(Patch(list(knots), p, p + 1), method="sumfact", precision="fp64")
    xs = plan.wq_points(0)
    assert len(xs) == 2
    for k in range(2):
        np.testing.assert_allclose(xs[k], oracle.wq_points(knots[k], p), rtol=0, atol=1e-15)
    n = plan.wq_grid_size(0)
    assert n == len(xs[0]) * len(xs[1])
    c = wl.lognormal(n, 97)
    ct = torch.as_tensor(c, device=DEV)
    ref = P.wq_mass(rp, ci, c=c)
    vals = plan.wq_mass(c=ct).cpu().numpy()
    assert np.abs(vals - ref).max() <= 1e-12 * np.abs(ref).max()
    if p >= 2:
        ref = P.wq_stiffness(rp, ci, c=c)
        vals = plan.wq_stiffness(c=ct).cpu().numpy()
        assert np.abs(vals - ref).max() <= 1e-12 * np.abs(ref).max()
    plan.close()
