"""GPU parity of the runtime-sized FP64 kernels against the oracle: patches with
a different degree and Gauss order per direction, degrees 6 to 8, Gauss orders
from 1 to 16, in 2D and 3D, for sum factorization, classical integration, the
dof map, the CSR pattern and the adjoint.  The paper takes one degree for every
direction and notes that the method extends to bases of different degrees
(Sec. 2.3); eq. 10 has P_1 P_2 P_3 points; its experiments run p up to 9
(Sec. 4).  Tolerance: per-element relative Frobenius error <= 1e-12 (FP64)."""
import numpy as np
import pytest
import torch

from gpu_util import FP64_TOL, rel_frob, run_gpu
from paper_2207_00280_gb300 import capi
from paper_2207_00280_gb300 import workloads as wl
from paper_2207_00280_gb300.plan import IgaPlan, Patch

pytestmark = pytest.mark.gpu
dev = torch.device("cuda")


def _knots(Ks, ps, nonuniform=False):
    out = []
    for k, (K, p) in enumerate(zip(Ks, ps)):
        t = wl.open_uniform_knots(K, p)
        if nonuniform and K > 1:
            # shift the interior knots (keeps them ordered, distinct and open)
            inner = t[p + 1:len(t) - p - 1]
            r = np.random.default_rng(50 + k).uniform(-0.3, 0.3, size=inner.size) / K
            t[p + 1:len(t) - p - 1] = inner + r
        out.append(t)
    return out


def _field_2d(E, Q, seed):
    """A smooth-enough invertible 2x2 Jacobian per point: I + small random."""
    rng = np.random.default_rng(seed)
    return np.eye(2)[None, None] + 0.15 * rng.standard_normal((E, Q, 2, 2))


def _check(oracle_mod, knots, ps, qs, method, geometry, mass=True, stiffness=True, seed=0):
    P = oracle_mod.Patch(knots, ps, qs)
    dim = len(knots)
    kappa = wl.lognormal(P.E * P.Q, 300 + seed)
    rho = wl.lognormal(P.E * P.Q, 400 + seed)
    if geometry == "curved":
        G = wl.curved_map_jacobian(knots, qs) if dim == 3 else _field_2d(P.E, P.Q, 500 + seed)
    else:
        G = None
    out = run_gpu(knots, ps, qs, kappa=kappa, rho=rho, G=G, method=method, mass=mass,
                  stiffness=stiffness)
    Kr, Mr = P.sumfact(kappa=kappa, rho=rho, G=G, stiffness=stiffness, mass=mass)
    errs = {}
    if stiffness:
        Kg = out["K"].cpu().numpy()
        assert np.isfinite(Kg).all()
        errs["K"] = rel_frob(Kg, Kr)
        assert np.array_equal(Kg, Kg.transpose(0, 2, 1))
    if mass:
        Mg = out["M"].cpu().numpy()
        assert np.isfinite(Mg).all()
        errs["M"] = rel_frob(Mg, Mr)
        assert np.array_equal(Mg, Mg.transpose(0, 2, 1))
    print(f"{method} p={ps} q={qs} {geometry}: {errs}")
    assert max(errs.values()) <= FP64_TOL, errs
    np.testing.assert_array_equal(out["dof"].cpu().numpy(), P.dofmap())
    out["plan"].close()
    return errs


ANISO_3D = [
    # degrees, Gauss points, elements, non-uniform knots
    ((1, 3, 2), (2, 4, 3), (3, 2, 4), False),
    ((2, 1, 4), (4, 2, 6), (2, 3, 2), True),
    ((6, 2, 1), (7, 3, 2), (2, 2, 3), False),
    ((3, 3, 3), (4, 5, 4), (2, 2, 2), True),     # one degree, Gauss order per direction
]


@pytest.mark.parametrize("method", ["sumfact", "classical"])
@pytest.mark.parametrize("geometry", ["identity", "curved"])
@pytest.mark.parametrize("case", range(len(ANISO_3D)))
def test_aniso_3d(oracle_mod, method, geometry, case):
    ps, qs, Ks, nu = ANISO_3D[case]
    _check(oracle_mod, _knots(Ks, ps, nu), ps, qs, method, geometry, seed=case)


@pytest.mark.parametrize("p", [6, 7, 8])
@pytest.mark.parametrize("method", ["sumfact", "classical"])
def test_high_degree_3d(oracle_mod, p, method):
    """3D p = 6, 7, 8 with q = p+1 on a curved map: the element matrices (N up
    to 729) no longer fit in shared memory and are produced block by block."""
    Ks = (2, 1, 1) if p == 8 else (2, 2, 1)
    _check(oracle_mod, _knots(Ks, (p,) * 3), p, p + 1, method, "curved", seed=p)


@pytest.mark.parametrize("ps,qs", [((3, 3, 3), (1, 1, 1)), ((2, 2, 2), (16, 16, 16)),
                                   ((1, 2, 1), (16, 1, 9)), ((4, 4, 4), (7, 7, 7))])
@pytest.mark.parametrize("geometry", ["identity", "curved"])
def test_gauss_orders(oracle_mod, ps, qs, geometry):
    """Gauss orders away from p+1, p+2: under-integration (q = 1), q = 16 in
    every direction (the curved map's coefficients then exceed shared memory and
    are recomputed at each use), mixed orders."""
    _check(oracle_mod, _knots((2, 2, 2), ps), ps, qs, "sumfact", geometry, seed=sum(qs))
    _check(oracle_mod, _knots((2, 2, 2), ps), ps, qs, "classical", geometry, seed=sum(qs))


@pytest.mark.parametrize("ps,qs", [((3, 1), (4, 3)), ((8, 3), (16, 2)), ((1, 5), (2, 1))])
@pytest.mark.parametrize("method", ["sumfact", "classical"])
@pytest.mark.parametrize("geometry", ["identity", "curved"])
def test_aniso_2d(oracle_mod, ps, qs, method, geometry):
    _check(oracle_mod, _knots((3, 4), ps, True), ps, qs, method, geometry, seed=ps[0])


@pytest.mark.parametrize("which", ["mass", "stiffness"])
def test_single_matrix_generic(oracle_mod, which):
    ps, qs = (2, 5, 1), (3, 6, 2)
    _check(oracle_mod, _knots((2, 2, 3), ps), ps, qs, "sumfact", "curved",
           mass=which == "mass", stiffness=which == "stiffness", seed=7)


@pytest.mark.parametrize("ps,qs,Ks", [((1, 3, 2), (2, 4, 3), (3, 2, 2)), ((7, 7, 7), (8, 8, 8), (2, 1, 1)),
                                      ((3, 3, 3), (2, 2, 2), (3, 2, 2)), ((2, 4), (3, 16), (3, 2))])
@pytest.mark.parametrize("geometry", ["identity", "curved"])
def test_adjoint_generic(oracle_mod, ps, qs, Ks, geometry):
    """The runtime-sized adjoint (FP64 plans): dJ/dkappa at every point and J
    against the oracle."""
    knots = _knots(Ks, ps)
    P = oracle_mod.Patch(knots, ps, qs)
    dim = len(knots)
    kappa = wl.lognormal(P.E * P.Q, 61)
    G = None
    if geometry == "curved":
        G = wl.curved_map_jacobian(knots, qs) if dim == 3 else _field_2d(P.E, P.Q, 62)
    u = wl.normal(P.n_dofs, 63)
    v = wl.normal(P.n_dofs, 64)
    gr, Jr = P.adjoint(u, v, kappa=kappa, G=G)
    guu, _ = P.adjoint(u, u, G=G)
    gvv, _ = P.adjoint(v, v, G=G)
    plan = IgaPlan(Patch(knots, ps, qs), method="sumfact", precision="fp64")
    g = torch.full((plan.n_qp,), float("nan"), dtype=torch.float64, device=dev)
    J = torch.empty(1, dtype=torch.float64, device=dev)
    jac = torch.as_tensor(np.ascontiguousarray(G), device=dev).reshape(-1) if G is not None else None
    plan.backward(torch.as_tensor(kappa, device=dev), torch.as_tensor(u, device=dev),
                  torch.as_tensor(v, device=dev), grad=g, J=J, jac=jac)
    torch.cuda.synchronize()
    gs = g.view(P.E, P.Q).cpu().numpy()
    ratio = np.abs(gs - gr) / (FP64_TOL * np.sqrt(guu * gvv) + 1e-300)
    assert ratio.max() <= 1.0, ratio.max()
    assert float(J.item()) == pytest.approx(Jr, rel=1e-12, abs=1e-12 * np.abs(kappa * gr.reshape(-1)).sum())
    plan.close()


@pytest.mark.parametrize("ps,Ks", [((1, 3, 2), (3, 2, 4)), ((2, 4), (3, 2)), ((6, 6, 6), (3, 1, 2))])
def test_csr_pattern_generic(oracle_mod, ps, Ks):
    """The sparsity pattern of the assembled matrix with a degree per direction,
    bit-exact against the oracle's."""
    knots = _knots(Ks, ps, True)
    P = oracle_mod.Patch(knots, ps, [p + 1 for p in ps])
    rp_r, ci_r = P.csr_pattern()
    plan = IgaPlan(Patch(knots, ps, [p + 1 for p in ps]), method="sumfact", precision="fp64")
    rp, ci = plan.csr_pattern()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(rp.cpu().numpy(), rp_r)
    np.testing.assert_array_equal(ci.cpu().numpy(), ci_r)
    plan.close()


def test_aniso_unsupported_forms_are_rejected():
    """Patches with a degree or Gauss order per direction run in FP64 only; the
    low-precision plans and the entry points with specialised kernels only
    reject them with IGA_ERR_UNSUPPORTED."""
    ps, qs = (1, 3, 2), (2, 4, 3)
    knots = _knots((2, 2, 2), ps)
    for prec in ("fp32", "bf16", "fp64_df"):
        with pytest.raises(capi.IgaError) as ei:
            IgaPlan(Patch(knots, ps, qs), method="sumfact", precision=prec)
        assert ei.value.code == capi.IGA_ERR_UNSUPPORTED
    plan = IgaPlan(Patch(knots, ps, qs), method="sumfact", precision="fp64")
    K, M, _ = plan.empty_outputs(dof=False)
    x = torch.zeros(plan.n_dofs, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    vals = torch.empty(max(1, plan.n_csr_nnz), dtype=torch.float64, device=dev)
    for call in (lambda: plan.apply(x, y=y), lambda: plan.assemble(K, values=vals),
                 lambda: plan.integrate_grad(GK=K, grad_kappa=torch.empty(plan.n_qp, dtype=torch.float64, device=dev)),
                 lambda: plan.wq_mass(values=vals)):
        with pytest.raises(capi.IgaError) as ei:
            call()
        assert ei.value.code == capi.IGA_ERR_UNSUPPORTED
    plan.close()
