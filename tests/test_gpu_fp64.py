"""GPU parity of the FP64 path (basis tables, dof map, sum factorization,
classical) against the oracle, element by element, through the C ABI."""
import numpy as np
import pytest
import torch

from gpu_util import FP64_TOL, rel_frob, run_gpu, sample_elements
from paper_2207_00280_gb300 import workloads as wl
from paper_2207_00280_gb300.plan import IgaPlan, Patch

pytestmark = pytest.mark.gpu


def _oracle(oracle_mod, knots, p, q):
    return oracle_mod.Patch(list(knots), p, q)


# --------------------------------------------------------------------------
# a3: basis/derivative tables (Cox--de Boor) and a2: Gauss rules
# --------------------------------------------------------------------------

@pytest.mark.parametrize("p,q", [(1, 2), (2, 3), (3, 4), (3, 5), (4, 5), (5, 6)])
def test_basis_tables(oracle_mod, p, q):
    rng = np.random.default_rng(p)
    inner = np.sort(np.concatenate([rng.uniform(0.05, 0.95, 5), [0.5] * min(p, 2)]))
    knots = [wl.open_uniform_knots(6, p), np.concatenate([[0.0] * (p + 1), inner, [1.0] * (p + 1)]),
             wl.open_uniform_knots(1, p)]
    plan = IgaPlan(Patch(knots, p, q), method="sumfact")
    tab = plan.basis_tables().cpu().numpy()
    n = p + 1
    rec = 2 * q * n + q
    off = 0
    for t in knots:
        for s in oracle_mod.spans(t, p):
            xi, w, val, der = oracle_mod.basis_1d(t, p, int(s), q)
            r = tab[off:off + rec]
            off += rec
            # the two sides place the Gauss nodes by different methods (Newton on
            # P_q vs Golub--Welsch), which agree to a few ulps of xi; that offset
            # moves B by up to |B'| ulps and B' by up to |B''| ulps.
            dscale = np.abs(der).max()
            h = t[int(s) + 1] - t[int(s)]
            np.testing.assert_allclose(r[:q * n].reshape(q, n), val, rtol=0, atol=2e-15 + 1e-15 * dscale)
            np.testing.assert_allclose(r[q * n:2 * q * n].reshape(q, n), der, rtol=0,
                                       atol=1e-14 * dscale * (1 + p / max(h, 1e-3) * 1e-1))
            np.testing.assert_allclose(r[2 * q * n:], w, rtol=1e-14, atol=0)
    assert off == len(tab)


# --------------------------------------------------------------------------
# small meshes, all elements
# --------------------------------------------------------------------------

def _check(oracle_mod, knots, p, q, kappa, rho, G, method, elems=None):
    P = _oracle(oracle_mod, knots, p, q)
    out = run_gpu(knots, p, q, kappa=kappa, rho=rho, G=G, method=method)
    el = np.arange(P.E) if elems is None else elems
    Kr, Mr = (P.sumfact if P.N >= 27 else P.classical)(el, kappa=kappa, rho=rho, G=G)
    Kg = out["K"].cpu().numpy()[el]
    Mg = out["M"].cpu().numpy()[el]
    assert not np.isnan(out["K"].cpu().numpy()).any() and not np.isnan(out["M"].cpu().numpy()).any()
    assert rel_frob(Kg, Kr) <= FP64_TOL, rel_frob(Kg, Kr)
    assert rel_frob(Mg, Mr) <= FP64_TOL, rel_frob(Mg, Mr)
    np.testing.assert_array_equal(out["dof"].cpu().numpy()[el], P.dofmap(el))
    return out


@pytest.mark.parametrize("method", ["sumfact", "classical"])
def test_2d_p2_16x16_unit_kappa(oracle_mod, method):
    """2D, p=2, 16x16 elements, 3x3 Gauss points, kappa = 1, identity geometry."""
    knots = [wl.open_uniform_knots(16, 2)] * 2
    _check(oracle_mod, knots, 2, 3, None, None, None, method)


@pytest.mark.parametrize("method", ["sumfact", "classical"])
@pytest.mark.parametrize("p,dq", [(1, 1), (2, 1), (3, 1), (4, 1), (5, 1), (2, 2), (4, 2)])
def test_3d_identity_geometry(oracle_mod, method, p, dq):
    q = p + dq
    knots = [wl.open_uniform_knots(K, p) for K in (3, 2, 4)]  # ragged element counts
    P = _oracle(oracle_mod, knots, p, q)
    kappa = wl.lognormal(P.E * P.Q, 100 + p)
    rho = wl.lognormal(P.E * P.Q, 200 + p)
    elems = None if p <= 3 else sample_elements(P.E, 0.3, seed=p, K=[3, 2, 4])
    _check(oracle_mod, knots, p, q, kappa, rho, None, method, elems)


@pytest.mark.parametrize("method", ["sumfact", "classical"])
@pytest.mark.parametrize("p,dq", [(1, 1), (2, 1), (3, 1), (3, 2), (4, 1), (5, 1)])
def test_3d_curved_geometry(oracle_mod, method, p, dq):
    q = p + dq
    knots = [wl.open_uniform_knots(K, p) for K in (2, 3, 2)]
    P = _oracle(oracle_mod, knots, p, q)
    kappa = wl.lognormal(P.E * P.Q, 300 + p)
    G = wl.curved_map_jacobian(knots, q)
    elems = None if p <= 3 else sample_elements(P.E, 0.3, seed=p, K=[2, 3, 2])
    _check(oracle_mod, knots, p, q, kappa, None, G, method, elems)


@pytest.mark.parametrize("method", ["sumfact", "classical"])
@pytest.mark.parametrize("p,dq", [(1, 1), (2, 2), (3, 1), (5, 1), (8, 1), (8, 2)])
def test_2d_general(oracle_mod, method, p, dq):
    q = p + dq
    knots = [wl.open_uniform_knots(5, p), wl.open_uniform_knots(3, p)]
    P = _oracle(oracle_mod, knots, p, q)
    kappa = wl.lognormal(P.E * P.Q, 400 + p)
    rho = wl.lognormal(P.E * P.Q, 500 + p)
    rng = np.random.default_rng(p)
    G = np.eye(2) + 0.2 * rng.standard_normal((P.E, P.Q, 2, 2))
    _check(oracle_mod, knots, p, q, kappa, rho, G, method)


def test_general_path_on_identity_matches_identity_path():
    """jac = explicit identity (general kernel) equals jac = NULL (diagonal kernel)."""
    p, q = 3, 4
    knots = [wl.open_uniform_knots(4, p)] * 3
    E, Q = 64, 64
    kappa = wl.lognormal(E * Q, 7)
    G = np.broadcast_to(np.eye(3), (E, Q, 3, 3)).copy()
    a = run_gpu(knots, p, q, kappa=kappa, G=G)
    b = run_gpu(knots, p, q, kappa=kappa)
    assert rel_frob(a["K"].cpu().numpy(), b["K"].cpu().numpy()) <= 1e-14
    assert rel_frob(a["M"].cpu().numpy(), b["M"].cpu().numpy()) <= 1e-14


def test_repeated_interior_knots_and_single_element(oracle_mod):
    p, q = 3, 4
    knots = [np.array([0.0] * 4 + [0.3, 0.3, 0.6, 0.6, 0.6] + [1.0] * 4),   # multiplicities 2, 3
             wl.open_uniform_knots(1, p),                                    # one element
             np.array([0.0] * 4 + [0.2, 0.45, 0.5] + [1.0] * 4)]            # non-uniform
    P = _oracle(oracle_mod, knots, p, q)
    kappa = wl.lognormal(P.E * P.Q, 9)
    G = wl.curved_map_jacobian(knots, q)
    for method in ("sumfact", "classical"):
        _check(oracle_mod, knots, p, q, kappa, None, G, method)


def test_mass_only_and_stiffness_only(oracle_mod):
    p, q = 2, 3
    knots = [wl.open_uniform_knots(3, p)] * 3
    P = _oracle(oracle_mod, knots, p, q)
    kappa = wl.lognormal(P.E * P.Q, 11)
    Kr, Mr = P.classical(kappa=kappa)
    a = run_gpu(knots, p, q, kappa=kappa, mass=False, dof=False)
    assert a["M"] is None and rel_frob(a["K"].cpu().numpy(), Kr) <= FP64_TOL
    b = run_gpu(knots, p, q, kappa=kappa, stiffness=False, dof=False)
    assert b["K"] is None and rel_frob(b["M"].cpu().numpy(), Mr) <= FP64_TOL


def test_integrate_argument_errors():
    from paper_2207_00280_gb300 import capi
    plan = IgaPlan(Patch([wl.open_uniform_knots(2, 2)] * 3, 2, 3), mass=False)
    with pytest.raises(capi.IgaError) as ei:
        plan.integrate()          # nothing requested
    assert ei.value.code == capi.IGA_ERR_ARG
    M = torch.empty(plan.info.n_mat_entries, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.IgaError):
        plan.integrate(M=M)       # mass not in the plan
    plan.close()


# --------------------------------------------------------------------------
# full size: 3D p=3, 32^3 elements, 4^3 Gauss points, lognormal kappa
# (the benchmark's workload and launch), sampled against the oracle
# --------------------------------------------------------------------------

@pytest.mark.parametrize("method", ["sumfact", "classical"])
def test_3d_p3_32_full_size(oracle_mod, method):
    W = wl.WORKLOADS["3d_p3_32"]
    sp = W.spec
    knots = sp.knots
    kappa = W.kappa()
    out = run_gpu(knots, sp.p, sp.q, kappa=kappa, method=method)
    K, M = out["K"], out["M"]
    # properties over every element, on the device
    one = torch.ones(sp.N, dtype=torch.float64, device="cuda")
    k1 = (K @ one).abs().amax(dim=1)
    kn = K.flatten(1).norm(dim=1)
    assert float((k1 / kn).max()) <= 1e-13
    assert float((K - K.transpose(1, 2)).abs().max()) == 0.0
    vol = M.sum(dim=(1, 2))
    assert float((vol - (1.0 / 32) ** 3).abs().max()) <= 1e-13 * (1.0 / 32) ** 3 * 64
    # sampled elements against the oracle
    P = _oracle(oracle_mod, knots, sp.p, sp.q)
    el = sample_elements(sp.E, 0.01, seed=2207, K=32)
    Kr, Mr = P.sumfact(el, kappa=kappa)
    assert rel_frob(K[torch.as_tensor(el, device="cuda")].cpu().numpy(), Kr) <= FP64_TOL
    assert rel_frob(M[torch.as_tensor(el, device="cuda")].cpu().numpy(), Mr) <= FP64_TOL
    # the dof map of every element, bit-exact
    np.testing.assert_array_equal(out["dof"].cpu().numpy(), P.dofmap())
