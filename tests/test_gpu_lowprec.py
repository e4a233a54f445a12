"""GPU parity of the FP32 and BF16 sum-factorization forms against the FP64
oracle: per-element relative Frobenius error <= 1e-5 (FP32) and <= 5e-3
(BF16 contractions on the tensor cores, FP32 accumulation)."""
import numpy as np
import pytest
import torch

from gpu_util import BF16_TOL, FP32_TOL, FP64_TOL, rel_frob, run_gpu, sample_elements
from paper_2207_00280_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"fp32": FP32_TOL, "bf16": BF16_TOL, "fp64": FP64_TOL, "fp64_df": FP64_TOL}


def _cmp(oracle_mod, knots, p, q, kappa, rho, G, prec, mass=True, stiffness=True, elems=None):
    P = oracle_mod.Patch(list(knots), p, q)
    out = run_gpu(knots, p, q, kappa=kappa, rho=rho, G=G, precision=prec, mass=mass,
                  stiffness=stiffness)
    el = np.arange(P.E) if elems is None else elems
    Kr, Mr = P.sumfact(el, kappa=kappa, rho=rho, G=G, stiffness=stiffness, mass=mass)
    errs = {}
    if stiffness:
        Kg = out["K"].cpu().numpy()[el]
        assert np.isfinite(out["K"].cpu().numpy()).all()
        errs["K"] = rel_frob(Kg, Kr)
        assert errs["K"] <= TOL[prec], errs
    if mass:
        Mg = out["M"].cpu().numpy()[el]
        assert np.isfinite(out["M"].cpu().numpy()).all()
        errs["M"] = rel_frob(Mg, Mr)
        assert errs["M"] <= TOL[prec], errs
    np.testing.assert_array_equal(out["dof"].cpu().numpy()[el], P.dofmap(el))
    print(f"{prec} p={p} q={q} curved={G is not None} errors {errs}")
    return out, errs


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("p,dq", [(1, 1), (2, 1), (3, 1), (3, 2), (4, 1), (4, 2), (5, 1)])
@pytest.mark.parametrize("curved", [False, True])
def test_small_meshes(oracle_mod, prec, p, dq, curved):
    q = p + dq
    knots = [wl.open_uniform_knots(K, p) for K in (2, 3, 2)]
    P = oracle_mod.Patch(knots, p, q)
    kappa = wl.lognormal(P.E * P.Q, 600 + p)
    rho = wl.lognormal(P.E * P.Q, 700 + p)
    G = wl.curved_map_jacobian(knots, q) if curved else None
    _cmp(oracle_mod, knots, p, q, kappa, rho, G, prec)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("which", ["stiffness", "mass"])
def test_single_matrix_modes(oracle_mod, prec, which):
    p, q = 3, 4
    knots = [wl.open_uniform_knots(3, p)] * 3
    P = oracle_mod.Patch(knots, p, q)
    kappa = wl.lognormal(P.E * P.Q, 800)
    G = wl.curved_map_jacobian(knots, q)
    _cmp(oracle_mod, knots, p, q, kappa, None, G, prec, mass=which == "mass",
         stiffness=which == "stiffness")


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("which", ["stiffness", "mass"])
@pytest.mark.parametrize("p,q", [(4, 5), (4, 6), (5, 6)])
def test_streamed_single_matrix_modes(oracle_mod, prec, which, p, q):
    """The streamed form (identity map, p = 4 and 5) with one matrix only: its
    row-vector stage 2 writes the C11/CM rows and the C00 rows from different
    threads, and each single-matrix mode drops one of them."""
    knots = [wl.open_uniform_knots(K, p) for K in (3, 2, 3)]
    P = oracle_mod.Patch(knots, p, q)
    kappa = wl.lognormal(P.E * P.Q, 820 + p)
    rho = wl.lognormal(P.E * P.Q, 830 + p)
    _cmp(oracle_mod, knots, p, q, kappa, rho, None, prec, mass=which == "mass",
         stiffness=which == "stiffness")


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_curved_p4_stiffness_only_every_element(oracle_mod, prec):
    """The stiffness alone with a general map at p = 4, q = 5 has a kernel of
    its own (symmetric operand rows, staged mirror, bulk-copy output, the next
    element's inputs prefetched): every element of a 7 x 7 x 8 mesh against
    the oracle -- more elements than resident CTAs, so CTAs take several
    elements and element matrices start at every 4-byte offset mod 16."""
    p, q = 4, 5
    knots = [wl.open_uniform_knots(K, p) for K in (7, 7, 8)]
    P = oracle_mod.Patch(knots, p, q)
    kappa = wl.lognormal(P.E * P.Q, 812)
    G = wl.curved_map_jacobian(knots, q)
    _cmp(oracle_mod, knots, p, q, kappa, None, G, prec, mass=False)


_ORACLE_48 = {}


def _oracle_48(oracle_mod, W, el, kappa, G):
    """The oracle's stiffness of the sampled 48^3 elements, computed once for
    every precision."""
    if "K" not in _ORACLE_48:
        sp = W.spec
        P = oracle_mod.Patch(sp.knots, sp.p, sp.q)
        _ORACLE_48["K"] = P.sumfact(el, kappa=kappa, G=G, mass=False)[0]
        _ORACLE_48["dof"] = P.dofmap()
    return _ORACLE_48["K"], _ORACLE_48["dof"]


@pytest.mark.parametrize("prec", ["fp64", "fp64_df", "fp32", "bf16"])
def test_3d_p4_48_curved_full_size(oracle_mod, prec):
    """3D, p=4, 48^3 elements, 5^3 Gauss points, cyclic sine map, lognormal kappa,
    in the benchmark's launch: the stiffness of every element is computed; a
    seeded 1% sample plus the corners is compared with the oracle, K 1 = 0 is
    checked on every element, and the dof map of every element is compared
    with the oracle's bit for bit."""
    W = wl.WORKLOADS["3d_p4_48_curved"]
    sp = W.spec
    kappa = W.kappa()
    G = W.jacobian()
    out = run_gpu(sp.knots, sp.p, sp.q, kappa=kappa, G=G, precision=prec, mass=False)
    K = out["K"]
    one = torch.ones(sp.N, dtype=K.dtype, device="cuda")
    r = (K @ one).abs().amax(dim=1) / K.flatten(1).norm(dim=1)
    assert float(r.max()) <= (1e-13 if prec in ("fp64", "fp64_df") else TOL[prec])
    el = sample_elements(sp.E, 0.01, seed=2208, K=48)
    Kr, dof = _oracle_48(oracle_mod, W, el, kappa, G)
    err = rel_frob(K[torch.as_tensor(el, device="cuda")].cpu().numpy(), Kr)
    print(f"{prec} 48^3 p=4 curved stiffness: max rel Frobenius error {err:.3e}")
    assert err <= TOL[prec]
    np.testing.assert_array_equal(out["dof"].cpu().numpy(), dof)
