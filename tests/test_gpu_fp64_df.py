"""GPU parity of the float-float FP64-accurate sum factorization
(precision IGA_FP64_DF) against the FP64 oracle: the same <= 1e-12 per-element
relative Frobenius bar as the FP64 path."""
import numpy as np
import pytest
import torch

from gpu_util import FP64_TOL, rel_frob, run_gpu, sample_elements
from paper_2207_00280_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("p,dq", [(1, 1), (2, 1), (3, 1), (3, 2), (4, 1), (4, 2), (5, 1)])
@pytest.mark.parametrize("curved", [False, True])
def test_small_meshes(oracle_mod, p, dq, curved):
    q = p + dq
    knots = [wl.open_uniform_knots(K, p) for K in (2, 3, 2)]
    P = oracle_mod.Patch(knots, p, q)
    kappa = wl.lognormal(P.E * P.Q, 1000 + p)
    rho = wl.lognormal(P.E * P.Q, 1100 + p)
    G = wl.curved_map_jacobian(knots, q) if curved else None
    out = run_gpu(knots, p, q, kappa=kappa, rho=rho, G=G, precision="fp64_df")
    el = np.arange(P.E) if p <= 3 else sample_elements(P.E, 0.5, seed=p, K=[2, 3, 2])
    Kr, Mr = P.sumfact(el, kappa=kappa, rho=rho, G=G)
    eK = rel_frob(out["K"].cpu().numpy()[el], Kr)
    eM = rel_frob(out["M"].cpu().numpy()[el], Mr)
    print(f"fp64_df p={p} q={q} curved={curved}: {eK:.2e} {eM:.2e}")
    assert eK <= FP64_TOL and eM <= FP64_TOL
    np.testing.assert_array_equal(out["dof"].cpu().numpy()[el], P.dofmap(el))


def test_single_matrices_and_repeated_knots(oracle_mod):
    p, q = 3, 4
    knots = [np.array([0.0] * 4 + [0.3, 0.3, 0.6] + [1.0] * 4), wl.open_uniform_knots(1, p),
             wl.open_uniform_knots(3, p)]
    P = oracle_mod.Patch(knots, p, q)
    kappa = wl.lognormal(P.E * P.Q, 1200)
    G = wl.curved_map_jacobian(knots, q)
    Kr, Mr = P.classical(kappa=kappa, G=G)
    a = run_gpu(knots, p, q, kappa=kappa, G=G, precision="fp64_df", mass=False, dof=False)
    b = run_gpu(knots, p, q, kappa=kappa, G=G, precision="fp64_df", stiffness=False, dof=False)
    assert rel_frob(a["K"].cpu().numpy(), Kr) <= FP64_TOL
    assert rel_frob(b["M"].cpu().numpy(), Mr) <= FP64_TOL


def test_3d_p3_32_full_size(oracle_mod):
    W = wl.WORKLOADS["3d_p3_32"]
    sp = W.spec
    kappa = W.kappa()
    out = run_gpu(sp.knots, sp.p, sp.q, kappa=kappa, precision="fp64_df")
    K, M = out["K"], out["M"]
    one = torch.ones(sp.N, dtype=torch.float64, device="cuda")
    assert float(((K @ one).abs().amax(dim=1) / K.flatten(1).norm(dim=1)).max()) <= 1e-13
    el = sample_elements(sp.E, 0.01, seed=2207, K=32)
    P = oracle_mod.Patch(sp.knots, sp.p, sp.q)
    Kr, Mr = P.sumfact(el, kappa=kappa)
    idx = torch.as_tensor(el, device="cuda")
    eK, eM = rel_frob(K[idx].cpu().numpy(), Kr), rel_frob(M[idx].cpu().numpy(), Mr)
    print(f"fp64_df 32^3 p=3: {eK:.2e} {eM:.2e}")
    assert eK <= FP64_TOL and eM <= FP64_TOL
