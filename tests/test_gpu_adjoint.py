"""GPU parity of the matrix-free adjoint (iga_integrate_backward) and its
torch.autograd.Function: g = dJ/dkappa and J = u^T K(kappa) v against the
oracle, the element-matrix path, Greville identities and central differences."""
import numpy as np
import pytest
import torch

from gpu_util import sample_elements, run_gpu
from paper_2207_00280_gb300 import workloads as wl
from paper_2207_00280_gb300.autograd import iga_bilinear
from paper_2207_00280_gb300.plan import IgaPlan, Patch

pytestmark = pytest.mark.gpu
dev = torch.device("cuda")


def _t(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), device=dev, dtype=dtype)


def _adj(plan, kappa, u, v, G=None, dtype=torch.float64):
    g = torch.empty(plan.n_qp, dtype=dtype, device=dev)
    J = torch.empty(1, dtype=torch.float64, device=dev)
    plan.backward(_t(kappa), _t(u, dtype), _t(v, dtype), grad=g, J=J,
                  jac=_t(G).reshape(-1) if G is not None else None)
    torch.cuda.synchronize()
    return g.cpu().numpy().astype(np.float64), float(J.item())


@pytest.mark.parametrize("p,dq,curved", [(1, 1, False), (2, 1, True), (3, 1, False), (3, 2, True),
                                         (4, 1, True), (5, 1, False)])
def test_adjoint_vs_oracle(oracle_mod, p, dq, curved):
    q = p + dq
    knots = [wl.open_uniform_knots(K, p) for K in (2, 3, 2)]
    P = oracle_mod.Patch(knots, p, q)
    kappa = wl.lognormal(P.E * P.Q, 900 + p)
    u = wl.normal(P.n_dofs, 901)
    v = wl.normal(P.n_dofs, 902)
    G = wl.curved_map_jacobian(knots, q) if curved else None
    gr, Jr = P.adjoint(u, v, kappa=kappa, G=G)
    plan = IgaPlan(Patch(knots, p, q), method="sumfact", precision="fp64")
    g, J = _adj(plan, kappa, u, v, G)
    assert np.abs(g - gr.reshape(-1)).max() <= 1e-12 * np.abs(gr).max()
    assert J == pytest.approx(Jr, rel=1e-12, abs=1e-13 * np.abs(kappa * gr.reshape(-1)).sum())
    # FP64_DF plans: float-float on the FP32 pipes, the FP64 bound
    pdf = IgaPlan(Patch(knots, p, q), method="sumfact", precision="fp64_df")
    gd, Jd = _adj(pdf, kappa, u, v, G)
    assert np.abs(gd - gr.reshape(-1)).max() <= 1e-12 * np.abs(gr).max()
    assert Jd == pytest.approx(Jr, rel=1e-12, abs=1e-13 * np.abs(kappa * gr.reshape(-1)).sum())
    plan32 = IgaPlan(Patch(knots, p, q), method="sumfact", precision="fp32")
    g32, J32 = _adj(plan32, kappa, u, v, G, dtype=torch.float32)
    assert np.linalg.norm(g32 - gr.reshape(-1)) <= 1e-5 * np.linalg.norm(gr)
    assert abs(J32 - Jr) <= 1e-5 * np.abs(kappa * gr.reshape(-1)).sum()


@pytest.mark.parametrize("curved", [False, True], ids=["identity", "general"])
@pytest.mark.parametrize("p,dq", [(1, 1), (2, 1), (2, 2), (3, 1), (4, 2), (5, 1)])
def test_adjoint_2d_vs_oracle(oracle_mod, p, dq, curved):
    """2D adjoint (FP64 plans): g and J against the oracle; J also equals
    u^T K v from the oracle's element matrices (a second oracle path)."""
    q = p + dq
    knots = [wl.open_uniform_knots(5, p), wl.open_uniform_knots(3, p)]
    P = oracle_mod.Patch(knots, p, q)
    kappa = wl.lognormal(P.E * P.Q, 930 + p)
    u = wl.normal(P.n_dofs, 931)
    v = wl.normal(P.n_dofs, 932)
    G = None
    if curved:
        G = np.eye(2)[None] + 0.15 * wl.normal(4 * P.E * P.Q, 933).reshape(P.E * P.Q, 2, 2)
    gr, Jr = P.adjoint(u, v, kappa=kappa, G=G)
    Ke, _ = P.classical(kappa=kappa, G=G, mass=False)
    dof = P.dofmap()
    Jm = float(np.einsum("ea,eab,eb->", u[dof], Ke, v[dof]))
    plan = IgaPlan(Patch(knots, p, q), method="sumfact", precision="fp64")
    g, J = _adj(plan, kappa, u, v, G)
    assert np.abs(g - gr.reshape(-1)).max() <= 1e-12 * np.abs(gr).max()
    scale = np.abs(kappa * gr.reshape(-1)).sum()
    assert abs(J - Jr) <= 1e-13 * scale and abs(J - Jm) <= 1e-12 * scale
    plan.close()


def test_adjoint_greville_identities():
    p, q, K = 3, 4, 4
    t = wl.open_uniform_knots(K, p)
    gr = np.array([t[i + 1:i + p + 1].mean() for i in range(len(t) - p - 1)])
    nf = len(gr)
    idx = np.arange(nf ** 3)
    ux, uy = gr[idx % nf], gr[(idx // nf) % nf]
    plan = IgaPlan(Patch([t] * 3, p, q), method="sumfact")
    ones = np.ones(plan.n_qp)
    g, J = _adj(plan, ones, ux, ux)
    assert J == pytest.approx(1.0, rel=1e-13) and g.sum() == pytest.approx(1.0, rel=1e-13)
    g, J = _adj(plan, ones, ux, uy)
    assert abs(J) <= 1e-14 and np.abs(g).max() <= 1e-14


def test_matrix_free_J_equals_element_matrix_J():
    """J from the adjoint kernel equals sum_e u_e^T K_e v_e from the FP64 stiffness kernel."""
    p, q = 3, 4
    knots = [wl.open_uniform_knots(K, p) for K in (5, 4, 3)]
    E, Q = 60, 64
    kappa = wl.lognormal(E * Q, 910)
    G = wl.curved_map_jacobian(knots, q)
    plan = IgaPlan(Patch(knots, p, q), method="sumfact")
    u = wl.normal(plan.n_dofs, 911)
    v = wl.normal(plan.n_dofs, 912)
    _, J = _adj(plan, kappa, u, v, G)
    out = run_gpu(knots, p, q, kappa=kappa, G=G, mass=False)
    K, D = out["K"], out["dof"].long()
    ue, ve = _t(u)[D], _t(v)[D]
    Jm = float(torch.einsum("ea,eab,eb->", ue, K, ve).item())
    assert J == pytest.approx(Jm, rel=1e-12)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_3d_p3_40_autograd_and_fd(oracle_mod, prec):
    """3D, p=3, 40^3 elements, 4^3 Gauss points, lognormal kappa, u, v ~ N(0,1):
    J and dJ/dkappa at all 4.1M quadrature points through torch.autograd; FD
    (h = 1e-6 kappa_q) on 1000 seeded points in FP64; FP32 against FP64."""
    W = wl.WORKLOADS["3d_p3_40_adjoint"]
    sp = W.spec
    plan = IgaPlan(Patch(sp.knots, sp.p, sp.q), method="sumfact", precision=prec)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    kappa = _t(W.kappa()).requires_grad_(True)
    u = _t(wl.normal(sp.n_dofs, wl.SEED_ADJ_U), dtype)
    v = _t(wl.normal(sp.n_dofs, wl.SEED_ADJ_V), dtype)
    J = iga_bilinear(kappa, u, v, plan)
    J.backward()
    g = kappa.grad.detach()
    assert torch.isfinite(g).all()
    # J = kappa . g exactly (linearity), any precision
    assert float((kappa.detach() * g).sum()) == pytest.approx(float(J), rel=1e-5 if prec == "fp32" else 1e-12)
    # a seeded 1% sample of the elements plus the corners against the oracle's
    # analytic gradient, point by point: |g - g_oracle| <= tol sqrt(g_uu g_vv)
    # with g_uu = w |det G| |G^{-T} grad u|^2 (Cauchy--Schwarz bounds |g| by it,
    # so the bound is relative to the magnitudes that meet at the point and
    # stays meaningful where the dot product cancels)
    P = oracle_mod.Patch(sp.knots, sp.p, sp.q)
    el = sample_elements(sp.E, 0.01, seed=wl.SEED_ADJ_KAPPA, K=40)
    uh, vh = u.double().cpu().numpy(), v.double().cpu().numpy()
    gr, _ = P.adjoint(uh, vh, kappa=kappa.detach().cpu().numpy(), elems=el)
    guu, _ = P.adjoint(uh, uh, elems=el)
    gvv, _ = P.adjoint(vh, vh, elems=el)
    gs = g.view(sp.E, sp.Q)[torch.as_tensor(el, device=dev)].double().cpu().numpy()
    tol = 1e-12 if prec == "fp64" else 1e-5
    ratio = np.abs(gs - gr) / (tol * np.sqrt(guu * gvv))
    print(f"{prec} adjoint 40^3: {gr.size} points, worst error / bound {ratio.max():.3e}")
    assert ratio.max() <= 1.0
    if prec == "fp64":
        rng = np.random.default_rng(wl.SEED_ADJ_FD)
        pts = rng.choice(sp.E * sp.Q, size=1000, replace=False)
        kap = kappa.detach().clone()
        Jb = torch.empty(1, dtype=torch.float64, device=dev)
        scale = float((kap * g).abs().sum())
        worst = 0.0
        for k in pts:
            h = 1e-6 * float(kap[k])
            kap[k] += h
            plan.backward(kap, u, v, grad=None, J=Jb)
            jp = float(Jb.item())
            kap[k] -= 2 * h
            plan.backward(kap, u, v, grad=None, J=Jb)
            jm = float(Jb.item())
            kap[k] += h
            fd = (jp - jm) / (2 * h)
            gk = float(g[k])
            bound = 1e-6 * abs(gk) + 1e-12 * scale / h
            worst = max(worst, abs(fd - gk) / bound)
        assert worst <= 1.0, worst
