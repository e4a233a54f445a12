"""GPU parity of the backward of the element matrices (iga_integrate_grad):
dL/dkappa and dL/drho at every quadrature point from upstream gradients
GK = dL/dK_e and GM = dL/dM_e, against the oracle's direct double sum over
(a, b) at every point; at the benchmark size on sampled elements and through
the linearity identity sum_q kappa_q dL/dkappa_q = <GK, K(kappa)>; and the
torch.autograd.Function over iga_integrate.  Inputs come from the seeded
generators; nothing expected comes from the CUDA path.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2207_00280_gb300 import capi
from paper_2207_00280_gb300 import workloads as wl
from paper_2207_00280_gb300.autograd import iga_integrate
from paper_2207_00280_gb300.plan import IgaPlan, Patch

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda")


def _t(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), device=DEV, dtype=dtype)


def _nonuniform_knots(p, seed, n_inner=4):
    rng = np.random.default_rng(seed)
    inner = np.sort(rng.uniform(0.08, 0.92, size=n_inner))
    if p >= 2:
        inner = np.sort(np.concatenate([inner, inner[1:2]]))
    return np.concatenate([[0.0] * (p + 1), inner, [1.0] * (p + 1)])


def _cases():
    return [
        ("p1_q2", [wl.open_uniform_knots(K, 1) for K in (3, 2, 4)], 1, 2),
        ("p1_q3", [wl.open_uniform_knots(K, 1) for K in (2, 3, 2)], 1, 3),
        ("p2_q3_nonuniform", [_nonuniform_knots(2, 31), wl.open_uniform_knots(2, 2),
                              _nonuniform_knots(2, 32)], 2, 3),
        ("p2_q4", [wl.open_uniform_knots(K, 2) for K in (2, 3, 2)], 2, 4),
        ("p3_q4", [wl.open_uniform_knots(K, 3) for K in (3, 2, 3)], 3, 4),
        ("p3_q5", [wl.open_uniform_knots(2, 3), _nonuniform_knots(3, 33), wl.open_uniform_knots(2, 3)],
         3, 5),
        ("p4_q5", [wl.open_uniform_knots(K, 4) for K in (2, 2, 3)], 4, 5),
        ("p3_c0_one_element", [np.array([0.0] * 4 + [0.3, 0.3, 0.3, 0.6] + [1.0] * 4),
                               wl.open_uniform_knots(1, 3),
                               np.array([0.0] * 4 + [0.5, 0.5] + [1.0] * 4)], 3, 4),
    ]


def _grad(plan, GK, GM, G, dtype):
    gk, gr = plan.integrate_grad(GK=_t(GK, dtype).reshape(-1) if GK is not None else None,
                                 GM=_t(GM, dtype).reshape(-1) if GM is not None else None,
                                 jac=_t(G).reshape(-1) if G is not None else None)
    torch.cuda.synchronize()
    f = (lambda x: x.cpu().numpy().astype(np.float64) if x is not None else None)
    return f(gk), f(gr)


@pytest.mark.parametrize("curved", [False, True], ids=["identity", "curved"])
@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_grad_matches_oracle(case, curved):
    _, knots, p, q = case
    P = oracle.Patch(knots, p, q)
    G = wl.curved_map_jacobian(knots, q) if curved else None
    GK = wl.normal(P.E * P.N * P.N, 1100 + p).reshape(P.E, P.N, P.N)
    GM = wl.normal(P.E * P.N * P.N, 1200 + p).reshape(P.E, P.N, P.N)
    rk, rr = P.integrate_grad(GK=GK, GM=GM, G=G)
    rk, rr = rk.reshape(-1), rr.reshape(-1)
    plan = IgaPlan(Patch(knots, p, q), method="sumfact", precision="fp64")
    gk, gr = _grad(plan, GK, GM, G, torch.float64)
    assert np.abs(gk - rk).max() <= 1e-12 * np.abs(rk).max()
    assert np.abs(gr - rr).max() <= 1e-12 * np.abs(rr).max()
    plan.close()
    if p <= 3:
        # FP64_DF plans: float-float arithmetic on the FP32 pipes, the FP64 bound
        pdf = IgaPlan(Patch(knots, p, q), method="sumfact", precision="fp64_df")
        gkd, grd = _grad(pdf, GK, GM, G, torch.float64)
        assert np.abs(gkd - rk).max() <= 1e-12 * np.abs(rk).max()
        assert np.abs(grd - rr).max() <= 1e-12 * np.abs(rr).max()
        pdf.close()
    plan32 = IgaPlan(Patch(knots, p, q), method="sumfact", precision="fp32")
    gk32, gr32 = _grad(plan32, GK, GM, G, torch.float32)
    assert np.linalg.norm(gk32 - rk) <= 1e-5 * np.linalg.norm(rk)
    assert np.linalg.norm(gr32 - rr) <= 1e-5 * np.linalg.norm(rr)
    plan32.close()


def test_one_side_only():
    """GK alone leaves grad_rho untouched and vice versa."""
    p, q = 2, 3
    knots = [wl.open_uniform_knots(K, p) for K in (2, 2, 3)]
    P = oracle.Patch(knots, p, q)
    GK = wl.normal(P.E * P.N * P.N, 1301).reshape(P.E, P.N, P.N)
    GM = wl.normal(P.E * P.N * P.N, 1302).reshape(P.E, P.N, P.N)
    rk, _ = P.integrate_grad(GK=GK)
    _, rr = P.integrate_grad(GM=GM)
    plan = IgaPlan(Patch(knots, p, q), method="sumfact", precision="fp64")
    sentinel = torch.full((plan.n_qp,), 7.0, dtype=torch.float64, device=DEV)
    gk, gr = plan.integrate_grad(GK=_t(GK).reshape(-1), grad_rho=sentinel)
    torch.cuda.synchronize()
    assert gr is None and torch.all(sentinel == 7.0)
    assert np.abs(gk.cpu().numpy() - rk.reshape(-1)).max() <= 1e-12 * np.abs(rk).max()
    _, gr = plan.integrate_grad(GM=_t(GM).reshape(-1))
    assert np.abs(gr.cpu().numpy() - rr.reshape(-1)).max() <= 1e-12 * np.abs(rr).max()
    plan.close()


def test_batch_matches_oracle():
    specs = [([wl.open_uniform_knots(K, 1) for K in (2, 3, 2)], 1),
             ([wl.open_uniform_knots(K, 3) for K in (2, 2, 3)], 3),
             ([_nonuniform_knots(2, 34)] * 3, 2)]
    plan = IgaPlan([Patch(list(k), p, p + 1) for k, p in specs], method="sumfact", precision="fp64")
    GKs, GMs, Gs, refk, refr = [], [], [], [], []
    for i, (knots, p) in enumerate(specs):
        P = oracle.Patch(knots, p, p + 1)
        GK = wl.normal(P.E * P.N * P.N, 1400 + i).reshape(P.E, P.N, P.N)
        GM = wl.normal(P.E * P.N * P.N, 1500 + i).reshape(P.E, P.N, P.N)
        G = wl.curved_map_jacobian(knots, p + 1)
        rk, rr = P.integrate_grad(GK=GK, GM=GM, G=G)
        GKs.append(GK.reshape(-1)), GMs.append(GM.reshape(-1)), Gs.append(np.asarray(G).reshape(-1))
        refk.append(rk.reshape(-1)), refr.append(rr.reshape(-1))
    gk, gr = _grad(plan, np.concatenate(GKs), np.concatenate(GMs), np.concatenate(Gs),
                   torch.float64)
    rk, rr = np.concatenate(refk), np.concatenate(refr)
    assert gk.shape == rk.shape
    assert np.abs(gk - rk).max() <= 1e-12 * np.abs(rk).max()
    assert np.abs(gr - rr).max() <= 1e-12 * np.abs(rr).max()
    plan.close()


def test_full_size_df_matches_fp64():
    """3D p=3 32^3, curved map: the float-float backward (FP64_DF plan) against
    the FP64 one within 1e-12 of the largest entry (both checked against the
    oracle on small patches), with upstream values over six decades."""
    K_el, p, q = 32, 3, 4
    t = wl.open_uniform_knots(K_el, p)
    knots = [t] * 3
    jac = _t(wl.curved_map_jacobian(knots, q)).reshape(-1)
    p64 = IgaPlan(Patch(knots, p, q), method="sumfact", precision="fp64")
    pdf = IgaPlan(Patch(knots, p, q), method="sumfact", precision="fp64_df")
    gen = torch.Generator(device=DEV).manual_seed(1651)
    n = p64.info.n_mat_entries
    GK = torch.randn(n, dtype=torch.float64, device=DEV, generator=gen)
    GK *= torch.exp(6.0 * torch.rand(n, dtype=torch.float64, device=DEV, generator=gen) - 3.0)
    GM = torch.randn(n, dtype=torch.float64, device=DEV, generator=gen)
    a_k, a_r = p64.integrate_grad(GK=GK, GM=GM, jac=jac)
    b_k, b_r = pdf.integrate_grad(GK=GK, GM=GM, jac=jac)
    torch.cuda.synchronize()
    assert float((a_k - b_k).abs().max()) <= 1e-12 * float(a_k.abs().max())
    assert float((a_r - b_r).abs().max()) <= 1e-12 * float(a_r.abs().max())
    p64.close()
    pdf.close()


def test_full_size_sampled_and_linearity():
    """3D p=3, 32^3 elements, curved map: 48 sampled elements against the
    oracle, and over the whole patch sum_q kappa_q dL/dkappa_q = <GK, K(kappa)>
    and sum_q rho_q dL/drho_q = <GM, M(rho)> with K, M from iga_integrate."""
    K_el, p, q = 32, 3, 4
    t = wl.open_uniform_knots(K_el, p)
    knots = [t] * 3
    plan = IgaPlan(Patch(knots, p, q), method="sumfact", precision="fp64")
    E, N, Q = plan.n_elements, (p + 1) ** 3, q ** 3
    G = wl.curved_map_jacobian(knots, q)
    jac = _t(G).reshape(-1)
    gen = torch.Generator(device=DEV).manual_seed(1601)
    GK = torch.randn(E * N * N, dtype=torch.float64, device=DEV, generator=gen)
    GM = torch.randn(E * N * N, dtype=torch.float64, device=DEV, generator=gen)
    kappa = _t(wl.lognormal(E * Q, 1602))
    rho = _t(wl.lognormal(E * Q, 1603))
    gk, gr = plan.integrate_grad(GK=GK, GM=GM, jac=jac)
    K, M, _ = plan.empty_outputs(dof=False)
    plan.integrate(kappa=kappa, rho=rho, jac=jac, K=K, M=M)
    torch.cuda.synchronize()
    lk, rk_ = float((kappa * gk).sum()), float((GK * K).sum())
    lm, rm_ = float((rho * gr).sum()), float((GM * M).sum())
    assert abs(lk - rk_) <= 1e-11 * float((GK * K).abs().sum())
    assert abs(lm - rm_) <= 1e-11 * float((GM * M).abs().sum())
    rng = np.random.default_rng(1604)
    elems = np.sort(rng.choice(E, size=48, replace=False))
    P = oracle.Patch(knots, p, q)
    GKs = GK.view(E, N, N)[torch.as_tensor(elems, device=DEV)].cpu().numpy()
    GMs = GM.view(E, N, N)[torch.as_tensor(elems, device=DEV)].cpu().numpy()
    ok, orr = P.integrate_grad(GK=GKs, GM=GMs, G=G, elems=elems)
    gks = gk.view(E, Q)[torch.as_tensor(elems, device=DEV)].cpu().numpy()
    grs = gr.view(E, Q)[torch.as_tensor(elems, device=DEV)].cpu().numpy()
    assert np.abs(gks - ok).max() <= 1e-12 * np.abs(ok).max()
    assert np.abs(grs - orr).max() <= 1e-12 * np.abs(orr).max()
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_autograd_integrate(precision):
    """L = <GK, K(kappa)> + <GM, M(rho)> through torch.autograd: the gradients
    equal the oracle's; L itself is checked against the oracle's matrices."""
    p, q = 2, 3
    knots = [wl.open_uniform_knots(K, p) for K in (3, 2, 2)]
    P = oracle.Patch(knots, p, q)
    G = wl.curved_map_jacobian(knots, q)
    GK = wl.normal(P.E * P.N * P.N, 1701).reshape(P.E, P.N, P.N)
    GM = wl.normal(P.E * P.N * P.N, 1702).reshape(P.E, P.N, P.N)
    kap = wl.lognormal(P.E * P.Q, 1703)
    rh = wl.lognormal(P.E * P.Q, 1704)
    rk, rr = P.integrate_grad(GK=GK, GM=GM, G=G)
    Ke, Me = P.classical(kappa=kap, rho=rh, G=G)
    plan = IgaPlan(Patch(knots, p, q), method="sumfact", precision=precision)
    dt = plan.out_dtype
    kappa = _t(kap).requires_grad_(True)
    rho = _t(rh).requires_grad_(True)
    K, M = iga_integrate(plan, kappa, rho, jac=_t(G).reshape(-1))
    L = (_t(GK, dt).reshape(-1) * K).sum() + (_t(GM, dt).reshape(-1) * M).sum()
    L.backward()
    tol = 1e-12 if precision == "fp64" else 1e-5
    Lref = float((GK * Ke).sum() + (GM * Me).sum())
    assert abs(float(L.detach()) - Lref) <= tol * 10 * float(np.abs(GK * Ke).sum() + np.abs(GM * Me).sum())
    gk, gr = kappa.grad.cpu().numpy(), rho.grad.cpu().numpy()
    assert np.linalg.norm(gk - rk.reshape(-1)) <= tol * np.linalg.norm(rk)
    assert np.linalg.norm(gr - rr.reshape(-1)) <= tol * np.linalg.norm(rr)
    plan.close()


def _jac2d(n_qp, seed):
    """Seeded non-symmetric 2x2 Jacobians with positive determinant."""
    a = wl.normal(4 * n_qp, seed).reshape(n_qp, 2, 2)
    return np.eye(2)[None] + 0.15 * a


@pytest.mark.parametrize("curved", [False, True], ids=["identity", "curved"])
@pytest.mark.parametrize("p,dq", [(1, 1), (2, 1), (2, 2), (3, 1), (4, 2), (5, 1)])
def test_grad_2d_matches_oracle(p, dq, curved):
    """2D (FP64 plans; the FP32 forms are 3D)."""
    q = p + dq
    knots = [wl.open_uniform_knots(4, p), _nonuniform_knots(p, 35 + p)]
    P = oracle.Patch(knots, p, q)
    G = _jac2d(P.E * P.Q, 1800 + p) if curved else None
    GK = wl.normal(P.E * P.N * P.N, 1810 + p).reshape(P.E, P.N, P.N)
    GM = wl.normal(P.E * P.N * P.N, 1820 + p).reshape(P.E, P.N, P.N)
    rk, rr = P.integrate_grad(GK=GK, GM=GM, G=G)
    rk, rr = rk.reshape(-1), rr.reshape(-1)
    plan = IgaPlan(Patch(knots, p, q), method="sumfact", precision="fp64")
    gk, gr = _grad(plan, GK, GM, G, torch.float64)
    assert np.abs(gk - rk).max() <= 1e-12 * np.abs(rk).max()
    assert np.abs(gr - rr).max() <= 1e-12 * np.abs(rr).max()
    plan.close()


@pytest.mark.parametrize("p,q,curved", [(4, 6, True), (5, 6, False), (5, 6, True)])
def test_grad_high_degree(p, q, curved):
    """3D p = 4 with q = 6 (FP64 and FP32) and p = 5 (FP32 only: the padded
    FP64 block of 216 x 217 values exceeds shared memory)."""
    knots = [wl.open_uniform_knots(K, p) for K in (2, 1, 2)]
    P = oracle.Patch(knots, p, q)
    G = wl.curved_map_jacobian(knots, q) if curved else None
    GK = wl.normal(P.E * P.N * P.N, 1900 + p).reshape(P.E, P.N, P.N)
    GM = wl.normal(P.E * P.N * P.N, 1910 + p).reshape(P.E, P.N, P.N)
    rk, rr = P.integrate_grad(GK=GK, GM=GM, G=G)
    rk, rr = rk.reshape(-1), rr.reshape(-1)
    for pr, dt, tol in (("fp64", torch.float64, 1e-12), ("fp32", torch.float32, 1e-5)):
        plan = IgaPlan(Patch(knots, p, q), method="sumfact", precision=pr)
        if pr == "fp64" and p == 5:
            g = torch.zeros(plan.info.n_mat_entries, dtype=dt, device=DEV)
            with pytest.raises(capi.IgaError) as ei:
                plan.integrate_grad(GK=g)
            assert ei.value.code == capi.IGA_ERR_UNSUPPORTED
            plan.close()
            continue
        gk, gr = _grad(plan, GK, GM, G, dt)
        assert np.linalg.norm(gk - rk) <= tol * np.linalg.norm(rk)
        assert np.linalg.norm(gr - rr) <= tol * np.linalg.norm(rr)
        plan.close()


def test_unsupported_and_bad_arguments():
    t2 = wl.open_uniform_knots(3, 6)
    plan2d = IgaPlan(Patch([t2] * 2, 6, 7), method="sumfact")
    g = torch.zeros(plan2d.info.n_mat_entries, dtype=torch.float64, device=DEV)
    with pytest.raises(capi.IgaError) as ei:
        plan2d.integrate_grad(GK=g)
    assert ei.value.code == capi.IGA_ERR_UNSUPPORTED
    plan2d.close()
    t5 = wl.open_uniform_knots(2, 5)
    plan5 = IgaPlan(Patch([t5] * 3, 5, 6), method="sumfact")
    g = torch.zeros(plan5.info.n_mat_entries, dtype=torch.float64, device=DEV)
    with pytest.raises(capi.IgaError) as ei:
        plan5.integrate_grad(GK=g)
    assert ei.value.code == capi.IGA_ERR_UNSUPPORTED
    plan5.close()
    t3 = wl.open_uniform_knots(2, 3)
    plan = IgaPlan(Patch([t3] * 3, 3, 4), method="sumfact")
    g = torch.zeros(plan.info.n_mat_entries, dtype=torch.float64, device=DEV)
    out = torch.zeros(plan.n_qp, dtype=torch.float64, device=DEV)
    s = torch.cuda.current_stream().cuda_stream
    assert capi.iga_integrate_grad(plan.handle, None, None, None, None, None, s) == capi.IGA_ERR_ARG
    assert capi.iga_integrate_grad(plan.handle, None, g.data_ptr(), None, None, None, s) == \
        capi.IGA_ERR_ARG
    assert capi.iga_integrate_grad(plan.handle, None, None, g.data_ptr(), out.data_ptr(), None, s) == \
        capi.IGA_ERR_ARG
    plan.close()
