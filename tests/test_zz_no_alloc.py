"""iga_adjoint_noalloc: the adjoint for callers that cannot allocate device
memory (they run inside a memory pool or arena they do not own, or in a loop
that must never enter the allocator, so they cannot build a plan).  Its
working memory is a fixed device array inside the library.

Checked through the C ABI against the oracle's adjoint and against the
plan-based iga_integrate_backward on the same inputs, for three calls in a row
(the shared array keeps the previous call's contents when the next one runs).
Collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2207_00280_gb300 import capi
from paper_2207_00280_gb300 import workloads as wl
from paper_2207_00280_gb300.plan import IgaPlan, Patch

pytestmark = pytest.mark.gpu
dev = torch.device("cuda")
TOL = 1e-12  # the FP64 tolerance of the other GPU tests


def _desc(knots, p, q):
    d = capi.PatchDesc()
    d.dim = 3
    d.set_order(p, q)
    keep = [np.ascontiguousarray(t, dtype=np.float64) for t in knots]
    for k, t in enumerate(keep):
        d.n_knots[k] = len(t)
        d.knots[k] = t.ctypes.data
    return d, keep


def _noalloc(knots, p, q, kappa, jac, u, v):
    d, keep = _desc(knots, p, q)
    n_qp = kappa.numel()
    g = torch.full((n_qp,), float("nan"), dtype=torch.float64, device=dev)
    J = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
    rc = capi.lib().iga_adjoint_noalloc(
        ctypes.byref(d), ptr(kappa), ptr(jac), ptr(u), ptr(v), ptr(g), ptr(J),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == capi.IGA_OK, capi.iga_status_str(rc)
    torch.cuda.synchronize()
    return g, float(J.item())


@pytest.mark.parametrize("curved", [False, True])
def test_noalloc_matches_oracle_and_plan(oracle_mod, curved):
    # different calls in a row; the last one (degree 7) runs the runtime-sized adjoint
    cases = [(3, 4, (7, 5, 6), 31), (2, 3, (9, 4, 5), 32), (7, 8, (2, 2, 1), 33)]
    for p, q, Ks, seed in cases:
        knots = [wl.open_uniform_knots(K, p) for K in Ks]
        E, Q = int(np.prod(Ks)), q ** 3
        kappa = torch.as_tensor(wl.lognormal(E * Q, seed), device=dev)
        jac = (torch.as_tensor(wl.curved_map_jacobian(knots, q), device=dev).reshape(-1)
               if curved else None)
        nd = int(np.prod([K + p for K in Ks]))
        u = torch.as_tensor(wl.normal(nd, seed + 1), device=dev)
        v = torch.as_tensor(wl.normal(nd, seed + 2), device=dev)
        plan = IgaPlan(Patch(knots, p, q), method="sumfact", precision="fp64")
        g_ref = torch.empty(plan.n_qp, dtype=torch.float64, device=dev)
        J_ref = torch.empty(1, dtype=torch.float64, device=dev)
        plan.backward(kappa, u, v, grad=g_ref, J=J_ref, jac=jac)
        g, J = _noalloc(knots, p, q, kappa, jac, u, v)
        # the oracle (plain C, FP64) on the same inputs
        P = oracle_mod.Patch(knots, p, q)
        G = wl.curved_map_jacobian(knots, q) if curved else None
        gr, Jr = P.adjoint(u.cpu().numpy(), v.cpu().numpy(), kappa=kappa.cpu().numpy(), G=G)
        gr = gr.reshape(-1)
        assert np.abs(g.cpu().numpy() - gr).max() <= TOL * np.abs(gr).max()
        assert J == pytest.approx(Jr, rel=TOL, abs=1e-13 * np.abs(kappa.cpu().numpy() * gr).sum())
        scale = float(g_ref.abs().max())
        assert float((g - g_ref).abs().max()) <= TOL * scale
        assert J == pytest.approx(float(J_ref.item()), rel=TOL)
        plan.close()


def test_noalloc_rejects_too_large():
    p, q = 3, 4
    knots = [wl.open_uniform_knots(1100, p), wl.open_uniform_knots(2, p), wl.open_uniform_knots(2, p)]
    d, keep = _desc(knots, p, q)
    x = torch.zeros(8, dtype=torch.float64, device=dev)
    ptr = ctypes.c_void_p(x.data_ptr())
    rc = capi.lib().iga_adjoint_noalloc(ctypes.byref(d), ptr, None, ptr, ptr, ptr, None, None)
    assert rc == capi.IGA_ERR_TOO_LARGE
    assert "IGA_ERR_TOO_LARGE" in capi.iga_status_str(rc)
