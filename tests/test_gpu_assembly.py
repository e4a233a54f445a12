"""GPU parity of the assembled (CSR) form and of the matrix-free operator.

Global assembly (iga_csr_pattern, iga_assemble) is integer and summation work
in a fixed order: the pattern must equal the oracle's bit for bit, and so must
the FP64 values (both sum the same element entries in ascending element
order).  The operator (iga_apply) is compared with the oracle's element-matrix
product within the FP64 / FP32 tolerances, and at the benchmark sizes with
closed forms (K 1 = 0, M 1 = integrals of the B-splines, boundary flux of a
linear field).  Inputs come from the seeded generators; nothing expected comes
from the CUDA path.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import run_gpu
from paper_2207_00280_gb300 import workloads as wl
from paper_2207_00280_gb300.autograd import iga_apply, iga_bilinear
from paper_2207_00280_gb300.plan import IgaPlan, Patch

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda")


def _nonuniform_knots(p, seed, n_inner=5):
    rng = np.random.default_rng(seed)
    inner = np.sort(rng.uniform(0.08, 0.92, size=n_inner))
    if p >= 2:
        inner = np.sort(np.concatenate([inner, inner[1:2]]))
    return np.concatenate([[0.0] * (p + 1), inner, [1.0] * (p + 1)])


def _patch_sets():
    return {
        "2d_p2_uniform": [([wl.open_uniform_knots(7, 2)] * 2, 2)],
        "2d_p5_mixed": [([wl.open_uniform_knots(4, 5), _nonuniform_knots(5, 3)], 5)],
        "3d_p1": [([wl.open_uniform_knots(5, 1)] * 3, 1)],
        "3d_p3_uniform": [([wl.open_uniform_knots(6, 3)] * 3, 3)],
        "3d_p2_nonuniform": [([_nonuniform_knots(2, 4), wl.open_uniform_knots(3, 2),
                               _nonuniform_knots(2, 5)], 2)],
        "3d_p5": [([wl.open_uniform_knots(3, 5)] * 3, 5)],
        # a C0 line (interior knot of multiplicity p), one element in y, a double knot in z
        "3d_p3_c0_one_element": [([np.array([0.0] * 4 + [0.3, 0.3, 0.3, 0.6] + [1.0] * 4),
                                   wl.open_uniform_knots(1, 3),
                                   np.array([0.0] * 4 + [0.5, 0.5] + [1.0] * 4)], 3)],
        "3d_batch": [([wl.open_uniform_knots(3, 1)] * 3, 1),
                     ([wl.open_uniform_knots(4, 3), wl.open_uniform_knots(3, 3),
                       wl.open_uniform_knots(5, 3)], 3),
                     ([_nonuniform_knots(2, 6)] * 3, 2)],
    }


def _oracle_pattern(specs):
    rows, cols, nnz, dofs = [np.zeros(1, dtype=np.int64)], [], 0, 0
    for knots, p in specs:
        P = oracle.Patch(knots, p, p + 1)
        rp, ci = P.csr_pattern()
        rows.append(rp[1:] + nnz)
        cols.append(ci + dofs)
        nnz += int(rp[-1])
        dofs += P.n_dofs
    return np.concatenate(rows), np.concatenate(cols)


def _plan(specs, precision="fp64", **kw):
    return IgaPlan([Patch(list(k), p, p + 1) for k, p in specs], method="sumfact",
                   precision=precision, **kw)


@pytest.mark.parametrize("name", sorted(_patch_sets()))
def test_csr_pattern_bit_exact(name):
    specs = _patch_sets()[name]
    plan = _plan(specs)
    rp, ci = plan.csr_pattern()
    torch.cuda.synchronize()
    rref, cref = _oracle_pattern(specs)
    assert plan.n_csr_nnz == len(cref)
    assert np.array_equal(rp.cpu().numpy(), rref)
    assert np.array_equal(ci.cpu().numpy(), cref)
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", sorted(_patch_sets()))
def test_assemble_bit_exact(name, precision):
    """Seeded random (non-symmetric) element matrices.  FP64: the GPU sums in
    ascending element order like the oracle, so the values agree bit for bit.
    FP32: the GPU sums in FP32 (same order), within 1e-6 of the FP64 sums of
    the same FP32 inputs relative to the row's largest entry, and the same
    bits on a second call."""
    if precision == "fp32" and name.startswith("2d"):
        pytest.skip("FP32 plans are 3D only")
    specs = _patch_sets()[name]
    plan = _plan(specs, precision=precision)
    n = plan.info.n_mat_entries
    A = wl.normal(n, 77)
    if precision == "fp32":
        A = A.astype(np.float32).astype(np.float64)
    At = torch.as_tensor(A, device=DEV, dtype=plan.out_dtype)
    vals = plan.assemble(At).cpu().numpy()
    ref = []
    for i, (knots, p) in enumerate(specs):
        P = oracle.Patch(knots, p, p + 1)
        rp, ci = P.csr_pattern()
        ref.append(P.assemble(A[plan.mat_offset[i]:plan.mat_offset[i + 1]], rp, ci))
    ref = np.concatenate(ref)
    if precision == "fp32":
        assert vals.dtype == np.float32
        # each value sums at most (p+1)^d terms of size O(1)
        assert np.abs(vals - ref).max() <= 1e-6 * np.abs(A).max() * 64
        again = plan.assemble(At).cpu().numpy()
        assert np.array_equal(vals, again)
    else:
        assert vals.dtype == ref.dtype
        assert np.array_equal(vals, ref)
    plan.close()


def test_assemble_mid_size_bit_exact():
    """3D p=3, 12^3 elements (7M element entries): bit-exact FP64 assembly."""
    specs = [([wl.open_uniform_knots(12, 3)] * 3, 3)]
    plan = _plan(specs)
    A = wl.normal(plan.info.n_mat_entries, 78)
    vals = plan.assemble(torch.as_tensor(A, device=DEV)).cpu().numpy()
    P = oracle.Patch(specs[0][0], 3, 4)
    rp, ci = P.csr_pattern()
    assert np.array_equal(vals, P.assemble(A, rp, ci))
    plan.close()


def _bspline_integrals(t, p):
    nf = len(t) - p - 1
    return np.array([(t[i + p + 1] - t[i]) / (p + 1) for i in range(nf)])


def test_assemble_full_size_row_sums():
    """3D p=3 32^3 (benchmark size): the assembled mass has row sums
    int phi_i (closed form) and the assembled stiffness has zero row sums."""
    K_el, p = 32, 3
    knots = [wl.open_uniform_knots(K_el, p)] * 3
    kappa = wl.lognormal(K_el ** 3 * 64, wl.SEED_KAPPA_P3)
    out = run_gpu(knots, p, p + 1, kappa=kappa, dof=False)
    plan = out["plan"]
    rp, ci = plan.csr_pattern()
    Mv = plan.assemble(out["M"].reshape(-1))
    Kv = plan.assemble(out["K"].reshape(-1))
    seg = torch.repeat_interleave(torch.arange(plan.n_dofs, device=DEV), rp[1:] - rp[:-1])
    msum = torch.zeros(plan.n_dofs, dtype=torch.float64, device=DEV).index_add_(0, seg, Mv)
    ksum = torch.zeros(plan.n_dofs, dtype=torch.float64, device=DEV).index_add_(0, seg, Kv)
    b = _bspline_integrals(knots[0], p)
    ref = np.einsum("k,j,i->kji", b, b, b).reshape(-1)
    assert np.abs(msum.cpu().numpy() - ref).max() <= 1e-13 * ref.max()
    assert float(ksum.abs().max()) <= 1e-12 * float(Kv.abs().max())
    plan.close()


def _apply_cases():
    return [
        ("uniform_p1", [wl.open_uniform_knots(4, 1)] * 3, 1, False),
        ("uniform_p3_curved", [wl.open_uniform_knots(4, 3)] * 3, 3, True),
        ("nonuniform_p2_curved", [_nonuniform_knots(2, 8), wl.open_uniform_knots(3, 2),
                                  _nonuniform_knots(2, 9)], 2, True),
        ("uniform_p4", [wl.open_uniform_knots(3, 4)] * 3, 4, False),
        ("uniform_p5_curved", [wl.open_uniform_knots(2, 5)] * 3, 5, True),
        ("c0_one_element_p3_curved", [np.array([0.0] * 4 + [0.3, 0.3, 0.3, 0.6] + [1.0] * 4),
                                      wl.open_uniform_knots(1, 3),
                                      np.array([0.0] * 4 + [0.5, 0.5] + [1.0] * 4)], 3, True),
    ]


@pytest.mark.parametrize("precision", ["fp64", "fp64_df", "fp32"])
@pytest.mark.parametrize("case", _apply_cases(), ids=lambda c: c[0])
def test_apply_matches_oracle(case, precision):
    _, knots, p, curved = case
    P = oracle.Patch(knots, p, p + 1)
    kappa = wl.lognormal(P.E * P.Q, 41)
    rho = wl.lognormal(P.E * P.Q, 42)
    G = wl.curved_map_jacobian(knots, p + 1) if curved else None
    x = wl.normal(P.n_dofs, 43)
    yK, yM = P.apply(x, kappa=kappa, rho=rho, G=G)
    plan = IgaPlan(Patch(list(knots), p, p + 1), method="sumfact", precision=precision)
    dt = plan.out_dtype
    kt = torch.as_tensor(kappa, device=DEV)
    rt = torch.as_tensor(rho, device=DEV)
    jt = torch.as_tensor(G, device=DEV).reshape(-1) if curved else None
    xt = torch.as_tensor(x, device=DEV, dtype=dt)
    tol = 1e-5 if precision == "fp32" else 1e-12   # fp64_df: float-float, FP64 accuracy
    for alpha, beta, ref in ((1.0, 0.0, yK), (0.0, 1.0, yM), (-0.25, 2.0, -0.25 * yK + 2.0 * yM)):
        y = plan.apply(xt, kappa=kt, rho=rt, jac=jt, alpha=alpha, beta=beta).cpu().numpy()
        err = np.abs(y - ref).max() / np.abs(ref).max()
        assert err <= tol, (alpha, beta, err)
    plan.close()


@pytest.mark.parametrize("curved", [False, True], ids=["identity", "general"])
@pytest.mark.parametrize("p,dq", [(1, 1), (2, 1), (2, 2), (3, 1), (4, 2), (5, 1)])
def test_apply_2d_matches_oracle(p, dq, curved):
    """2D operator (FP64 plans; the FP32 forms are 3D): against the oracle's
    element-matrix product, alpha K + beta M for three (alpha, beta), and
    K 1 = 0 on a general map."""
    q = p + dq
    knots = [wl.open_uniform_knots(5, p), _nonuniform_knots(p, 70 + p)]
    P = oracle.Patch(knots, p, q)
    kappa = wl.lognormal(P.E * P.Q, 71)
    rho = wl.lognormal(P.E * P.Q, 72)
    G = None
    if curved:
        G = np.eye(2)[None] + 0.15 * wl.normal(4 * P.E * P.Q, 73).reshape(P.E * P.Q, 2, 2)
    x = wl.normal(P.n_dofs, 74)
    yK, yM = P.apply(x, kappa=kappa, rho=rho, G=G)
    plan = IgaPlan(Patch(list(knots), p, q), method="sumfact", precision="fp64")
    kt = torch.as_tensor(kappa, device=DEV)
    rt = torch.as_tensor(rho, device=DEV)
    jt = torch.as_tensor(G, device=DEV).reshape(-1) if curved else None
    xt = torch.as_tensor(x, device=DEV)
    for alpha, beta, ref in ((1.0, 0.0, yK), (0.0, 1.0, yM), (-0.25, 2.0, -0.25 * yK + 2.0 * yM)):
        y = plan.apply(xt, kappa=kt, rho=rt, jac=jt, alpha=alpha, beta=beta).cpu().numpy()
        assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max(), (alpha, beta)
    ones = torch.ones(plan.n_dofs, dtype=torch.float64, device=DEV)
    y1 = plan.apply(ones, kappa=kt, jac=jt).cpu().numpy()
    assert np.abs(y1).max() <= 1e-12 * np.abs(yK).max()
    plan.close()


def test_apply_batch_matches_oracle():
    specs = _patch_sets()["3d_batch"]
    plan = _plan(specs)
    kappa = wl.lognormal(plan.n_qp, 44)
    x = wl.normal(plan.n_dofs, 45)
    y = plan.apply(torch.as_tensor(x, device=DEV), kappa=torch.as_tensor(kappa, device=DEV),
                   beta=0.5).cpu().numpy()
    for i, (knots, p) in enumerate(specs):
        P = oracle.Patch(knots, p, p + 1)
        d0, d1 = plan.dof_offset[i], plan.dof_offset[i + 1]
        q0, q1 = plan.qp_offset[i], plan.qp_offset[i + 1]
        yK, yM = P.apply(x[d0:d1], kappa=kappa[q0:q1])
        ref = yK + 0.5 * yM
        assert np.abs(y[d0:d1] - ref).max() <= 1e-12 * np.abs(ref).max()
    plan.close()


def test_apply_deterministic():
    knots = [wl.open_uniform_knots(6, 3)] * 3
    plan = IgaPlan(Patch(knots, 3, 4), method="sumfact", precision="fp64")
    kappa = torch.as_tensor(wl.lognormal(plan.n_qp, 46), device=DEV)
    x = torch.as_tensor(wl.normal(plan.n_dofs, 47), device=DEV)
    y1 = plan.apply(x, kappa=kappa, beta=1.0)
    y2 = plan.apply(x, kappa=kappa, beta=1.0)
    assert torch.equal(y1, y2)
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_apply_full_size_closed_forms(precision):
    """3D p=3 40^3 (adjoint workload size), kappa = 1, identity geometry:
    K 1 = 0, M 1 = int phi_i, and K x = boundary flux for x the Greville
    abscissae of direction 0 (a linear field)."""
    K_el, p = 40, 3
    t = wl.open_uniform_knots(K_el, p)
    plan = IgaPlan(Patch([t] * 3, p, p + 1), method="sumfact", precision=precision)
    dt = plan.out_dtype
    nf = len(t) - p - 1
    ones = torch.ones(plan.n_dofs, dtype=dt, device=DEV)
    yK = plan.apply(ones).cpu().numpy()
    yM = plan.apply(ones, alpha=0.0, beta=1.0).cpu().numpy()
    b = _bspline_integrals(t, p)
    ref = np.einsum("k,j,i->kji", b, b, b).reshape(-1)
    tol = 1e-12 if precision == "fp64" else 1e-5
    assert np.abs(yM - ref).max() <= tol * ref.max()
    gre = np.array([np.mean(t[i + 1:i + p + 1]) for i in range(nf)])
    x = np.broadcast_to(gre[None, None, :], (nf, nf, nf)).reshape(-1)
    yx = plan.apply(torch.as_tensor(x.copy(), device=DEV, dtype=dt)).cpu().numpy()
    jump = np.zeros(nf)
    jump[0], jump[-1] = -1.0, 1.0
    flux = np.einsum("k,j,i->kji", b, b, jump).reshape(-1)
    scale = np.abs(flux).max()
    assert np.abs(yK).max() <= tol * 1e2 * scale
    assert np.abs(yx - flux).max() <= tol * 1e2 * scale
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_bilinear_grads_wrt_u_v(precision):
    """dJ/du = K v and dJ/dv = K u for J = u^T K(kappa) v, against the oracle."""
    knots = [wl.open_uniform_knots(3, 2)] * 3
    P = oracle.Patch(knots, 2, 3)
    kappa = wl.lognormal(P.E * P.Q, 48)
    G = wl.curved_map_jacobian(knots, 3)
    u, v = wl.normal(P.n_dofs, 49), wl.normal(P.n_dofs, 50)
    plan = IgaPlan(Patch(knots, 2, 3), method="sumfact", precision=precision)
    dt = plan.out_dtype
    kt = torch.as_tensor(kappa, device=DEV).requires_grad_(True)
    ut = torch.as_tensor(u, device=DEV, dtype=dt).requires_grad_(True)
    vt = torch.as_tensor(v, device=DEV, dtype=dt).requires_grad_(True)
    jt = torch.as_tensor(G, device=DEV).reshape(-1)
    J = iga_bilinear(kt, ut, vt, plan, jac=jt)
    (2.0 * J).backward()
    Kv, _ = P.apply(v, kappa=kappa, G=G, mass=False)
    Ku, _ = P.apply(u, kappa=kappa, G=G, mass=False)
    tol = 1e-12 if precision == "fp64" else 1e-5
    for got, ref in ((ut.grad, 2 * Kv), (vt.grad, 2 * Ku)):
        g = got.detach().cpu().numpy()
        assert np.abs(g - ref).max() <= tol * np.abs(ref).max()
    g_ref, _ = P.adjoint(u, v, kappa=kappa, G=G)
    gk = kt.grad.detach().cpu().numpy()
    assert np.abs(gk - 2 * g_ref.reshape(-1)).max() <= tol * 2 * np.abs(g_ref).max()
    plan.close()


def test_apply_function_gradients():
    """IgaApply: dL/dx = K g_y (symmetric operator) and dL/dkappa equal the
    oracle's operator and adjoint, for L = w . y, y = K(kappa) x + 0.5 M x."""
    knots = [wl.open_uniform_knots(3, 3)] * 3
    P = oracle.Patch(knots, 3, 4)
    kappa = wl.lognormal(P.E * P.Q, 51)
    x, w = wl.normal(P.n_dofs, 52), wl.normal(P.n_dofs, 53)
    plan = IgaPlan(Patch(knots, 3, 4), method="sumfact", precision="fp64")
    kt = torch.as_tensor(kappa, device=DEV).requires_grad_(True)
    xt = torch.as_tensor(x, device=DEV).requires_grad_(True)
    y = iga_apply(kt, xt, plan, alpha=1.0, beta=0.5)
    (torch.as_tensor(w, device=DEV) * y).sum().backward()
    Kw, Mw = P.apply(w, kappa=kappa)
    ref_x = Kw + 0.5 * Mw
    assert np.abs(xt.grad.cpu().numpy() - ref_x).max() <= 1e-12 * np.abs(ref_x).max()
    g_ref, _ = P.adjoint(w, x, kappa=kappa)
    assert np.abs(kt.grad.cpu().numpy() - g_ref.reshape(-1)).max() <= 1e-12 * np.abs(g_ref).max()
    plan.close()
