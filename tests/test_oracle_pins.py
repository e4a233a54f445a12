"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed forms,
library routines (numpy's Gauss--Legendre, scipy's B-splines), exact rational
integrals, structural identities, or a different computation of the same
quantity.  CPU only.
"""
import math

import numpy as np
import pytest

from exact1d import element_matrices_1d, rational_open_uniform
from paper_2207_00280_gb300 import workloads as wl


# --------------------------------------------------------------------------
# Gauss--Legendre (the quadrature of eq. 10)
# --------------------------------------------------------------------------

def test_gauss_closed_forms(oracle_mod):
    x, w = oracle_mod.gauss_legendre(1)
    assert x[0] == pytest.approx(0.0, abs=1e-16) and w[0] == pytest.approx(2.0, rel=1e-15)
    x, w = oracle_mod.gauss_legendre(2)
    np.testing.assert_allclose(x, [-1 / math.sqrt(3), 1 / math.sqrt(3)], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, [1.0, 1.0], rtol=2e-15)
    x, w = oracle_mod.gauss_legendre(3)
    np.testing.assert_allclose(x, [-math.sqrt(0.6), 0.0, math.sqrt(0.6)], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, [5 / 9, 8 / 9, 5 / 9], rtol=2e-15)


@pytest.mark.parametrize("q", range(1, 17))
def test_gauss_exactness_and_numpy(oracle_mod, q):
    x, w = oracle_mod.gauss_legendre(q)
    assert np.all(np.diff(x) > 0)
    assert w.sum() == pytest.approx(2.0, rel=1e-14)
    for k in range(2 * q):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14, k
    # degree 2q is not integrated exactly: the Gauss error for x^(2q) is
    # 2^(2q+1) (q!)^4 / ((2q+1) ((2q)!)^2)
    err = 2.0 / (2 * q + 1) - np.dot(w, x ** (2 * q))
    ref = 2.0 ** (2 * q + 1) * math.factorial(q) ** 4 / ((2 * q + 1) * math.factorial(2 * q) ** 2)
    assert err == pytest.approx(ref, rel=1e-4)
    xn, wn = np.polynomial.legendre.leggauss(q)
    np.testing.assert_allclose(x, xn, rtol=0, atol=4e-16 * q)
    np.testing.assert_allclose(w, wn, rtol=2e-14 * q, atol=0)


# --------------------------------------------------------------------------
# Cox--de Boor (eqs. cox1/cox2) and its derivative
# --------------------------------------------------------------------------

def _knot_vectors():
    out = []
    for p in range(1, 9):
        out.append((wl.open_uniform_knots(7, p), p))
    rng = np.random.default_rng(5)
    for p in range(1, 6):
        inner = np.sort(rng.uniform(0.05, 0.95, size=6))
        inner = np.concatenate([inner, inner[:1]]) if p >= 2 else inner  # one double knot
        inner = np.sort(inner)
        out.append((np.concatenate([[0.0] * (p + 1), inner, [1.0] * (p + 1)]), p))
    return out


@pytest.mark.parametrize("t,p", _knot_vectors())
def test_bspline_vs_scipy(oracle_mod, t, p):
    from scipy.interpolate import BSpline
    nf = len(t) - p - 1
    rng = np.random.default_rng(11)
    pts = rng.uniform(0.0, 1.0, size=60)
    for i in range(nf):
        c = np.zeros(nf); c[i] = 1.0
        sp = BSpline(t, c, p, extrapolate=False)
        dsp = sp.derivative()
        for xi in pts:
            ref = float(sp(xi))
            assert abs(oracle_mod.bspline(t, i, p, xi) - ref) < 1e-14
            assert abs(oracle_mod.bspline_deriv(t, i, p, xi) - float(dsp(xi))) < 1e-11 * max(1, len(t))


@pytest.mark.parametrize("p", range(1, 9))
def test_partition_of_unity_and_support(oracle_mod, p):
    t = wl.open_uniform_knots(9, p)
    nf = len(t) - p - 1
    assert nf == 9 + p  # K + p functions (Sec. 2.3)
    rng = np.random.default_rng(p)
    pts = list(rng.uniform(0.0, 1.0, size=200))
    for s in oracle_mod.spans(t, p):
        xi, _, _, _ = oracle_mod.basis_1d(t, p, int(s), p + 1)
        pts += list(xi)
    for xi in pts:
        vals = np.array([oracle_mod.bspline(t, i, p, xi) for i in range(nf)])
        ders = np.array([oracle_mod.bspline_deriv(t, i, p, xi) for i in range(nf)])
        assert abs(vals.sum() - 1.0) <= 1e-15 * 4
        assert abs(ders.sum()) <= 1e-12
        assert np.all(vals >= 0.0)
        assert np.count_nonzero(vals) == p + 1  # interior point: exactly p+1 non-zeros


@pytest.mark.parametrize("p", range(1, 7))
def test_derivative_vs_central_difference(oracle_mod, p):
    t = wl.open_uniform_knots(6, p)
    h = 1e-6
    rng = np.random.default_rng(100 + p)
    for xi in rng.uniform(0.01, 0.99, size=40):
        for i in range(len(t) - p - 1):
            fd = (oracle_mod.bspline(t, i, p, xi + h) - oracle_mod.bspline(t, i, p, xi - h)) / (2 * h)
            d = oracle_mod.bspline_deriv(t, i, p, xi)
            # a knot inside [xi-h, xi+h] makes the difference one-sided; skip those
            if np.any(np.abs(t - xi) < 2 * h):
                continue
            assert abs(fd - d) <= 1e-8 * max(1.0, abs(d)) * 40


def test_cardinal_quadratic(oracle_mod):
    K, p = 10, 2
    t = wl.open_uniform_knots(K, p)
    h = 1.0 / K
    spans = oracle_mod.spans(t, p)
    for e in range(2, K - 2):
        s = int(spans[e])
        for tt in np.linspace(0.05, 0.95, 7):
            xi = t[s] + tt * h
            ref = [(1 - tt) ** 2 / 2, (-2 * tt * tt + 2 * tt + 1) / 2, tt * tt / 2]
            got = [oracle_mod.bspline(t, s - 2 + r, p, xi) for r in range(3)]
            np.testing.assert_allclose(got, ref, rtol=0, atol=2e-15)


def test_spans_brute_force(oracle_mod):
    rng = np.random.default_rng(3)
    for p in range(1, 6):
        inner = np.sort(rng.choice(np.linspace(0.1, 0.9, 9), size=7))  # repeats likely
        t = np.concatenate([[0.0] * (p + 1), inner, [1.0] * (p + 1)])
        ref = [s for s in range(p, len(t) - p - 1) if t[s] < t[s + 1]]
        assert list(oracle_mod.spans(t, p)) == ref
        # every interior point lies in exactly one reported span
        for xi in rng.uniform(0, 1, 50):
            assert sum(t[s] <= xi < t[s + 1] for s in ref) == 1


# --------------------------------------------------------------------------
# Element matrices: exact closed forms
# --------------------------------------------------------------------------

def _kron_all(mats):
    """mats[0] (x) mats[1] (x) ... ; the last factor's index runs fastest."""
    out = mats[0]
    for m in mats[1:]:
        out = np.kron(out, m)
    return out


@pytest.mark.parametrize("dim", [2, 3])
def test_p1_closed_forms(oracle_mod, dim):
    K = 3
    P = oracle_mod.Patch([wl.open_uniform_knots(K, 1)] * dim, 1, 2)
    h = 1.0 / K
    M1 = h / 6 * np.array([[2.0, 1.0], [1.0, 2.0]])
    K1 = 1 / h * np.array([[1.0, -1.0], [-1.0, 1.0]])
    if dim == 2:
        Mref = np.kron(M1, M1)
        Kref = np.kron(M1, K1) + np.kron(K1, M1)
    else:
        Mref = _kron_all([M1, M1, M1])
        Kref = _kron_all([M1, M1, K1]) + _kron_all([M1, K1, M1]) + _kron_all([K1, M1, M1])
    for fn in (P.classical, P.sumfact):
        Km, Mm = fn()
        for e in range(P.E):
            np.testing.assert_allclose(Mm[e], Mref, rtol=0, atol=1e-15)
            np.testing.assert_allclose(Km[e], Kref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("dim,p,K", [(2, 2, 6), (2, 3, 5), (3, 2, 5), (3, 3, 4), (2, 5, 3), (3, 4, 2)])
def test_exact_rational_kronecker(oracle_mod, dim, p, K):
    """kappa = 1, identity geometry, q = p+1 (exact): the element matrices are
    Kronecker products of exactly integrated 1D element matrices."""
    t = wl.open_uniform_knots(K, p)
    tr = rational_open_uniform(K, p)
    P = oracle_mod.Patch([t] * dim, p, p + 1)
    spans = oracle_mod.spans(t, p)
    one_d = [element_matrices_1d(tr, p, int(s)) for s in spans]
    elems = np.arange(P.E)
    Kc, Mc = P.classical(elems)
    Ks, Ms = P.sumfact(elems)
    for e in range(P.E):
        ek = [e % K, (e // K) % K, e // (K * K)][:dim]
        Ms1 = [one_d[i][0] for i in ek]
        Ks1 = [one_d[i][1] for i in ek]
        # kron order: last direction outermost so that x is fastest
        Mref = _kron_all(Ms1[::-1])
        Kref = 0
        for d in range(dim):
            fac = [Ks1[j] if j == d else Ms1[j] for j in range(dim)]
            Kref = Kref + _kron_all(fac[::-1])
        scale_m, scale_k = np.abs(Mref).max(), np.abs(Kref).max()
        for Km, Mm in ((Kc, Mc), (Ks, Ms)):
            assert np.abs(Mm[e] - Mref).max() <= 1e-14 * scale_m
            assert np.abs(Km[e] - Kref).max() <= 1e-13 * scale_k


def test_interior_quadratic_closed_form(oracle_mod):
    K, p = 8, 2
    h = 1.0 / K
    M1 = h / 120 * np.array([[6, 13, 1], [13, 54, 13], [1, 13, 6]], dtype=float)
    K1 = 1 / (6 * h) * np.array([[2, -1, -1], [-1, 2, -1], [-1, -1, 2]], dtype=float)
    P = oracle_mod.Patch([wl.open_uniform_knots(K, p)] * 2, p, 3)
    for e1 in range(2, K - 2):
        for e2 in range(2, K - 2):
            e = e1 + K * e2
            Km, Mm = P.classical([e])
            np.testing.assert_allclose(Mm[0], np.kron(M1, M1), rtol=0, atol=1e-16)
            np.testing.assert_allclose(Km[0], np.kron(M1, K1) + np.kron(K1, M1), rtol=0, atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_affine_geometry_exact(oracle_mod, dim):
    """A constant, non-symmetric Jacobian G and constant kappa: the stiffness is
    sum_ij C_ij (tensor product of exact 1D integrals) with
    C = kappa |det G| G^{-1} G^{-T}; the mass is |det G| times the identity-case mass.
    Catches transposed or dropped geometry terms."""
    p, K = 2, 3
    t = wl.open_uniform_knots(K, p)
    tr = rational_open_uniform(K, p)
    rng = np.random.default_rng(17)
    G = np.eye(dim) + 0.3 * rng.standard_normal((dim, dim))
    kap = 1.7
    P = oracle_mod.Patch([t] * dim, p, p + 1)
    Garr = np.broadcast_to(G, (P.E, P.Q, dim, dim)).copy()
    kappa = np.full(P.E * P.Q, kap)
    Km, Mm = P.classical(kappa=kappa, G=Garr)
    Ks, Ms = P.sumfact(kappa=kappa, G=Garr)
    Gi = np.linalg.inv(G)
    C = kap * abs(np.linalg.det(G)) * Gi @ Gi.T
    spans = oracle_mod.spans(t, p)
    one_d = [element_matrices_1d(tr, p, int(s)) for s in spans]
    for e in range(P.E):
        ek = [e % K, (e // K) % K, e // (K * K)][:dim]
        Mref = abs(np.linalg.det(G)) * _kron_all([one_d[i][0] for i in ek][::-1])
        Kref = 0
        for i in range(dim):
            for j in range(dim):
                fac = []
                for k, ei in enumerate(ek):
                    M1, K1, X1 = one_d[ei]
                    if i == k and j == k:
                        fac.append(K1)
                    elif i == k:
                        fac.append(X1)        # int B'_a B_b
                    elif j == k:
                        fac.append(X1.T)      # int B_a B'_b
                    else:
                        fac.append(M1)
                Kref = Kref + C[i, j] * _kron_all(fac[::-1])
        for Kx, Mx in ((Km, Mm), (Ks, Ms)):
            assert np.abs(Mx[e] - Mref).max() <= 1e-14 * np.abs(Mref).max()
            assert np.abs(Kx[e] - Kref).max() <= 1e-13 * np.abs(Kref).max()


# --------------------------------------------------------------------------
# Invariants for any kappa and geometry
# --------------------------------------------------------------------------

def _curved_case(oracle_mod, p=2, K=3, q=None):
    q = q or p + 1
    knots = [wl.open_uniform_knots(K, p)] * 3
    P = oracle_mod.Patch(knots, p, q)
    G = wl.curved_map_jacobian(knots, q)
    kappa = wl.lognormal(P.E * P.Q, 99)
    rho = wl.lognormal(P.E * P.Q, 98)
    return P, G, kappa, rho


def test_invariants_curved(oracle_mod):
    P, G, kappa, rho = _curved_case(oracle_mod)
    Km, Mm = P.classical(kappa=kappa, G=G)
    _, Mr = P.classical(kappa=kappa, rho=rho, G=G, stiffness=False)
    one = np.ones(P.N)
    dets = np.abs(np.linalg.det(G.reshape(P.E, P.Q, 3, 3)))
    for e in range(P.E):
        # constants are in the kernel of the stiffness
        assert np.abs(Km[e] @ one).max() <= 1e-13 * np.linalg.norm(Km[e])
        # symmetric, mass positive definite
        assert np.abs(Km[e] - Km[e].T).max() <= 1e-15 * np.abs(Km[e]).max() * 10
        np.linalg.cholesky(Mm[e])
        # mass entries sum to the (quadrature) element volume: sum_q w_q |det G_q|
        ek = [e % 3, (e // 3) % 3, e // 9]
        wq = 1.0
        ws = []
        for k in range(3):
            s = int(oracle_mod.spans(P.knots[k], P.p)[ek[k]])
            _, w, _, _ = oracle_mod.basis_1d(P.knots[k], P.p, s, P.q)
            ws.append(w)
        W = np.einsum("k,j,i->kji", ws[2], ws[1], ws[0]).reshape(-1) * dets[e]
        assert Mm[e].sum() == pytest.approx(W.sum(), rel=1e-13)
        assert Mr[e].sum() == pytest.approx((W * rho[e * P.Q:(e + 1) * P.Q]).sum(), rel=1e-13)


def test_mass_sums_to_volume_identity(oracle_mod):
    for dim, p, K in [(2, 3, 5), (3, 2, 4)]:
        P = oracle_mod.Patch([wl.open_uniform_knots(K, p)] * dim, p, p + 1)
        _, Mm = P.classical(stiffness=False)
        np.testing.assert_allclose(Mm.sum(axis=(1, 2)), (1.0 / K) ** dim, rtol=1e-13)
        assert Mm.sum() == pytest.approx(1.0, rel=1e-13)


@pytest.mark.parametrize("dim,p,curved", [(2, 1, False), (2, 3, False), (3, 1, True), (3, 2, True), (3, 3, True), (3, 4, False)])
def test_classical_equals_sumfact(oracle_mod, dim, p, curved):
    """Algorithm 1 and Algorithm 2 reorder one finite sum (Sec. 3.2)."""
    K = 3
    knots = [wl.open_uniform_knots(K, p)] * dim
    P = oracle_mod.Patch(knots, p, p + 1)
    kappa = wl.lognormal(P.E * P.Q, 7)
    rho = wl.lognormal(P.E * P.Q, 8)
    if curved:
        G = wl.curved_map_jacobian(knots, p + 1)
    else:
        rng = np.random.default_rng(1)
        G = (np.eye(dim) + 0.2 * rng.standard_normal((P.E, P.Q, dim, dim)))
    el = np.arange(min(P.E, 9))
    Kc, Mc = P.classical(el, kappa=kappa, rho=rho, G=G)
    Ks, Ms = P.sumfact(el, kappa=kappa, rho=rho, G=G)
    for e in range(len(el)):
        assert np.linalg.norm(Kc[e] - Ks[e]) <= 1e-13 * np.linalg.norm(Kc[e])
        assert np.linalg.norm(Mc[e] - Ms[e]) <= 1e-13 * np.linalg.norm(Mc[e])


def test_over_integration_constant_kappa(oracle_mod):
    """q = p+1 is exact for constant kappa and affine geometry: q = p+4 agrees."""
    for dim, p in [(2, 2), (3, 2), (3, 3)]:
        knots = [wl.open_uniform_knots(2, p)] * dim
        a = oracle_mod.Patch(knots, p, p + 1)
        b = oracle_mod.Patch(knots, p, p + 4)
        Ka, Ma = a.classical(kappa=np.full(a.E * a.Q, 2.5))
        Kb, Mb = b.classical(kappa=np.full(b.E * b.Q, 2.5))
        assert np.abs(Ka - Kb).max() <= 1e-14 * np.abs(Ka).max() * 10
        assert np.abs(Ma - Mb).max() <= 1e-14 * np.abs(Ma).max() * 10


# --------------------------------------------------------------------------
# Dof map (support set of the Remark in Sec. 3.1)
# --------------------------------------------------------------------------

def test_dofmap_brute_force(oracle_mod):
    for dim, p, K in [(2, 2, 4), (3, 3, 3), (3, 1, 5)]:
        t = wl.open_uniform_knots(K, p)
        P = oracle_mod.Patch([t] * dim, p, p + 1)
        dof = P.dofmap()
        nf = K + p
        for e in range(P.E):
            ek = [e % K, (e // K) % K, e // (K * K)][:dim]
            # functions whose support meets the open element, brute force
            centre = [(ek[k] + 0.5) / K for k in range(dim)]
            supp = []
            for g in range(nf ** dim):
                gi = [g % nf, (g // nf) % nf, g // (nf * nf)][:dim]
                if all(oracle_mod.bspline(t, gi[k], p, centre[k]) > 0 for k in range(dim)):
                    supp.append(g)
            assert sorted(dof[e].tolist()) == supp
            # local index a = a1 + n a2 + n^2 a3 maps to consecutive global indices, x fastest
            assert dof[e][1] - dof[e][0] == 1


# --------------------------------------------------------------------------
# Adjoint: J(kappa) = u^T K(kappa) v and dJ/dkappa
# --------------------------------------------------------------------------

def _greville(t, p):
    return np.array([t[i + 1:i + p + 1].mean() for i in range(len(t) - p - 1)])


def test_adjoint_greville_identities(oracle_mod):
    p, K = 3, 3
    t = wl.open_uniform_knots(K, p)
    P = oracle_mod.Patch([t] * 3, p, p + 1)
    gr = _greville(t, p)
    nf = len(gr)
    idx = np.arange(P.n_dofs)
    ux = gr[idx % nf]
    uy = gr[(idx // nf) % nf]
    # u = v = x reproduces x exactly: J = int |grad x|^2 = 1 on the unit cube
    g, J = P.adjoint(ux, ux, kappa=np.ones(P.E * P.Q))
    assert J == pytest.approx(1.0, rel=1e-13)
    assert g.sum() == pytest.approx(1.0, rel=1e-13)
    # grad x . grad y = 0
    g, J = P.adjoint(ux, uy, kappa=np.ones(P.E * P.Q))
    assert abs(J) <= 1e-14
    assert np.abs(g).max() <= 1e-14


@pytest.mark.parametrize("dim", [2, 3])
def test_adjoint_affine_closed_form(oracle_mod, dim):
    """A constant non-symmetric Jacobian G (an affine map of the unit square
    or cube): the Greville interpolants of xi_i reproduce xi_i, whose
    physical gradients are the columns of G^{-T}, so J(u = xi_i, v = xi_j)
    with kappa = 1 equals (G^{-T} e_i).(G^{-T} e_j) |det G| exactly."""
    p = 2
    knots = [wl.open_uniform_knots(K, p) for K in (3, 4, 2)[:dim]]
    P = oracle_mod.Patch(knots, p, p + 1)
    Gc = np.array([[1.2, 0.3, -0.2], [-0.1, 0.9, 0.25], [0.15, -0.05, 1.1]])[:dim, :dim]
    G = np.broadcast_to(Gc, (P.E * P.Q, dim, dim)).copy()
    GinvT = np.linalg.inv(Gc).T
    det = abs(np.linalg.det(Gc))
    nf = [len(t) - p - 1 for t in knots]
    idx = np.arange(P.n_dofs)
    comp = [idx % nf[0], (idx // nf[0]) % nf[1]] + ([idx // (nf[0] * nf[1])] if dim == 3 else [])
    xi = [_greville(knots[k], p)[comp[k]] for k in range(dim)]
    ones = np.ones(P.E * P.Q)
    for i in range(dim):
        for j in range(dim):
            g, J = P.adjoint(xi[i], xi[j], kappa=ones, G=G)
            ref = float(GinvT[:, i] @ GinvT[:, j]) * det
            assert J == pytest.approx(ref, rel=1e-12, abs=1e-14), (i, j)
            assert g.sum() == pytest.approx(ref, rel=1e-12, abs=1e-14)


@pytest.mark.parametrize("curved", [False, True])
def test_adjoint_vs_matrices_and_fd(oracle_mod, curved):
    p, K = 2, 3
    knots = [wl.open_uniform_knots(K, p)] * 3
    P = oracle_mod.Patch(knots, p, p + 1)
    G = wl.curved_map_jacobian(knots, p + 1) if curved else None
    kappa = wl.lognormal(P.E * P.Q, 21)
    u = wl.normal(P.n_dofs, 22)
    v = wl.normal(P.n_dofs, 23)
    g, J = P.adjoint(u, v, kappa=kappa, G=G)
    dof = P.dofmap()

    def J_direct(kap):
        Km, _ = P.classical(kappa=kap, G=G, mass=False)
        return sum(u[dof[e]] @ Km[e] @ v[dof[e]] for e in range(P.E))

    Jd = J_direct(kappa)
    assert J == pytest.approx(Jd, rel=1e-12)
    rng = np.random.default_rng(24)
    for k in rng.choice(P.E * P.Q, size=6, replace=False):
        h = 1e-6 * kappa[k]
        kp = kappa.copy(); kp[k] += h
        km = kappa.copy(); km[k] -= h
        fd = (J_direct(kp) - J_direct(km)) / (2 * h)
        gk = g.reshape(-1)[k]
        scale = np.abs(kappa * g.reshape(-1)).sum() / (h)
        assert abs(fd - gk) <= 1e-6 * abs(gk) + 1e-12 * scale
