"""Pins of the oracle for patches with a degree and a number of Gauss points per
direction, and for degrees 6 to 8.

The paper takes one degree in every direction and states that the method
extends to bases of different degrees (Sec. 2.3); its element sum (eq. 10) has
P_1 P_2 P_3 quadrature points, one count per direction, and its experiments
run degrees up to 9 (Sec. 4).  Every expected value here comes from exact
rational 1D integrals (tests/exact1d.py), closed forms or brute force, not
from the oracle itself.  Mixing up two directions' degrees or point counts in
any index of the oracle breaks the Kronecker structure these pins check.
"""
from fractions import Fraction

import numpy as np
import pytest

from exact1d import element_matrices_1d
from paper_2207_00280_gb300 import workloads as wl


def _kron_all(mats):
    out = mats[0]
    for m in mats[1:]:
        out = np.kron(out, m)
    return out


def _rational_knots(K, p, breaks=None):
    """Open knot vector with rational interior breaks (uniform if None)."""
    inner = breaks if breaks is not None else [Fraction(i, K) for i in range(1, K)]
    return [Fraction(0)] * (p + 1) + list(inner) + [Fraction(1)] * (p + 1)


def _elem_index(e, Ks):
    out, r = [], e
    for K in Ks:
        out.append(r % K)
        r //= K
    return out


def _one_d(tr, p):
    t = np.array([float(x) for x in tr])
    spans = [s for s in range(p, len(t) - p - 1) if t[s] < t[s + 1]]
    return t, [element_matrices_1d(tr, p, s) for s in spans]


CASES = [
    # dim, degrees, Gauss points, elements (breaks: non-uniform interior knots)
    (3, (1, 3, 2), (2, 4, 3), (3, 2, 4), None),
    (3, (2, 1, 4), (4, 2, 6), (2, 3, 2), [(Fraction(1, 3),), (Fraction(1, 5), Fraction(1, 2)),
                                         (Fraction(2, 7),)]),
    (2, (3, 1), (4, 3), (3, 4), None),
    (2, (1, 4), (2, 7), (4, 2), [(Fraction(1, 7), Fraction(3, 7), Fraction(5, 6)), (Fraction(3, 5),)]),
    (3, (6, 2, 1), (7, 3, 2), (2, 2, 3), None),
    (3, (7, 6, 8), (8, 7, 9), (1, 1, 1), None),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_aniso_exact_kronecker(oracle_mod, case):
    """kappa = 1, identity geometry, q_k >= p_k + 1 (exact in every direction):
    M = Mz (x) My (x) Mx and K = Mz (x) My (x) Kx + Mz (x) Ky (x) Mx + Kz (x) My (x) Mx
    with each direction's own exactly integrated 1D element matrices."""
    dim, ps, qs, Ks, breaks = CASES[case]
    trs = [_rational_knots(Ks[k], ps[k], breaks[k] if breaks else None) for k in range(dim)]
    one = [_one_d(trs[k], ps[k]) for k in range(dim)]
    knots = [o[0] for o in one]
    P = oracle_mod.Patch(knots, ps, qs)
    assert P.N == int(np.prod([p + 1 for p in ps])) and P.Q == int(np.prod(qs))
    assert P.n_el == list(Ks)
    big = P.N > 200
    methods = [P.sumfact] if big else [P.classical, P.sumfact]
    elems = np.arange(P.E)
    res = [fn(elems) for fn in methods]
    for e in range(P.E):
        ek = _elem_index(e, Ks)
        Ms1 = [one[k][1][ek[k]][0] for k in range(dim)]
        Ks1 = [one[k][1][ek[k]][1] for k in range(dim)]
        Mref = _kron_all(Ms1[::-1])
        Kref = 0
        for d in range(dim):
            fac = [Ks1[j] if j == d else Ms1[j] for j in range(dim)]
            Kref = Kref + _kron_all(fac[::-1])
        # rounding of the FP64 tables grows with the degree (the 1D degree-8
        # Gauss mass alone is off by ~1.3e-14 relative to its largest entry)
        tol_m = 1e-14 if max(ps) <= 4 else 1e-13
        for Km, Mm in res:
            assert np.abs(Mm[e] - Mref).max() <= tol_m * np.abs(Mref).max()
            assert np.abs(Km[e] - Kref).max() <= 1e-12 * np.abs(Kref).max()


def test_degree_8_classical_one_element(oracle_mod):
    """Algorithm 1 at degree 8 (N = 729, Q = 729) on one element of a curved
    patch equals Algorithm 2 (the latter is pinned to exact values above)."""
    p, q = 8, 9
    knots = [wl.open_uniform_knots(1, p)] * 3
    P = oracle_mod.Patch(knots, p, q)
    G = wl.curved_map_jacobian(knots, q)
    kappa = wl.lognormal(P.E * P.Q, 81)
    Kc, Mc = P.classical(kappa=kappa, G=G)
    Ks, Ms = P.sumfact(kappa=kappa, G=G)
    assert np.abs(Kc - Ks).max() <= 1e-13 * np.abs(Ks).max()
    assert np.abs(Mc - Ms).max() <= 1e-13 * np.abs(Ms).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_aniso_affine_geometry_exact(oracle_mod, dim):
    """A constant non-symmetric Jacobian with a different degree and Gauss order
    per direction: K = sum_ij C_ij (tensor product of exact 1D integrals, the
    derivative factor in directions i (test) and j (trial)),
    C = kappa |det G| G^{-1} G^{-T}."""
    ps, qs, Ks = (2, 3, 1)[:dim], (3, 5, 2)[:dim], (2, 3, 2)[:dim]
    trs = [_rational_knots(Ks[k], ps[k]) for k in range(dim)]
    one = [_one_d(trs[k], ps[k]) for k in range(dim)]
    knots = [o[0] for o in one]
    P = oracle_mod.Patch(knots, ps, qs)
    rng = np.random.default_rng(31)
    G = np.eye(dim) + 0.3 * rng.standard_normal((dim, dim))
    kap = 1.3
    Garr = np.broadcast_to(G, (P.E, P.Q, dim, dim)).copy()
    kappa = np.full(P.E * P.Q, kap)
    Gi = np.linalg.inv(G)
    C = kap * abs(np.linalg.det(G)) * Gi @ Gi.T
    for fn in (P.classical, P.sumfact):
        Km, Mm = fn(kappa=kappa, G=Garr)
        for e in range(P.E):
            ek = _elem_index(e, Ks)
            mats = [one[k][1][ek[k]] for k in range(dim)]
            Mref = abs(np.linalg.det(G)) * _kron_all([m[0] for m in mats][::-1])
            Kref = 0
            for i in range(dim):
                for j in range(dim):
                    fac = []
                    for k in range(dim):
                        M1, K1, X1 = mats[k]
                        if i == k and j == k:
                            fac.append(K1)
                        elif i == k:
                            fac.append(X1)
                        elif j == k:
                            fac.append(X1.T)
                        else:
                            fac.append(M1)
                    Kref = Kref + C[i, j] * _kron_all(fac[::-1])
            assert np.abs(Mm[e] - Mref).max() <= 1e-14 * np.abs(Mref).max()
            assert np.abs(Km[e] - Kref).max() <= 1e-13 * np.abs(Kref).max()


def test_aniso_classical_equals_sumfact_curved(oracle_mod):
    ps, qs, Ks = (2, 3, 1), (3, 5, 2), (2, 2, 3)
    knots = [wl.open_uniform_knots(K, p) for K, p in zip(Ks, ps)]
    P = oracle_mod.Patch(knots, ps, qs)
    G = wl.curved_map_jacobian(knots, qs)
    kappa = wl.lognormal(P.E * P.Q, 41)
    rho = wl.lognormal(P.E * P.Q, 42)
    Kc, Mc = P.classical(kappa=kappa, rho=rho, G=G)
    Ks_, Ms = P.sumfact(kappa=kappa, rho=rho, G=G)
    assert np.abs(Kc - Ks_).max() <= 1e-13 * np.abs(Kc).max()
    assert np.abs(Mc - Ms).max() <= 1e-13 * np.abs(Mc).max()
    # K 1 = 0 and sum M = sum_q w_q |det G| rho_q (quadrature volume) per element
    for e in range(P.E):
        assert np.abs(Kc[e].sum(axis=1)).max() <= 1e-13 * np.linalg.norm(Kc[e])
    dets = np.abs(np.linalg.det(G.reshape(P.E, P.Q, 3, 3)))
    w = []
    for k, (t, p, q) in enumerate(zip(knots, ps, qs)):
        xr, wr = np.polynomial.legendre.leggauss(q)
        b = np.unique(t)
        w.append(0.5 * (b[1:] - b[:-1])[:, None] * wr[None, :])
    for e in range(P.E):
        e1, e2, e3 = _elem_index(e, Ks)
        W = np.einsum("c,b,a->cba", w[2][e3], w[1][e2], w[0][e1]).reshape(-1)
        vol = float((W * dets[e] * rho.reshape(P.E, P.Q)[e]).sum())
        assert Mc[e].sum() == pytest.approx(vol, rel=1e-13)


def test_aniso_dofmap_brute_force(oracle_mod):
    ps, Ks = (1, 3, 2), (3, 2, 2)
    knots = [wl.open_uniform_knots(K, p) for K, p in zip(Ks, ps)]
    P = oracle_mod.Patch(knots, ps, (2, 4, 3))
    nf = [K + p for K, p in zip(Ks, ps)]
    assert P.n_fun == nf
    dof = P.dofmap()
    for e in range(P.E):
        ek = _elem_index(e, Ks)
        centre = [(ek[k] + 0.5) / Ks[k] for k in range(3)]
        supp = []
        for g in range(int(np.prod(nf))):
            gi = [g % nf[0], (g // nf[0]) % nf[1], g // (nf[0] * nf[1])]
            if all(oracle_mod.bspline(knots[k], gi[k], ps[k], centre[k]) > 0 for k in range(3)):
                supp.append(g)
        assert sorted(dof[e].tolist()) == supp
        # local a = a1 + n1 (a2 + n2 a3) maps x fastest
        n1, n2 = ps[0] + 1, ps[1] + 1
        assert dof[e][1] - dof[e][0] == 1
        assert dof[e][n1] - dof[e][0] == nf[0]
        assert dof[e][n1 * n2] - dof[e][0] == nf[0] * nf[1]


def _greville(t, p):
    return np.array([t[i + 1:i + p + 1].mean() for i in range(len(t) - p - 1)])


@pytest.mark.parametrize("ps,qs", [((3, 1, 2), (4, 2, 3)), ((6, 2, 8), (7, 4, 9))])
def test_aniso_adjoint_greville(oracle_mod, ps, qs):
    """The Greville interpolant of x_k reproduces x_k in its own direction's
    degree: with u = v = x_k, J = int |grad x_k|^2 = 1; with u = x, v = y, J = 0."""
    Ks = (2, 3, 1)
    knots = [wl.open_uniform_knots(K, p) for K, p in zip(Ks, ps)]
    P = oracle_mod.Patch(knots, ps, qs)
    nf = P.n_fun
    idx = np.arange(P.n_dofs)
    comp = [idx % nf[0], (idx // nf[0]) % nf[1], idx // (nf[0] * nf[1])]
    x = [_greville(knots[k], ps[k])[comp[k]] for k in range(3)]
    ones = np.ones(P.E * P.Q)
    for k in range(3):
        g, J = P.adjoint(x[k], x[k], kappa=ones)
        assert J == pytest.approx(1.0, rel=1e-12)
    g, J = P.adjoint(x[0], x[1], kappa=ones)
    assert abs(J) <= 1e-13
