"""Pins of the oracle's weighted quadrature for the mass matrix (the variant
named in Sec. 1.2 of the paper; the rule is defined in oracle/iga_oracle.h).

The defining property of the rule of test function B_i is exactness against
the spline space: sum_q w_{i,q} B_j(x_q) = int B_i B_j for every j.  The pins
check it against exact rational integrals and scipy's B-spline evaluation,
the least-norm choice against the row space of the collocation matrix, and
the assembled matrices against exact Kronecker products (constant
coefficient, where weighted quadrature is exact) and against Gauss
quadrature for a smooth coefficient (consistency under refinement).  CPU only.
"""
import numpy as np
import pytest

from exact1d import element_matrices_1d, rational_open_uniform
from paper_2207_00280_gb300 import workloads as wl


def _bspline_values(t, p, x):
    """B_j(x_q) for all j, by scipy (right end of the domain included)."""
    from scipy.interpolate import BSpline
    nf = len(t) - p - 1
    V = np.zeros((nf, len(x)))
    for j in range(nf):
        c = np.zeros(nf)
        c[j] = 1.0
        V[j] = BSpline(t, c, p, extrapolate=False)(x)
    return np.nan_to_num(V)


def _exact_gram_1d(t, tr, p):
    nf = len(t) - p - 1
    G = np.zeros((nf, nf))
    for s in range(p, len(t) - p - 1):
        if t[s] < t[s + 1]:
            G[s - p:s + 1, s - p:s + 1] += element_matrices_1d(tr, p, s)[0]
    return G


@pytest.mark.parametrize("p,K", [(1, 3), (2, 2), (2, 5), (3, 3), (3, 8), (4, 4), (5, 2), (5, 11)])
def test_weights_exact_against_rational_integrals(oracle_mod, p, K):
    t = wl.open_uniform_knots(K, p)
    tr = rational_open_uniform(K, p)
    x = oracle_mod.wq_points(t, p)
    W = oracle_mod.wq_weights(t, p, x)
    V = _bspline_values(t, p, x)
    G = _exact_gram_1d(t, tr, p)
    assert np.abs(W @ V.T - G).max() <= 1e-13 * np.abs(G).max()
    # zero outside the closed support of each test function
    for i in range(W.shape[0]):
        outside = (x < t[i]) | (x > t[i + p + 1])
        assert np.all(W[i, outside] == 0.0)


@pytest.mark.parametrize("p,K", [(2, 6), (3, 7), (4, 9)])
def test_point_set(oracle_mod, p, K):
    """Left end and midpoint per element; p + 1 points in the p boundary
    elements at each end; the right end of the domain last."""
    t = wl.open_uniform_knots(K, p)
    x = oracle_mod.wq_points(t, p)
    h = 1.0 / K
    ref = []
    for e in range(K):
        a = e * h
        ref.append(a)
        if e < p or e >= K - p:
            ref += [a + h * r / (p + 1) for r in range(1, p + 1)]
        else:
            ref.append(a + h / 2)
    ref.append(1.0)
    np.testing.assert_allclose(x, ref, rtol=0, atol=1e-15)
    assert np.all(np.diff(x) > 0)


@pytest.mark.parametrize("p,K", [(2, 5), (3, 6), (5, 12)])
def test_weights_least_norm(oracle_mod, p, K):
    """Among exact rules the least-norm one lies in the row space of the
    collocation matrix A[j][q] = B_j(x_q) (j overlapping i, q in the support)."""
    t = wl.open_uniform_knots(K, p)
    x = oracle_mod.wq_points(t, p)
    W = oracle_mod.wq_weights(t, p, x)
    V = _bspline_values(t, p, x)
    for i in range(W.shape[0]):
        q = np.where((x >= t[i]) & (x <= t[i + p + 1]))[0]
        js = [j for j in range(W.shape[0])
              if min(t[i + p + 1], t[j + p + 1]) > max(t[i], t[j])]
        A = V[np.ix_(js, q)]
        y, *_ = np.linalg.lstsq(A.T, W[i, q], rcond=None)
        assert np.abs(A.T @ y - W[i, q]).max() <= 1e-12 * np.abs(W[i, q]).max()


def _kron_all(mats):
    out = mats[0]
    for m in mats[1:]:
        out = np.kron(out, m)
    return out


def _dense(row_ptr, col_idx, vals, n):
    A = np.zeros((n, n))
    for i in range(n):
        A[i, col_idx[row_ptr[i]:row_ptr[i + 1]]] = vals[row_ptr[i]:row_ptr[i + 1]]
    return A


@pytest.mark.parametrize("dim,p,K", [(2, 2, 5), (3, 1, 4), (3, 2, 3), (3, 3, 3), (3, 4, 2)])
def test_constant_coefficient_is_exact(oracle_mod, dim, p, K):
    """c = 1: the weighted-quadrature mass is the exact Gram matrix, the
    Kronecker product of exact rational 1D Gram matrices (x fastest), and it
    equals the assembled Gauss-quadrature mass (q = p + 1, also exact)."""
    t = wl.open_uniform_knots(K, p)
    tr = rational_open_uniform(K, p)
    P = oracle_mod.Patch([t] * dim, p, p + 1)
    rp, ci = P.csr_pattern()
    vals = P.wq_mass(rp, ci)
    Mw = _dense(rp, ci, vals, P.n_dofs)
    G = _exact_gram_1d(t, tr, p)
    ref = _kron_all([G] * dim)
    assert np.abs(Mw - ref).max() <= 1e-13 * np.abs(ref).max()
    _, Me = P.classical(stiffness=False)
    gauss = P.assemble(Me, rp, ci)
    assert np.abs(vals - gauss).max() <= 1e-13 * np.abs(gauss).max()


def test_smooth_coefficient_consistency(oracle_mod):
    """c(x, y, z) = 1 + x/2 + y^2 + z/4: weighted quadrature approaches the
    Gauss-quadrature mass as the mesh is refined.  The rule is exact on the
    spline space only and c B_j is not a spline, so entry-wise the difference
    falls at first order in h (a sanity check, not an exactness pin)."""
    p = 2
    errs = []
    for K in (3, 6):
        t = wl.open_uniform_knots(K, p)
        P = oracle_mod.Patch([t] * 3, p, p + 1)
        xw = oracle_mod.wq_points(t, p)
        X, Y, Z = np.meshgrid(xw, xw, xw, indexing="ij")
        cw = (1 + X / 2 + Y ** 2 + Z / 4).transpose(2, 1, 0).reshape(-1)   # x fastest
        rp, ci = P.csr_pattern()
        vw = P.wq_mass(rp, ci, c=cw)
        qp = wl.qp_coordinates(P.knots, p + 1)
        rho = 1 + qp[..., 0] / 2 + qp[..., 1] ** 2 + qp[..., 2] / 4
        _, Me = P.classical(rho=rho.reshape(-1), stiffness=False)
        vg = P.assemble(Me, rp, ci)
        errs.append(np.abs(vw - vg).max() / np.abs(vg).max())
    assert errs[1] < 1e-2
    assert errs[1] < errs[0] / 2, errs


def test_rows_see_the_coefficient_on_their_own_support(oracle_mod):
    """Row i uses the rule of its test function, whose weights vanish outside
    the closed support of B_i: with c = 0 at every point of y <= 0.5 and 1
    above, the rows whose y-support ends at or below 0.5 are exactly zero, and
    rows reaching above are not (a rule taken from the trial side instead
    would make them non-zero and vice versa)."""
    p, K = 2, 6
    t = wl.open_uniform_knots(K, p)
    P = oracle_mod.Patch([t] * 3, p, p + 1)
    xw = oracle_mod.wq_points(t, p)
    n = len(xw)
    cy = (xw > 0.5).astype(float)
    c = np.broadcast_to(cy[None, :, None], (n, n, n)).reshape(-1)   # [q3][q2][q1], x fastest
    rp, ci = P.csr_pattern()
    vals = P.wq_mass(rp, ci, c=np.ascontiguousarray(c))
    nf = P.n_fun[0]
    for i in range(P.n_dofs):
        i2 = (i // nf) % nf
        row = vals[rp[i]:rp[i + 1]]
        if t[i2 + p + 1] <= 0.5:
            assert np.all(row == 0.0), i
        elif t[i2] >= 0.5:
            assert np.abs(row).max() > 0.0, i


def test_point_coefficient_gives_trial_values_in_every_row(oracle_mod):
    """c = 1 at one interior grid point x* and 0 elsewhere: every term of
    row i is w_i(x*) c(x*) B_j(x*), so each row is proportional to the trial
    functions evaluated at x* (scipy), whatever the weights are."""
    p, K = 2, 5
    t = wl.open_uniform_knots(K, p)
    P = oracle_mod.Patch([t] * 3, p, p + 1)
    xw = oracle_mod.wq_points(t, p)
    n = len(xw)
    qs = (n // 2, n // 3, (2 * n) // 3)            # the point (x, y, z) indices
    c = np.zeros((n, n, n))
    c[qs[2], qs[1], qs[0]] = 1.0                    # [q3][q2][q1]
    rp, ci = P.csr_pattern()
    vals = P.wq_mass(rp, ci, c=c.reshape(-1))
    V = _bspline_values(t, p, xw)                   # [j][q]
    nf = P.n_fun[0]
    nonzero = 0
    for i in range(P.n_dofs):
        row = vals[rp[i]:rp[i + 1]]
        if not np.any(row):
            continue
        nonzero += 1
        cols = ci[rp[i]:rp[i + 1]]
        v = V[cols % nf, qs[0]] * V[(cols // nf) % nf, qs[1]] * V[cols // (nf * nf), qs[2]]
        lam = np.dot(row, v) / np.dot(v, v)
        assert np.abs(row - lam * v).max() <= 1e-13 * np.abs(row).max(), i
    assert nonzero > 0


# --------------------------------------------------------------------------
# The derivative rule and the weighted-quadrature stiffness
# --------------------------------------------------------------------------

def _exact_stiff_1d(t, tr, p):
    nf = len(t) - p - 1
    S = np.zeros((nf, nf))
    for s in range(p, len(t) - p - 1):
        if t[s] < t[s + 1]:
            S[s - p:s + 1, s - p:s + 1] += element_matrices_1d(tr, p, s)[1]
    return S


def _bspline_derivs(t, p, x):
    """B'_j(x_q) for all j, by scipy (the right end of the domain as the left limit)."""
    from scipy.interpolate import BSpline
    nf = len(t) - p - 1
    V = np.zeros((nf, len(x)))
    for j in range(nf):
        c = np.zeros(nf)
        c[j] = 1.0
        V[j] = BSpline(t, c, p, extrapolate=False)(x, nu=1)
    return np.nan_to_num(V)


@pytest.mark.parametrize("p,K", [(2, 2), (2, 5), (3, 3), (3, 8), (4, 4), (5, 2), (5, 11)])
def test_deriv_weights_exact_against_rational_integrals(oracle_mod, p, K):
    """sum_q w'_{i,q} B'_j(x_q) = int B'_i B'_j for every pair, against exact
    rational integrals and scipy's derivatives; zero outside the support."""
    t = wl.open_uniform_knots(K, p)
    tr = rational_open_uniform(K, p)
    x = oracle_mod.wq_points(t, p)
    W = oracle_mod.wq_weights(t, p, x, deriv=True)
    D = _bspline_derivs(t, p, x)
    S = _exact_stiff_1d(t, tr, p)
    assert np.abs(W @ D.T - S).max() <= 1e-12 * np.abs(S).max()
    for i in range(W.shape[0]):
        outside = (x < t[i]) | (x > t[i + p + 1])
        assert np.all(W[i, outside] == 0.0)


def test_deriv_weights_nonuniform_knots(oracle_mod):
    """Exactness on a non-uniform knot vector with a repeated interior knot,
    against Gauss integration of scipy's derivatives (p + 1 points per span)."""
    from scipy.interpolate import BSpline
    p = 3
    t = np.array([0, 0, 0, 0, 0.15, 0.4, 0.4, 0.55, 0.8, 1, 1, 1, 1.0])
    x = oracle_mod.wq_points(t, p)
    W = oracle_mod.wq_weights(t, p, x, deriv=True)
    D = _bspline_derivs(t, p, x)
    nf = len(t) - p - 1
    gx, gw = np.polynomial.legendre.leggauss(p + 1)
    S = np.zeros((nf, nf))
    for s in range(p, len(t) - p - 1):
        a, b = t[s], t[s + 1]
        if b <= a:
            continue
        xs = 0.5 * (a + b) + 0.5 * (b - a) * gx
        Dq = np.array([BSpline(t, np.eye(nf)[j], p)(xs, nu=1) for j in range(nf)])
        S += (Dq * (0.5 * (b - a) * gw)) @ Dq.T
    assert np.abs(W @ D.T - S).max() <= 1e-12 * np.abs(S).max()


@pytest.mark.parametrize("p,K", [(2, 5), (3, 6), (5, 12)])
def test_deriv_weights_least_norm(oracle_mod, p, K):
    """The derivative rule lies in the row space of its collocation matrix
    A[j][q] = B'_j(x_q) (the least-norm member of the exact rules)."""
    t = wl.open_uniform_knots(K, p)
    x = oracle_mod.wq_points(t, p)
    W = oracle_mod.wq_weights(t, p, x, deriv=True)
    D = _bspline_derivs(t, p, x)
    for i in range(W.shape[0]):
        q = np.where((x >= t[i]) & (x <= t[i + p + 1]))[0]
        js = [j for j in range(W.shape[0])
              if min(t[i + p + 1], t[j + p + 1]) > max(t[i], t[j])]
        A = D[np.ix_(js, q)]
        y, *_ = np.linalg.lstsq(A.T, W[i, q], rcond=None)
        assert np.abs(A.T @ y - W[i, q]).max() <= 1e-12 * np.abs(W[i, q]).max()


def test_deriv_rule_needs_p2(oracle_mod):
    t = wl.open_uniform_knots(4, 1)
    x = oracle_mod.wq_points(t, 1)
    with pytest.raises(ValueError):
        oracle_mod.wq_weights(t, 1, x, deriv=True)


def _kron3(a3, a2, a1):
    return np.kron(a3, np.kron(a2, a1))   # x fastest


@pytest.mark.parametrize("p,Ks", [(2, (4, 2, 3)), (3, (3, 2, 4)), (4, (2, 3, 2))])
def test_stiffness_constant_coefficient_is_exact(oracle_mod, p, Ks):
    """c = 1: the weighted-quadrature stiffness is the exact Kronecker sum
    S1 x G2 x G3 + G1 x S2 x G3 + G1 x G2 x S3 of exact rational 1D stiffness
    and Gram matrices (different sizes per direction), and equals the
    assembled Gauss-quadrature stiffness with kappa = 1."""
    ts = [wl.open_uniform_knots(K, p) for K in Ks]
    trs = [rational_open_uniform(K, p) for K in Ks]
    P = oracle_mod.Patch(ts, p, p + 1)
    rp, ci = P.csr_pattern()
    vals = P.wq_stiffness(rp, ci)
    A = _dense(rp, ci, vals, P.n_dofs)
    G = [_exact_gram_1d(t, tr, p) for t, tr in zip(ts, trs)]
    S = [_exact_stiff_1d(t, tr, p) for t, tr in zip(ts, trs)]
    ref = _kron3(G[2], G[1], S[0]) + _kron3(G[2], S[1], G[0]) + _kron3(S[2], G[1], G[0])
    assert np.abs(A - ref).max() <= 1e-13 * np.abs(ref).max()
    Ke, _ = P.classical(mass=False)
    gauss = P.assemble(Ke, rp, ci)
    assert np.abs(vals - gauss).max() <= 1e-13 * np.abs(gauss).max()


def test_stiffness_2d_constant_coefficient(oracle_mod):
    p, Ks = 3, (5, 3)
    ts = [wl.open_uniform_knots(K, p) for K in Ks]
    trs = [rational_open_uniform(K, p) for K in Ks]
    P = oracle_mod.Patch(ts, p, p + 1)
    rp, ci = P.csr_pattern()
    A = _dense(rp, ci, P.wq_stiffness(rp, ci), P.n_dofs)
    G = [_exact_gram_1d(t, tr, p) for t, tr in zip(ts, trs)]
    S = [_exact_stiff_1d(t, tr, p) for t, tr in zip(ts, trs)]
    ref = np.kron(G[1], S[0]) + np.kron(S[1], G[0])
    assert np.abs(A - ref).max() <= 1e-13 * np.abs(ref).max()


def test_stiffness_rows_sum_to_zero(oracle_mod):
    """Any coefficient: sum_j K_ij = 0, since the trial gradients sum to zero
    at every point (sum_j B_j = 1 in every direction)."""
    p = 3
    ts = [wl.open_uniform_knots(4, p), _nonuniform(p), wl.open_uniform_knots(3, p)]
    P = oracle_mod.Patch(ts, p, p + 1)
    n = int(np.prod([len(oracle_mod.wq_points(t, p)) for t in ts]))
    c = wl.lognormal(n, 93)
    rp, ci = P.csr_pattern()
    vals = P.wq_stiffness(rp, ci, c=c)
    rows = np.add.reduceat(vals, rp[:-1])
    assert np.abs(rows).max() <= 1e-13 * np.abs(vals).max()


def _nonuniform(p):
    return np.concatenate([[0.0] * (p + 1), [0.2, 0.35, 0.35, 0.7], [1.0] * (p + 1)])


def test_stiffness_point_coefficient_spans_trial_gradients(oracle_mod):
    """c = 1 at one grid point x* and 0 elsewhere: row i is
    sum_k w^k_i(x*) T^k_j(x*) with T^k_j = prod_l B^(l == k)_{j_l}(x*_l), so
    every row lies in the span of the three trial vectors T^1, T^2, T^3 at x*
    (a rule taken from the trial side would not)."""
    p, K = 2, 5
    t = wl.open_uniform_knots(K, p)
    P = oracle_mod.Patch([t] * 3, p, p + 1)
    xw = oracle_mod.wq_points(t, p)
    n = len(xw)
    qs = (n // 2, n // 3, (2 * n) // 3)
    c = np.zeros((n, n, n))
    c[qs[2], qs[1], qs[0]] = 1.0
    rp, ci = P.csr_pattern()
    vals = P.wq_stiffness(rp, ci, c=c.reshape(-1))
    V = _bspline_values(t, p, xw)
    D = _bspline_derivs(t, p, xw)
    nf = P.n_fun[0]
    checked = 0
    for i in range(P.n_dofs):
        row = vals[rp[i]:rp[i + 1]]
        if not np.any(row):
            continue
        cols = ci[rp[i]:rp[i + 1]]
        j1, j2, j3 = cols % nf, (cols // nf) % nf, cols // (nf * nf)
        T = np.stack([D[j1, qs[0]] * V[j2, qs[1]] * V[j3, qs[2]],
                      V[j1, qs[0]] * D[j2, qs[1]] * V[j3, qs[2]],
                      V[j1, qs[0]] * V[j2, qs[1]] * D[j3, qs[2]]], axis=1)
        lam, *_ = np.linalg.lstsq(T, row, rcond=None)
        assert np.abs(T @ lam - row).max() <= 1e-12 * np.abs(row).max(), i
        checked += 1
    assert checked > 0


def test_stiffness_smooth_coefficient_consistency(oracle_mod):
    """c(x, y, z) = 1 + x/2 + y^2 + z/4: weighted quadrature approaches the
    Gauss-quadrature stiffness as the mesh is refined (first order, a sanity
    check like the mass's)."""
    p = 2
    errs = []
    for K in (3, 6):
        t = wl.open_uniform_knots(K, p)
        P = oracle_mod.Patch([t] * 3, p, p + 1)
        xw = oracle_mod.wq_points(t, p)
        X, Y, Z = np.meshgrid(xw, xw, xw, indexing="ij")
        cw = (1 + X / 2 + Y ** 2 + Z / 4).transpose(2, 1, 0).reshape(-1)
        rp, ci = P.csr_pattern()
        vw = P.wq_stiffness(rp, ci, c=cw)
        qp = wl.qp_coordinates(P.knots, p + 1)
        kap = 1 + qp[..., 0] / 2 + qp[..., 1] ** 2 + qp[..., 2] / 4
        Ke, _ = P.classical(kappa=kap.reshape(-1), mass=False)
        vg = P.assemble(Ke, rp, ci)
        errs.append(np.abs(vw - vg).max() / np.abs(vg).max())
    assert errs[1] < 5e-2
    assert errs[1] < errs[0] / 1.5, errs
