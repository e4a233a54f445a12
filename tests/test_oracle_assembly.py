"""Pins of the oracle's global assembly and operator application.

The global matrix sums the element matrices over the support index sets of
the elements (Sec. 3.1, eq. 10 and the Remark on K^Delta_alpha; the insertion
step of Table 3).  Each test checks the oracle against something other than
itself: supports of the 1D B-splines written out from the knots, the closed
form of the integral of a B-spline, exact rational 1D integrals assembled in
1D and combined by Kronecker products, the boundary flux of a linear field,
and a second oracle path (the quadrature-point interpolation of the adjoint).
CPU only.
"""
import numpy as np
import pytest

from exact1d import element_matrices_1d, rational_open_uniform
from paper_2207_00280_gb300 import workloads as wl


def _nonuniform_knots(p, seed):
    """Open knots with uneven interior breaks and one knot of multiplicity 2."""
    rng = np.random.default_rng(seed)
    inner = np.sort(rng.uniform(0.08, 0.92, size=4))
    if p >= 2:
        inner = np.sort(np.concatenate([inner, inner[1:2]]))
    return np.concatenate([[0.0] * (p + 1), inner, [1.0] * (p + 1)])


def _cases():
    return [
        (2, 2, [wl.open_uniform_knots(5, 2)] * 2),
        (2, 3, [wl.open_uniform_knots(4, 3), _nonuniform_knots(3, 1)]),
        (3, 1, [wl.open_uniform_knots(3, 1)] * 3),
        (3, 2, [wl.open_uniform_knots(3, 2), _nonuniform_knots(2, 2), wl.open_uniform_knots(2, 2)]),
        (3, 3, [wl.open_uniform_knots(3, 3)] * 3),
    ]


def _multi(i, nf):
    out = []
    for n in nf:
        out.append(i % n)
        i //= n
    return out


def _dense(row_ptr, col_idx, vals, n):
    A = np.zeros((n, n))
    for i in range(n):
        for z in range(row_ptr[i], row_ptr[i + 1]):
            A[i, col_idx[z]] += vals[z]
    return A


def _bspline_integral(t, p, i):
    """int B_{i;p} = (t_{i+p+1} - t_i) / (p + 1) (any knot vector)."""
    return (t[i + p + 1] - t[i]) / (p + 1)


@pytest.mark.parametrize("dim,p,knots", _cases())
def test_pattern_is_support_overlap(oracle_mod, dim, p, knots):
    """Entry (i, j) is present iff, in every direction, the supports
    [t_i, t_{i+p+1}] and [t_j, t_{j+p+1}] overlap on an interval of positive
    length, i.e. some element holds both functions."""
    P = oracle_mod.Patch(knots, p, p + 1)
    row_ptr, col_idx = P.csr_pattern()
    nf = P.n_fun
    for i in range(P.n_dofs):
        ii = _multi(i, nf)
        ref = []
        for j in range(P.n_dofs):
            jj = _multi(j, nf)
            ok = True
            for k, t in enumerate(knots):
                lo = max(t[ii[k]], t[jj[k]])
                hi = min(t[ii[k] + p + 1], t[jj[k] + p + 1])
                ok = ok and hi > lo
            if ok:
                ref.append(j)
        assert list(col_idx[row_ptr[i]:row_ptr[i + 1]]) == ref, i


@pytest.mark.parametrize("dim,p,knots", _cases())
def test_mass_row_sums_are_basis_integrals(oracle_mod, dim, p, knots):
    """Identity geometry, rho = 1: sum_j M_ij = int phi_i = prod_k int B_{i_k},
    and the sum of all entries is the volume 1 (partition of unity)."""
    P = oracle_mod.Patch(knots, p, p + 1)
    _, Me = P.classical(stiffness=False)
    row_ptr, col_idx = P.csr_pattern()
    vals = P.assemble(Me, row_ptr, col_idx)
    sums = np.add.reduceat(vals, row_ptr[:-1])
    for i in range(P.n_dofs):
        ii = _multi(i, P.n_fun)
        ref = np.prod([_bspline_integral(knots[k], p, ii[k]) for k in range(dim)])
        assert abs(sums[i] - ref) <= 1e-15 * max(1.0, ref) * 8
    assert vals.sum() == pytest.approx(1.0, rel=1e-14)


def _global_1d(t, tr, p, which):
    """Exact 1D global matrix assembled from exact rational element integrals:
    which = 0 mass, 1 stiffness, 2 mixed int B'_a B_b (not symmetric)."""
    nf = len(t) - p - 1
    A = np.zeros((nf, nf))
    for s in range(p, len(t) - p - 1):
        if not t[s] < t[s + 1]:
            continue
        mats = element_matrices_1d(tr, p, s)
        A[s - p:s + 1, s - p:s + 1] += mats[which]
    return A


def _kron_all(mats):
    out = mats[0]
    for m in mats[1:]:
        out = np.kron(out, m)
    return out


@pytest.mark.parametrize("dim,p,K", [(2, 2, 4), (3, 1, 3), (3, 2, 3), (3, 3, 2)])
def test_global_matrices_are_kronecker_sums(oracle_mod, dim, p, K):
    """kappa = 1, identity geometry, q = p+1: the assembled global matrices are
    Kronecker sums of exactly integrated 1D global matrices (tensor
    separability, x fastest)."""
    t = wl.open_uniform_knots(K, p)
    tr = rational_open_uniform(K, p)
    P = oracle_mod.Patch([t] * dim, p, p + 1)
    Ke, Me = P.classical()
    row_ptr, col_idx = P.csr_pattern()
    Kg = _dense(row_ptr, col_idx, P.assemble(Ke, row_ptr, col_idx), P.n_dofs)
    Mg = _dense(row_ptr, col_idx, P.assemble(Me, row_ptr, col_idx), P.n_dofs)
    M1, K1 = _global_1d(t, tr, p, 0), _global_1d(t, tr, p, 1)
    Mref = _kron_all([M1] * dim)
    Kref = 0
    for d in range(dim):
        Kref = Kref + _kron_all([K1 if j == d else M1 for j in range(dim)][::-1])
    assert np.abs(Mg - Mref).max() <= 1e-14 * np.abs(Mref).max()
    assert np.abs(Kg - Kref).max() <= 1e-13 * np.abs(Kref).max()
    assert np.array_equal(Kg, Kg.T) or np.abs(Kg - Kg.T).max() <= 1e-15 * np.abs(Kg).max()


@pytest.mark.parametrize("dim,p,K", [(2, 2, 4), (3, 2, 3)])
def test_assembly_of_nonsymmetric_elements(oracle_mod, dim, p, K):
    """A non-symmetric element matrix (x-derivative of the test function times
    the trial function, exact 1D integrals in Kronecker form) assembles to the
    Kronecker product of the assembled 1D matrices: catches a transposed
    insertion that symmetric element matrices cannot."""
    t = wl.open_uniform_knots(K, p)
    tr = rational_open_uniform(K, p)
    P = oracle_mod.Patch([t] * dim, p, p + 1)
    spans = oracle_mod.spans(t, p)
    ed = [element_matrices_1d(tr, p, int(s)) for s in spans]
    Ae = np.zeros((P.E, P.N, P.N))
    for e in range(P.E):
        ek = [e % K, (e // K) % K, e // (K * K)][:dim]
        fac = [ed[ek[0]][2]] + [ed[ek[j]][0] for j in range(1, dim)]
        Ae[e] = _kron_all(fac[::-1])
    row_ptr, col_idx = P.csr_pattern()
    Ag = _dense(row_ptr, col_idx, P.assemble(Ae, row_ptr, col_idx), P.n_dofs)
    X1, M1 = _global_1d(t, tr, p, 2), _global_1d(t, tr, p, 0)
    ref = _kron_all(([X1] + [M1] * (dim - 1))[::-1])
    assert np.abs(ref - ref.T).max() > 1e-3          # the pin is not symmetric
    assert np.abs(Ag - ref).max() <= 1e-14 * np.abs(ref).max()


def _random_inputs(P, seed, curved):
    kappa = wl.lognormal(P.E * P.Q, seed)
    G = wl.curved_map_jacobian(P.knots, P.q) if curved and P.dim == 3 else None
    return kappa, G


@pytest.mark.parametrize("dim,p,knots", _cases())
def test_apply_constants_in_kernel(oracle_mod, dim, p, knots):
    """K(kappa) 1 = 0 for any kappa and geometry (gradient of a constant)."""
    P = oracle_mod.Patch(knots, p, p + 1)
    kappa, G = _random_inputs(P, 31, True)
    yK, _ = P.apply(np.ones(P.n_dofs), kappa=kappa, G=G, mass=False)
    Ke, _ = P.classical(np.arange(min(P.E, 4)), kappa=kappa, G=G, mass=False)
    assert np.abs(yK).max() <= 1e-13 * np.abs(Ke).max()


@pytest.mark.parametrize("dim,p,knots", _cases())
def test_apply_mass_to_ones(oracle_mod, dim, p, knots):
    """(M 1)_i = int phi_i = prod_k (t_{i_k+p+1} - t_{i_k}) / (p+1)."""
    P = oracle_mod.Patch(knots, p, p + 1)
    _, yM = P.apply(np.ones(P.n_dofs), stiffness=False)
    for i in range(P.n_dofs):
        ii = _multi(i, P.n_fun)
        ref = np.prod([_bspline_integral(knots[k], p, ii[k]) for k in range(dim)])
        assert abs(yM[i] - ref) <= 1e-15 * 8


def _greville(t, p):
    nf = len(t) - p - 1
    return np.array([np.mean(t[i + 1:i + p + 1]) for i in range(nf)])


@pytest.mark.parametrize("dim,p,knots", _cases())
def test_apply_linear_field_boundary_flux(oracle_mod, dim, p, knots):
    """x = Greville abscissae of direction k interpolates the coordinate x_k
    exactly, so with kappa = 1 and identity geometry
    (K x)_i = int d phi_i / dx_k = (B_{i_k}(1) - B_{i_k}(0)) prod_{l != k} int B_{i_l},
    with B_i(0) = [i == 0] and B_i(1) = [i == n_k - 1] on open knots."""
    P = oracle_mod.Patch(knots, p, p + 1)
    for k in range(dim):
        g = _greville(knots[k], p)
        x = np.array([g[_multi(i, P.n_fun)[k]] for i in range(P.n_dofs)])
        yK, _ = P.apply(x, mass=False)
        for i in range(P.n_dofs):
            ii = _multi(i, P.n_fun)
            jump = float(ii[k] == P.n_fun[k] - 1) - float(ii[k] == 0)
            ref = jump * np.prod([_bspline_integral(knots[l], p, ii[l]) for l in range(dim) if l != k])
            assert abs(yK[i] - ref) <= 1e-13, (k, i)


@pytest.mark.parametrize("dim,p,knots", _cases())
def test_apply_equals_assembled_product(oracle_mod, dim, p, knots):
    """The operator applied element by element equals the assembled CSR matrix
    times the vector (random kappa, curved geometry in 3D)."""
    P = oracle_mod.Patch(knots, p, p + 1)
    kappa, G = _random_inputs(P, 32, True)
    x = wl.normal(P.n_dofs, 33)
    yK, yM = P.apply(x, kappa=kappa, G=G)
    Ke, Me = P.classical(kappa=kappa, G=G)
    row_ptr, col_idx = P.csr_pattern()
    for A, y in ((Ke, yK), (Me, yM)):
        vals = P.assemble(A, row_ptr, col_idx)
        ref = np.array([np.dot(vals[row_ptr[i]:row_ptr[i + 1]], x[col_idx[row_ptr[i]:row_ptr[i + 1]]])
                        for i in range(P.n_dofs)])
        assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("p,K", [(2, 3), (3, 2)])
def test_apply_bilinear_matches_adjoint(oracle_mod, p, K):
    """u . (K(kappa) v) equals J = sum_q kappa_q g_q of the adjoint, which
    interpolates the gradients at the quadrature points instead of forming
    element matrices (a second path through the oracle)."""
    t = wl.open_uniform_knots(K, p)
    P = oracle_mod.Patch([t] * 3, p, p + 1)
    kappa, G = _random_inputs(P, 34, True)
    u, v = wl.normal(P.n_dofs, 35), wl.normal(P.n_dofs, 36)
    yK, _ = P.apply(v, kappa=kappa, G=G, mass=False)
    _, J = P.adjoint(u, v, kappa=kappa, G=G)
    assert float(np.dot(u, yK)) == pytest.approx(J, rel=1e-12)


# --------------------------------------------------------------------------
# Backward of the element matrices with respect to kappa and rho
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dim,p,K", [(2, 2, 3), (3, 2, 2), (3, 3, 2)])
def test_integrate_grad_linearity(oracle_mod, dim, p, K):
    """K and M are linear in kappa and rho, so for any upstream GK, GM:
    sum_q kappa_q dL/dkappa_q = <GK, K(kappa)> and sum_q rho_q dL/drho_q =
    <GM, M(rho)>, with K, M from the classical element matrices (another
    oracle path)."""
    t = wl.open_uniform_knots(K, p)
    P = oracle_mod.Patch([t] * dim, p, p + 1)
    kappa = wl.lognormal(P.E * P.Q, 71)
    rho = wl.lognormal(P.E * P.Q, 72)
    G = wl.curved_map_jacobian(P.knots, P.q) if dim == 3 else None
    GK = wl.normal(P.E * P.N * P.N, 73).reshape(P.E, P.N, P.N)
    GM = wl.normal(P.E * P.N * P.N, 74).reshape(P.E, P.N, P.N)
    gk, gr = P.integrate_grad(GK=GK, GM=GM, G=G)
    Ke, Me = P.classical(kappa=kappa, rho=rho, G=G)
    lhs_k = float((kappa.reshape(P.E, P.Q) * gk).sum())
    lhs_m = float((rho.reshape(P.E, P.Q) * gr).sum())
    assert lhs_k == pytest.approx(float((GK * Ke).sum()), rel=1e-12)
    assert lhs_m == pytest.approx(float((GM * Me).sum()), rel=1e-12)


def test_integrate_grad_outer_product_is_adjoint(oracle_mod):
    """GK_e = u_e v_e^T (the gathered global vectors) gives dL/dkappa of
    L = u^T K(kappa) v, which the adjoint computes by interpolation at the
    quadrature points (another oracle path)."""
    p, K = 2, 3
    t = wl.open_uniform_knots(K, p)
    P = oracle_mod.Patch([t] * 3, p, p + 1)
    G = wl.curved_map_jacobian(P.knots, P.q)
    u, v = wl.normal(P.n_dofs, 75), wl.normal(P.n_dofs, 76)
    dof = P.dofmap()
    GK = u[dof][:, :, None] * v[dof][:, None, :]
    gk, _ = P.integrate_grad(GK=GK, G=G)
    g, _ = P.adjoint(u, v, G=G)
    assert np.abs(gk - g).max() <= 1e-12 * np.abs(g).max()


def test_integrate_grad_central_differences(oracle_mod):
    """d<GK, K(kappa)>/dkappa_q by central differences on sampled points."""
    p, K = 2, 2
    t = wl.open_uniform_knots(K, p)
    P = oracle_mod.Patch([t] * 3, p, p + 1)
    kappa = wl.lognormal(P.E * P.Q, 77)
    GK = wl.normal(P.E * P.N * P.N, 78).reshape(P.E, P.N, P.N)
    gk, _ = P.integrate_grad(GK=GK)
    rng = np.random.default_rng(79)
    for idx in rng.choice(P.E * P.Q, size=6, replace=False):
        h = 1e-6 * kappa[idx]
        kp, km = kappa.copy(), kappa.copy()
        kp[idx] += h
        km[idx] -= h
        Kp, _ = P.classical(kappa=kp, mass=False)
        Km, _ = P.classical(kappa=km, mass=False)
        fd = float((GK * (Kp - Km)).sum()) / (2 * h)
        assert fd == pytest.approx(gk.reshape(-1)[idx], rel=1e-6, abs=1e-10)
