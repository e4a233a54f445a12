"""FP64 CPU oracle for IGA-FEM element-matrix integration (arxiv 2207.00280).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library (``paper_2207_00280_gb300``)
and never serves as a fallback for it.

The arithmetic lives in ``iga_oracle.c`` (plain C, ``-O2 -ffp-contract=off``);
this module only compiles it, loads it with ctypes and marshals numpy arrays.
Every routine cites the passage of the paper it follows in ``iga_oracle.h``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "iga_oracle.c")
_HDR = os.path.join(_HERE, "iga_oracle.h")
_SO = os.path.join(_HERE, "libiga_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libiga_oracle.so`` (gcc, FP64, no FMA contraction)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Patch(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("p", ctypes.c_int), ("q", ctypes.c_int),
                ("m", ctypes.c_int * 3), ("t", ctypes.c_void_p * 3),
                ("pd", ctypes.c_int * 3), ("qd", ctypes.c_int * 3)]


def lib():
    """Load the oracle.  IGA_ORACLE_SO may name another build of iga_oracle.c
    (the mutation tests use it to check that the pins reject planted bugs)."""
    global _lib
    with _lock:
        if _lib is None:
            alt = os.environ.get("IGA_ORACLE_SO")
            if alt:
                L = ctypes.CDLL(alt)
            else:
                build()
                L = ctypes.CDLL(_SO)
            dp = ctypes.c_void_p
            L.ora_gauss_legendre.argtypes = [ctypes.c_int, dp, dp]
            L.ora_gauss_legendre.restype = ctypes.c_int
            L.ora_bspline.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_double]
            L.ora_bspline.restype = ctypes.c_double
            L.ora_bspline_deriv.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_double]
            L.ora_bspline_deriv.restype = ctypes.c_double
            L.ora_spans.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
            L.ora_spans.restype = ctypes.c_int
            L.ora_basis_1d.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
            L.ora_basis_1d.restype = None
            pp = ctypes.POINTER(_Patch)
            for name in ("ora_classical", "ora_sumfact"):
                f = getattr(L, name)
                f.argtypes = [pp, dp, ctypes.c_int64, dp, dp, dp, dp, dp]
                f.restype = ctypes.c_int
            L.ora_dofmap.argtypes = [pp, dp, ctypes.c_int64, dp]
            L.ora_dofmap.restype = ctypes.c_int
            L.ora_adjoint.argtypes = [pp, dp, ctypes.c_int64, dp, dp, dp, dp, dp, dp]
            L.ora_adjoint.restype = ctypes.c_int
            L.ora_csr_pattern.argtypes = [pp, dp, dp]
            L.ora_csr_pattern.restype = ctypes.c_int
            L.ora_assemble.argtypes = [pp, dp, dp, dp, dp]
            L.ora_assemble.restype = ctypes.c_int
            L.ora_apply.argtypes = [pp, dp, dp, dp, dp, dp, dp]
            L.ora_apply.restype = ctypes.c_int
            L.ora_wq_points.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int]
            L.ora_wq_points.restype = ctypes.c_int
            L.ora_wq_weights.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp]
            L.ora_wq_weights.restype = ctypes.c_int
            L.ora_wq_mass.argtypes = [pp, dp, dp, dp, dp]
            L.ora_wq_mass.restype = ctypes.c_int
            L.ora_wq_weights_deriv.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp]
            L.ora_wq_weights_deriv.restype = ctypes.c_int
            L.ora_wq_stiffness.argtypes = [pp, dp, dp, dp, dp]
            L.ora_wq_stiffness.restype = ctypes.c_int
            L.ora_integrate_grad.argtypes = [pp, dp, ctypes.c_int64, dp, dp, dp, dp, dp]
            L.ora_integrate_grad.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def gauss_legendre(q: int):
    """Gauss--Legendre nodes and weights on [-1, 1] (Golub--Welsch)."""
    x = np.zeros(q)
    w = np.zeros(q)
    if lib().ora_gauss_legendre(q, _ptr(x), _ptr(w)) != 0:
        raise ValueError(f"bad q={q}")
    return x, w


def bspline(t, i: int, p: int, xi: float) -> float:
    t = _f64(t)
    return lib().ora_bspline(_ptr(t), i, p, float(xi))


def bspline_deriv(t, i: int, p: int, xi: float) -> float:
    t = _f64(t)
    return lib().ora_bspline_deriv(_ptr(t), i, p, float(xi))


def spans(t, p: int) -> np.ndarray:
    t = _f64(t)
    out = np.zeros(len(t), dtype=np.int32)
    c = lib().ora_spans(_ptr(t), len(t), p, _ptr(out))
    return out[:c].copy()


def basis_1d(t, p: int, s: int, q: int):
    """(xi[q], w[q], val[q][p+1], der[q][p+1]) of span s."""
    t = _f64(t)
    xi = np.zeros(q); w = np.zeros(q)
    val = np.zeros((q, p + 1)); der = np.zeros((q, p + 1))
    lib().ora_basis_1d(_ptr(t), p, s, q, _ptr(xi), _ptr(w), _ptr(val), _ptr(der))
    return xi, w, val, der


def wq_points(t, p: int) -> np.ndarray:
    """Global weighted-quadrature points of one direction (see iga_oracle.h)."""
    t = _f64(t)
    cap = 4 * len(t) + 8
    x = np.zeros(cap)
    n = lib().ora_wq_points(_ptr(t), len(t), p, _ptr(x), cap)
    if n < 1:
        raise ValueError("oracle rejected its arguments")
    return x[:n].copy()


def wq_weights(t, p: int, x, deriv: bool = False) -> np.ndarray:
    """W[n_functions][n_points]: least-norm weighted-quadrature weights, the
    mass rule or (deriv) the derivative rule."""
    t = _f64(t)
    x = _f64(x)
    W = np.zeros((len(t) - p - 1, len(x)))
    fn = lib().ora_wq_weights_deriv if deriv else lib().ora_wq_weights
    if fn(_ptr(t), len(t), p, _ptr(x), len(x), _ptr(W)) != 0:
        raise ValueError("oracle: singular weighted-quadrature system")
    return W


def _per_dir(x, dim):
    if np.ndim(x) == 0:
        return [int(x)] * dim
    x = [int(v) for v in x]
    if len(x) != dim:
        raise ValueError(f"expected {dim} values per direction")
    return x


class Patch:
    """One tensor-product patch: dimension, knot vectors, and the degree and
    Gauss points of each direction (an int for all directions, or one per
    direction)."""

    def __init__(self, knots, p, q):
        self.knots = [_f64(t) for t in knots]
        self.dim = len(self.knots)
        if self.dim not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        self.pd = _per_dir(p, self.dim)
        self.qd = _per_dir(q, self.dim)
        # p, q, n: the common value when every direction has the same one
        self.p = self.pd[0] if len(set(self.pd)) == 1 else None
        self.q = self.qd[0] if len(set(self.qd)) == 1 else None
        self.n = self.p + 1 if self.p is not None else None
        self.nd = [pk + 1 for pk in self.pd]
        self.N = int(np.prod(self.nd))
        self.Q = int(np.prod(self.qd))
        self.n_el = [len(spans(t, pk)) for t, pk in zip(self.knots, self.pd)]
        self.E = int(np.prod(self.n_el))
        self.n_fun = [len(t) - pk - 1 for t, pk in zip(self.knots, self.pd)]
        self.n_dofs = int(np.prod(self.n_fun))
        s = _Patch()
        s.dim, s.p, s.q = self.dim, self.pd[0], self.qd[0]
        for k, t in enumerate(self.knots):
            s.m[k] = len(t)
            s.t[k] = t.ctypes.data
            s.pd[k] = self.pd[k]
            s.qd[k] = self.qd[k]
        self._s = s

    def _elems(self, elems):
        if elems is None:
            elems = np.arange(self.E, dtype=np.int64)
        return np.ascontiguousarray(elems, dtype=np.int64)

    def _check_qp(self, a, per_qp):
        if a is None:
            return None
        a = _f64(a)
        if a.size != self.E * self.Q * per_qp:
            raise ValueError(f"expected {self.E * self.Q * per_qp} values, got {a.size}")
        return a

    def _mats(self, fn, elems, kappa, rho, G, stiffness, mass):
        el = self._elems(elems)
        kappa = self._check_qp(kappa, 1)
        rho = self._check_qp(rho, 1)
        G = self._check_qp(G, self.dim * self.dim)
        if stiffness and kappa is None:
            kappa = np.ones(self.E * self.Q)
        K = np.zeros((len(el), self.N, self.N)) if stiffness else None
        M = np.zeros((len(el), self.N, self.N)) if mass else None
        rc = fn(ctypes.byref(self._s), _ptr(el), len(el), _ptr(kappa), _ptr(rho), _ptr(G),
                _ptr(K), _ptr(M))
        if rc != 0:
            raise ValueError("oracle rejected its arguments")
        return K, M

    def classical(self, elems=None, kappa=None, rho=None, G=None, stiffness=True, mass=True):
        """Element matrices by Algorithm 1 (the naive nested loop)."""
        return self._mats(lib().ora_classical, elems, kappa, rho, G, stiffness, mass)

    def sumfact(self, elems=None, kappa=None, rho=None, G=None, stiffness=True, mass=True):
        """Element matrices by Algorithm 2 (sum factorization, literal)."""
        return self._mats(lib().ora_sumfact, elems, kappa, rho, G, stiffness, mass)

    def dofmap(self, elems=None) -> np.ndarray:
        el = self._elems(elems)
        out = np.zeros((len(el), self.N), dtype=np.int32)
        if lib().ora_dofmap(ctypes.byref(self._s), _ptr(el), len(el), _ptr(out)) != 0:
            raise ValueError("oracle rejected its arguments")
        return out

    def adjoint(self, u, v, kappa=None, G=None, elems=None):
        """(g[n_sel][Q], J) with g = dJ/dkappa for J = u^T K(kappa) v."""
        el = self._elems(elems)
        u = _f64(u); v = _f64(v)
        if u.size != self.n_dofs or v.size != self.n_dofs:
            raise ValueError("u, v must have one value per global dof")
        kappa = self._check_qp(kappa, 1)
        G = self._check_qp(G, self.dim * self.dim)
        g = np.zeros((len(el), self.Q))
        J = np.zeros(1)
        rc = lib().ora_adjoint(ctypes.byref(self._s), _ptr(el), len(el), _ptr(kappa), _ptr(G),
                               _ptr(u), _ptr(v), _ptr(g), _ptr(J))
        if rc != 0:
            raise ValueError("oracle rejected its arguments")
        return g, float(J[0])

    def csr_pattern(self):
        """(row_ptr[n_dofs + 1] int64, col_idx[nnz] int32) of the assembled global matrix."""
        row_ptr = np.zeros(self.n_dofs + 1, dtype=np.int64)
        if lib().ora_csr_pattern(ctypes.byref(self._s), _ptr(row_ptr), None) != 0:
            raise ValueError("oracle rejected its arguments")
        col_idx = np.zeros(int(row_ptr[-1]), dtype=np.int32)
        if lib().ora_csr_pattern(ctypes.byref(self._s), _ptr(row_ptr), _ptr(col_idx)) != 0:
            raise ValueError("oracle rejected its arguments")
        return row_ptr, col_idx

    def assemble(self, Ae, row_ptr, col_idx):
        """CSR values of sum_e P_e^T Ae[e] P_e for element matrices Ae[E][N][N]."""
        Ae = _f64(Ae)
        if Ae.size != self.E * self.N * self.N:
            raise ValueError("Ae must hold every element's matrix")
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        vals = np.zeros(len(col_idx))
        rc = lib().ora_assemble(ctypes.byref(self._s), _ptr(row_ptr), _ptr(col_idx), _ptr(Ae),
                                _ptr(vals))
        if rc != 0:
            raise ValueError(f"oracle assembly failed ({rc})")
        return vals

    def apply(self, x, kappa=None, rho=None, G=None, stiffness=True, mass=True):
        """(K x, M x) of the assembled operators (either may be None if not asked for)."""
        x = _f64(x)
        if x.size != self.n_dofs:
            raise ValueError("x must have one value per global dof")
        kappa = self._check_qp(kappa, 1)
        rho = self._check_qp(rho, 1)
        G = self._check_qp(G, self.dim * self.dim)
        yK = np.zeros(self.n_dofs) if stiffness else None
        yM = np.zeros(self.n_dofs) if mass else None
        rc = lib().ora_apply(ctypes.byref(self._s), _ptr(kappa), _ptr(rho), _ptr(G), _ptr(x),
                             _ptr(yK), _ptr(yM))
        if rc != 0:
            raise ValueError("oracle rejected its arguments")
        return yK, yM

    def wq_mass(self, row_ptr, col_idx, c=None):
        """CSR values of the weighted-quadrature mass matrix; c at the tensor grid
        of wq_points (x fastest) or None (= 1)."""
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        c = _f64(c)
        vals = np.zeros(len(col_idx))
        if lib().ora_wq_mass(ctypes.byref(self._s), _ptr(c), _ptr(row_ptr), _ptr(col_idx),
                             _ptr(vals)) != 0:
            raise ValueError("oracle: weighted quadrature failed")
        return vals

    def wq_stiffness(self, row_ptr, col_idx, c=None):
        """CSR values of the weighted-quadrature diffusion stiffness (p >= 2);
        c as for wq_mass."""
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        c = _f64(c)
        vals = np.zeros(len(col_idx))
        if lib().ora_wq_stiffness(ctypes.byref(self._s), _ptr(c), _ptr(row_ptr), _ptr(col_idx),
                                  _ptr(vals)) != 0:
            raise ValueError("oracle: weighted-quadrature stiffness failed")
        return vals

    def integrate_grad(self, GK=None, GM=None, G=None, elems=None):
        """(dL/dkappa [n_sel][Q], dL/drho [n_sel][Q]) from upstream gradients of the
        element matrices GK, GM [n_sel][N][N] (either may be None)."""
        el = self._elems(elems)
        G = self._check_qp(G, self.dim * self.dim)
        GK = _f64(GK)
        GM = _f64(GM)
        gk = np.zeros((len(el), self.Q)) if GK is not None else None
        gr = np.zeros((len(el), self.Q)) if GM is not None else None
        rc = lib().ora_integrate_grad(ctypes.byref(self._s), _ptr(el), len(el), _ptr(G), _ptr(GK),
                                      _ptr(GM), _ptr(gk), _ptr(gr))
        if rc != 0:
            raise ValueError("oracle rejected its arguments")
        return gk, gr
