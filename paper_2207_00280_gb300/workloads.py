"""Seeded synthetic inputs for IGA-FEM element-matrix integration.

This module is shared by the CUDA path's tests/benchmark and by the oracle's
tests.  It holds none of the method's arithmetic (no B-spline evaluation, no
integration rule of the method, no contraction): only the inputs the paper's
problem statement takes -- knot vectors (Sec. 2.3, eq. knot_vector), a
coefficient per quadrature point, a geometry Jacobian per quadrature point and
coefficient vectors per global dof -- generated from fixed seeds.

The curved-geometry Jacobian must be sampled where the quadrature points lie;
those parametric positions are placed with numpy's Gauss--Legendre routine
(``numpy.polynomial.legendre.leggauss``), a library routine independent of both
the oracle and the CUDA path.  Both sides consume the same arrays.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Seeds of the five standard workloads.
SEED_KAPPA_P3 = 2207      # 3D p=3 32^3 kappa
SEED_KAPPA_P4 = 2208      # 3D p=4 48^3 curved kappa
SEED_BATCH_SHAPES = 2209  # 64-patch batch: degrees and sizes
SEED_BATCH_KAPPA = 2210   # 64-patch batch: kappa
SEED_ADJ_KAPPA = 2211     # adjoint workload kappa
SEED_ADJ_U = 2212
SEED_ADJ_V = 2213
SEED_ADJ_FD = 2214        # finite-difference sample points
SEED_KAPPA_P8 = 2215      # 3D p=8 8^3 kappa (high-degree workload)


def open_uniform_knots(K: int, p: int) -> np.ndarray:
    """Open knot vector on [0, 1]: p+1 zeros, interior knots i/K, p+1 ones (K+2p+1 knots)."""
    inner = [i / K for i in range(1, K)]
    return np.array([0.0] * (p + 1) + inner + [1.0] * (p + 1), dtype=np.float64)


def element_breaks(t: np.ndarray) -> np.ndarray:
    """Distinct knot values in increasing order (element boundaries)."""
    return np.unique(np.asarray(t, dtype=np.float64))


def qp_coordinates(knots, q):
    """Parametric coordinates of every quadrature point: array [E][Q][d].

    q is the number of Gauss points of every direction, or one number per
    direction.  Elements are the spans between distinct knots, x fastest;
    points inside an element are ordered x fastest as well.  Gauss--Legendre
    positions come from numpy (see module docstring)."""
    d = len(knots)
    qs = [int(q)] * d if np.ndim(q) == 0 else [int(v) for v in q]
    per_dir = []
    for t, qk in zip(knots, qs):
        xr, _ = np.polynomial.legendre.leggauss(qk)
        b = element_breaks(t)
        lo, hi = b[:-1], b[1:]
        per_dir.append(0.5 * (lo + hi)[:, None] + 0.5 * (hi - lo)[:, None] * xr[None, :])
    if d == 2:
        q1, q2 = qs
        X = per_dir[0][None, :, None, :]          # [e2][e1][k2][k1]
        Y = per_dir[1][:, None, :, None]
        shape = (per_dir[1].shape[0], per_dir[0].shape[0], q2, q1)
        X = np.broadcast_to(X, shape); Y = np.broadcast_to(Y, shape)
        E = shape[0] * shape[1]
        return np.stack([X.reshape(E, q1 * q2), Y.reshape(E, q1 * q2)], axis=-1)
    q1, q2, q3 = qs
    K1, K2, K3 = (a.shape[0] for a in per_dir)
    shape = (K3, K2, K1, q3, q2, q1)               # [e3][e2][e1][k3][k2][k1]
    X = np.broadcast_to(per_dir[0][None, None, :, None, None, :], shape)
    Y = np.broadcast_to(per_dir[1][None, :, None, None, :, None], shape)
    Z = np.broadcast_to(per_dir[2][:, None, None, :, None, None], shape)
    E, Q = K1 * K2 * K3, q1 * q2 * q3
    return np.stack([X.reshape(E, Q), Y.reshape(E, Q), Z.reshape(E, Q)], axis=-1)


def curved_map_jacobian(knots, q, amp: float = 0.05) -> np.ndarray:
    """G[E][Q][3][3] = d x / d xi of the cyclic sine map

        x = xi  + amp sin(2 pi eta ) sin(2 pi zeta)
        y = eta + amp sin(2 pi zeta) sin(2 pi xi  )
        z = zeta+ amp sin(2 pi xi  ) sin(2 pi eta )

    evaluated analytically at the quadrature points (row i = component of x,
    column j = parametric direction)."""
    P = qp_coordinates(knots, q)
    tp = 2.0 * math.pi
    sx, cx = np.sin(tp * P[..., 0]), np.cos(tp * P[..., 0])
    sy, cy = np.sin(tp * P[..., 1]), np.cos(tp * P[..., 1])
    sz, cz = np.sin(tp * P[..., 2]), np.cos(tp * P[..., 2])
    a = amp * tp
    G = np.zeros(P.shape[:2] + (3, 3))
    G[..., 0, 0] = 1.0
    G[..., 0, 1] = a * cy * sz
    G[..., 0, 2] = a * sy * cz
    G[..., 1, 0] = a * sz * cx
    G[..., 1, 1] = 1.0
    G[..., 1, 2] = a * cz * sx
    G[..., 2, 0] = a * cx * sy
    G[..., 2, 1] = a * sx * cy
    G[..., 2, 2] = 1.0
    return G


def lognormal(size: int, seed: int, sigma: float = 0.5) -> np.ndarray:
    """kappa = exp(sigma Z), Z ~ N(0,1) (lognormal(0, sigma)), from a seed."""
    rng = np.random.default_rng(seed)
    return np.exp(sigma * rng.standard_normal(size))


def normal(size: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(size)


@dataclass
class PatchSpec:
    dim: int
    p: int
    K: int          # elements per side
    q: int

    @property
    def knots(self):
        return [open_uniform_knots(self.K, self.p) for _ in range(self.dim)]

    @property
    def E(self) -> int:
        return self.K ** self.dim

    @property
    def N(self) -> int:
        return (self.p + 1) ** self.dim

    @property
    def Q(self) -> int:
        return self.q ** self.dim

    @property
    def n_dofs(self) -> int:
        return (self.K + self.p) ** self.dim


def batch_specs(n_patches: int = 64, seed: int = SEED_BATCH_SHAPES, pmin: int = 1,
                pmax: int = 5, kmin: int = 4, kmax: int = 24):
    """Mixed batch of independent 3D patches: p ~ U{pmin..pmax}, K ~ U{kmin..kmax}, q = p+1."""
    rng = np.random.default_rng(seed)
    ps = rng.integers(pmin, pmax + 1, size=n_patches)
    ks = rng.integers(kmin, kmax + 1, size=n_patches)
    return [PatchSpec(3, int(p), int(k), int(p) + 1) for p, k in zip(ps, ks)]


@dataclass
class Workload:
    name: str
    spec: PatchSpec
    kappa_seed: int | None
    curved: bool = False
    extra: dict = field(default_factory=dict)

    def kappa(self) -> np.ndarray:
        if self.kappa_seed is None:
            return np.ones(self.spec.E * self.spec.Q)
        return lognormal(self.spec.E * self.spec.Q, self.kappa_seed)

    def jacobian(self):
        if not self.curved:
            return None
        return curved_map_jacobian(self.spec.knots, self.spec.q)


# The five standard workloads (2D p=2 16^2; 3D p=3 32^3; 3D p=4 48^3 curved;
# 64-patch batch; adjoint 3D p=3 40^3).
WORKLOADS = {
    "2d_p2_16": Workload("2d_p2_16", PatchSpec(2, 2, 16, 3), None),
    "3d_p3_32": Workload("3d_p3_32", PatchSpec(3, 3, 32, 4), SEED_KAPPA_P3),
    "3d_p4_48_curved": Workload("3d_p4_48_curved", PatchSpec(3, 4, 48, 5), SEED_KAPPA_P4, curved=True),
    "3d_p3_40_adjoint": Workload("3d_p3_40_adjoint", PatchSpec(3, 3, 40, 4), SEED_ADJ_KAPPA),
    # reduced sizes of the same workloads, for profiler captures (inputs + outputs > L2)
    "3d_p3_16": Workload("3d_p3_16", PatchSpec(3, 3, 16, 4), SEED_KAPPA_P3),
    "3d_p3_20": Workload("3d_p3_20", PatchSpec(3, 3, 20, 4), SEED_KAPPA_P3),
    # the largest degree class of the 64-patch batch, alone
    "3d_p5_16": Workload("3d_p5_16", PatchSpec(3, 5, 16, 6), SEED_BATCH_KAPPA),
    "3d_p5_10": Workload("3d_p5_10", PatchSpec(3, 5, 10, 6), SEED_BATCH_KAPPA),
    "3d_p4_16": Workload("3d_p4_16", PatchSpec(3, 4, 16, 5), SEED_BATCH_KAPPA),
    "3d_p4_24_curved": Workload("3d_p4_24_curved", PatchSpec(3, 4, 24, 5), SEED_KAPPA_P4, curved=True),
    # high degree (the paper's experiments run p up to 9, Sec. 4): 3D p=8,
    # 8^3 elements, 9^3 Gauss points, lognormal kappa, identity geometry; the
    # element matrices (729 x 729) are formed by the runtime-sized FP64 kernels
    "3d_p8_8": Workload("3d_p8_8", PatchSpec(3, 8, 8, 9), SEED_KAPPA_P8),
}
