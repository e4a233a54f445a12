"""Helpers shared by the GPU parity tests: run the CUDA library through the
C ABI and compare with the oracle on the same seeded inputs."""
import numpy as np
import torch

from paper_2207_00280_gb300 import workloads as wl
from paper_2207_00280_gb300.plan import IgaPlan, Patch

FP64_TOL = 1e-12   # per-element relative Frobenius error, FP64
FP32_TOL = 1e-5
BF16_TOL = 5e-3


def rel_frob(gpu, ref):
    """max over elements of ||gpu - ref||_F / ||ref||_F (arrays [E][N][N])."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    num = np.sqrt(((gpu - ref) ** 2).sum(axis=(1, 2)))
    den = np.sqrt((ref ** 2).sum(axis=(1, 2)))
    return float((num / den).max())


def run_gpu(knots, p, q, kappa=None, rho=None, G=None, method="sumfact", precision="fp64",
            mass=True, stiffness=True, dof=True):
    plan = IgaPlan(Patch(list(knots), p, q), method=method, precision=precision, mass=mass,
                   stiffness=stiffness, blocking=True)
    dev = torch.device("cuda")
    kap = torch.as_tensor(kappa, device=dev, dtype=torch.float64) if kappa is not None else None
    rh = torch.as_tensor(rho, device=dev, dtype=torch.float64) if rho is not None else None
    jac = torch.as_tensor(np.ascontiguousarray(G), device=dev, dtype=torch.float64).reshape(-1) \
        if G is not None else None
    K, M, D = plan.empty_outputs(dof=dof)
    if K is not None:
        K.fill_(float("nan"))
    if M is not None:
        M.fill_(float("nan"))
    plan.integrate(kappa=kap, rho=rh, jac=jac, K=K, M=M, dof=D)
    torch.cuda.synchronize()
    N = plan.patches[0].N
    out = {
        "K": K.view(-1, N, N) if K is not None else None,
        "M": M.view(-1, N, N) if M is not None else None,
        "dof": D.view(-1, N) if D is not None else None,
        "plan": plan,
    }
    return out


def sample_elements(E, frac=0.01, seed=0, K=None, dim=3):
    """Seeded sample of element ids plus all corner elements."""
    rng = np.random.default_rng(seed)
    n = max(1, int(E * frac))
    s = set(rng.choice(E, size=min(n, E), replace=False).tolist())
    if K is not None:
        Ks = K if isinstance(K, (list, tuple)) else [K] * dim
        for c in range(2 ** dim):
            idx = [(Ks[k] - 1) if (c >> k) & 1 else 0 for k in range(dim)]
            e = idx[0] + Ks[0] * idx[1] + (Ks[0] * Ks[1] * idx[2] if dim == 3 else 0)
            s.add(e)
    return np.array(sorted(s), dtype=np.int64)
