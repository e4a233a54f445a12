"""Thin ctypes binding of the C ABI in include/iga.h (argument marshalling only).

The functions keep the C names: ``iga_plan``, ``iga_integrate``,
``iga_integrate_backward``, ``iga_destroy``, ``iga_status_str``.  They take
plain integers for device pointers (e.g. ``tensor.data_ptr()``) and streams
(``torch.cuda.current_stream().cuda_stream``).  Every step of the computation
runs in the CUDA library; there is no fallback: if ``libiga.so`` is missing
the import of this module's functions raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libiga.so")

IGA_OK = 0
IGA_ERR_ARG = 1
IGA_ERR_KNOTS = 2
IGA_ERR_UNSUPPORTED = 3
IGA_ERR_CUDA = 4
IGA_ERR_OOM = 5
IGA_ERR_TIMEOUT = 6
IGA_ERR_DEVICE = 7
IGA_ERR_TOO_LARGE = 8
IGA_CLASSICAL = 0
IGA_SUMFACT = 1
IGA_FP64 = 0
IGA_FP32 = 1
IGA_BF16 = 2
IGA_FP64_DF = 3
IGA_MASS = 1
IGA_STIFF = 2
IGA_SCHED_AUTO = 0
IGA_SCHED_PER_PATCH = 1
IGA_SCHED_PERSISTENT = 2
IGA_SCHED_PERSISTENT_GRAPH = 3
IGA_PROBE_DFMA = 0
IGA_PROBE_DMMA = 1
IGA_PROBE_FFMA = 2

# Every exported symbol of include/iga.h and include/iga_probe.h (checked by
# tests/test_capi_host.py).
EXPORTED = ("iga_plan", "iga_integrate", "iga_integrate_backward", "iga_integrate_grad",
            "iga_basis_tables",
            "iga_csr_pattern", "iga_assemble", "iga_apply", "iga_wq_points", "iga_wq_mass",
            "iga_wq_stiffness",
            "iga_profile_read", "iga_adjoint_noalloc", "iga_destroy", "iga_status_str",
            "iga_probe_rate")


class IgaError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {iga_status_str(code)} ({code})")
        self.code = code


class PatchDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("degree", ctypes.c_int * 3), ("n_gauss", ctypes.c_int * 3),
                ("n_knots", ctypes.c_int * 3), ("knots", ctypes.c_void_p * 3)]

    def set_order(self, degree, n_gauss):
        """Degree and Gauss points of every direction: an int for all, or one per direction."""
        ps = [int(degree)] * 3 if isinstance(degree, (int,)) or getattr(degree, "ndim", 1) == 0 \
            else [int(v) for v in degree] + [0] * (3 - len(degree))
        qs = [int(n_gauss)] * 3 if isinstance(n_gauss, (int,)) or getattr(n_gauss, "ndim", 1) == 0 \
            else [int(v) for v in n_gauss] + [0] * (3 - len(n_gauss))
        for k in range(3):
            self.degree[k] = ps[k]
            self.n_gauss[k] = qs[k]


class PlanOpts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("precision", ctypes.c_int),
                ("matrices", ctypes.c_int), ("schedule", ctypes.c_int),
                ("blocking", ctypes.c_int), ("profile", ctypes.c_int)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_elements", ctypes.c_int64), ("n_qp", ctypes.c_int64),
                ("n_dofs", ctypes.c_int64), ("n_mat_entries", ctypes.c_int64),
                ("n_dofmap_entries", ctypes.c_int64), ("n_table_entries", ctypes.c_int64),
                ("dim", ctypes.c_int),
                ("n_patches", ctypes.c_int), ("local_n", ctypes.c_int),
                ("elem_offset", ctypes.POINTER(ctypes.c_int64)),
                ("qp_offset", ctypes.POINTER(ctypes.c_int64)),
                ("dof_offset", ctypes.POINTER(ctypes.c_int64)),
                ("mat_offset", ctypes.POINTER(ctypes.c_int64)),
                ("dofmap_offset", ctypes.POINTER(ctypes.c_int64)),
                ("n_csr_nnz", ctypes.c_int64)]


_lib = None
_lock = threading.Lock()


def lib() -> ctypes.CDLL:
    """Load libiga.so.  Raises (never falls back) if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(
                    f"CUDA library {LIB_PATH} is not built; run "
                    "`python -m paper_2207_00280_gb300.build` (needs nvcc)")
            L = ctypes.CDLL(LIB_PATH)
            vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
            L.iga_plan.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(PatchDesc), i32,
                                   ctypes.POINTER(PlanOpts), ctypes.POINTER(PlanInfo)]
            L.iga_plan.restype = i32
            L.iga_integrate.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
            L.iga_integrate.restype = i32
            L.iga_integrate_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
            L.iga_integrate_backward.restype = i32
            L.iga_integrate_grad.argtypes = [vp, vp, vp, vp, vp, vp, vp]
            L.iga_integrate_grad.restype = i32
            L.iga_basis_tables.argtypes = [vp, vp, vp]
            L.iga_basis_tables.restype = i32
            L.iga_csr_pattern.argtypes = [vp, vp, vp, vp]
            L.iga_csr_pattern.restype = i32
            L.iga_assemble.argtypes = [vp, vp, vp, vp]
            L.iga_assemble.restype = i32
            L.iga_apply.argtypes = [vp, vp, vp, vp, vp, ctypes.c_double, ctypes.c_double, vp, vp]
            L.iga_apply.restype = i32
            L.iga_wq_points.argtypes = [vp, i32, i32, vp, ctypes.POINTER(ctypes.c_int64)]
            L.iga_wq_points.restype = i32
            L.iga_wq_mass.argtypes = [vp, vp, vp, vp]
            L.iga_wq_mass.restype = i32
            L.iga_wq_stiffness.argtypes = [vp, vp, vp, vp]
            L.iga_wq_stiffness.restype = i32
            L.iga_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_int64)]
            L.iga_profile_read.restype = i32
            L.iga_adjoint_noalloc.argtypes = [ctypes.POINTER(PatchDesc), vp, vp, vp, vp, vp, vp, vp]
            L.iga_adjoint_noalloc.restype = i32
            L.iga_destroy.argtypes = [vp]
            L.iga_destroy.restype = i32
            L.iga_status_str.argtypes = [i32]
            L.iga_status_str.restype = ctypes.c_char_p
            L.iga_probe_rate.argtypes = [i32, i64, i32, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double), vp]
            L.iga_probe_rate.restype = i32
            _lib = L
    return _lib


def iga_status_str(code: int) -> str:
    return lib().iga_status_str(int(code)).decode()


def iga_plan(patches, opts: PlanOpts):
    """patches: sequence of PatchDesc (knot arrays must stay alive during the call).
    Returns (plan handle, PlanInfo)."""
    arr = (PatchDesc * len(patches))(*patches)
    h = ctypes.c_void_p()
    info = PlanInfo()
    rc = lib().iga_plan(ctypes.byref(h), arr, len(patches), ctypes.byref(opts), ctypes.byref(info))
    if rc != IGA_OK:
        raise IgaError(rc, "iga_plan")
    return h, info


def iga_integrate(plan, kappa, rho, jac, K_out, M_out, dof_out, stream) -> int:
    return lib().iga_integrate(plan, kappa, rho, jac, K_out, M_out, dof_out, stream)


def iga_integrate_backward(plan, kappa, jac, u, v, grad_kappa, J_out, stream) -> int:
    return lib().iga_integrate_backward(plan, kappa, jac, u, v, grad_kappa, J_out, stream)


def iga_integrate_grad(plan, jac, GK, GM, grad_kappa, grad_rho, stream) -> int:
    return lib().iga_integrate_grad(plan, jac, GK, GM, grad_kappa, grad_rho, stream)


def iga_basis_tables(plan, out, stream) -> int:
    return lib().iga_basis_tables(plan, out, stream)


def iga_csr_pattern(plan, row_ptr, col_idx, stream) -> int:
    return lib().iga_csr_pattern(plan, row_ptr, col_idx, stream)


def iga_assemble(plan, A_elem, values, stream) -> int:
    return lib().iga_assemble(plan, A_elem, values, stream)


def iga_apply(plan, kappa, rho, jac, x, alpha, beta, y, stream) -> int:
    return lib().iga_apply(plan, kappa, rho, jac, x, float(alpha), float(beta), y, stream)


def iga_wq_points(plan, patch, dir_, x_out, n_out) -> int:
    return lib().iga_wq_points(plan, int(patch), int(dir_), x_out, n_out)


def iga_wq_mass(plan, c, values, stream) -> int:
    return lib().iga_wq_mass(plan, c, values, stream)


def iga_wq_stiffness(plan, c, values, stream) -> int:
    return lib().iga_wq_stiffness(plan, c, values, stream)


def iga_profile_read(plan):
    """(kernel ms, launches) since the last read; raises if profiling is off."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    rc = lib().iga_profile_read(plan, ctypes.byref(ms), ctypes.byref(n))
    if rc != IGA_OK:
        raise IgaError(rc, "iga_profile_read")
    return ms.value, n.value


def iga_destroy(plan) -> int:
    return lib().iga_destroy(plan)


def iga_probe_rate(kind: int, iters: int, ctas_per_sm: int, stream) -> tuple:
    """(device ms, flops) of one arithmetic-rate probe (include/iga_probe.h)."""
    ms = ctypes.c_double()
    fl = ctypes.c_double()
    rc = lib().iga_probe_rate(int(kind), int(iters), int(ctas_per_sm), ctypes.byref(ms),
                              ctypes.byref(fl), stream)
    if rc != IGA_OK:
        raise IgaError(rc, "iga_probe_rate")
    return ms.value, fl.value
