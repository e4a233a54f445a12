"""Torch-facing wrapper of the C ABI: owns a plan, allocates outputs as torch
tensors and passes raw device pointers and the current stream to the library.
Torch supplies device memory and streams only; all computation is in libiga.so.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import capi

_METHODS = {"classical": capi.IGA_CLASSICAL, "sumfact": capi.IGA_SUMFACT}
_PRECISIONS = {"fp64": capi.IGA_FP64, "fp32": capi.IGA_FP32, "bf16": capi.IGA_BF16,
               "fp64_df": capi.IGA_FP64_DF}


@dataclass
class Patch:
    knots: list          # one 1D array per direction
    degree: object       # int (every direction) or one int per direction
    n_gauss: object      # int (every direction) or one int per direction

    @property
    def dim(self) -> int:
        return len(self.knots)

    def per_dir(self, v):
        return [int(v)] * self.dim if np.ndim(v) == 0 else [int(x) for x in v]

    @property
    def degrees(self):
        return self.per_dir(self.degree)

    @property
    def gauss(self):
        return self.per_dir(self.n_gauss)

    @property
    def N(self) -> int:
        return int(np.prod([p + 1 for p in self.degrees]))

    @property
    def Q(self) -> int:
        return int(np.prod(self.gauss))


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class IgaPlan:
    """Plan for one patch or a batch of patches (same dimension)."""

    def __init__(self, patches, method: str = "sumfact", precision: str = "fp64",
                 mass: bool = True, stiffness: bool = True, schedule: int = 0,
                 blocking: bool = True, profile: bool = False):
        if isinstance(patches, Patch):
            patches = [patches]
        self.patches = list(patches)
        self.precision = precision
        self.method = method
        self._knots = []
        descs = []
        for pt in self.patches:
            d = capi.PatchDesc()
            d.dim = pt.dim
            d.set_order(pt.degrees, pt.gauss)
            for k, t in enumerate(pt.knots):
                arr = np.ascontiguousarray(t, dtype=np.float64)
                self._knots.append(arr)
                d.n_knots[k] = len(arr)
                d.knots[k] = arr.ctypes.data
            descs.append(d)
        opts = capi.PlanOpts()
        opts.method = _METHODS[method]
        opts.precision = _PRECISIONS[precision]
        opts.matrices = (capi.IGA_MASS if mass else 0) | (capi.IGA_STIFF if stiffness else 0)
        opts.schedule = int(schedule)
        opts.blocking = 1 if blocking else 0
        opts.profile = 1 if profile else 0
        self.mass, self.stiffness = mass, stiffness
        self.handle, info = capi.iga_plan(descs, opts)
        self.info = info
        npt = info.n_patches
        self.elem_offset = [info.elem_offset[i] for i in range(npt + 1)]
        self.qp_offset = [info.qp_offset[i] for i in range(npt + 1)]
        self.dof_offset = [info.dof_offset[i] for i in range(npt + 1)]
        self.mat_offset = [info.mat_offset[i] for i in range(npt + 1)]
        self.dofmap_offset = [info.dofmap_offset[i] for i in range(npt + 1)]
        self.out_dtype = torch.float64 if precision in ("fp64", "fp64_df") else torch.float32

    # -- sizes ---------------------------------------------------------------
    @property
    def n_elements(self) -> int:
        return self.info.n_elements

    @property
    def n_qp(self) -> int:
        return self.info.n_qp

    @property
    def n_dofs(self) -> int:
        return self.info.n_dofs

    def empty_outputs(self, device="cuda", dof: bool = True):
        n = self.info.n_mat_entries
        K = torch.empty(n, dtype=self.out_dtype, device=device) if self.stiffness else None
        M = torch.empty(n, dtype=self.out_dtype, device=device) if self.mass else None
        D = torch.empty(self.info.n_dofmap_entries, dtype=torch.int32, device=device) if dof else None
        return K, M, D

    # -- calls -----------------------------------------------------------------
    def integrate(self, kappa=None, rho=None, jac=None, K=None, M=None, dof=None, stream=None):
        rc = capi.iga_integrate(self.handle, _ptr(kappa), _ptr(rho), _ptr(jac), _ptr(K), _ptr(M),
                                _ptr(dof), _stream(stream))
        if rc != capi.IGA_OK:
            raise capi.IgaError(rc, "iga_integrate")
        return K, M, dof

    def backward(self, kappa, u, v, grad=None, J=None, jac=None, stream=None):
        rc = capi.iga_integrate_backward(self.handle, _ptr(kappa), _ptr(jac), _ptr(u), _ptr(v),
                                         _ptr(grad), _ptr(J), _stream(stream))
        if rc != capi.IGA_OK:
            raise capi.IgaError(rc, "iga_integrate_backward")
        return grad, J

    def integrate_grad(self, GK=None, GM=None, jac=None, grad_kappa=None, grad_rho=None,
                       stream=None):
        """(dL/dkappa, dL/drho) at every quadrature point from upstream gradients
        GK = dL/dK and GM = dL/dM (layout and dtype of integrate's K and M)."""
        ref = GK if GK is not None else GM
        if ref is None:
            raise ValueError("integrate_grad needs GK or GM")
        if GK is not None and grad_kappa is None:
            grad_kappa = torch.empty(self.n_qp, dtype=ref.dtype, device=ref.device)
        if GM is not None and grad_rho is None:
            grad_rho = torch.empty(self.n_qp, dtype=ref.dtype, device=ref.device)
        rc = capi.iga_integrate_grad(self.handle, _ptr(jac), _ptr(GK), _ptr(GM),
                                     _ptr(grad_kappa if GK is not None else None),
                                     _ptr(grad_rho if GM is not None else None), _stream(stream))
        if rc != capi.IGA_OK:
            raise capi.IgaError(rc, "iga_integrate_grad")
        return (grad_kappa if GK is not None else None), (grad_rho if GM is not None else None)

    @property
    def n_csr_nnz(self) -> int:
        return self.info.n_csr_nnz

    def csr_pattern(self, stream=None):
        """(row_ptr int64 [n_dofs + 1], col_idx int32 [nnz]) of the assembled matrix."""
        row_ptr = torch.empty(self.n_dofs + 1, dtype=torch.int64, device="cuda")
        col_idx = torch.empty(self.n_csr_nnz, dtype=torch.int32, device="cuda")
        rc = capi.iga_csr_pattern(self.handle, _ptr(row_ptr), _ptr(col_idx), _stream(stream))
        if rc != capi.IGA_OK:
            raise capi.IgaError(rc, "iga_csr_pattern")
        return row_ptr, col_idx

    def assemble(self, A_elem, values=None, stream=None):
        """CSR values of the global matrix assembled from per-element matrices
        (a K or M output of integrate)."""
        if values is None:
            values = torch.empty(self.n_csr_nnz, dtype=self.out_dtype, device=A_elem.device)
        rc = capi.iga_assemble(self.handle, _ptr(A_elem), _ptr(values), _stream(stream))
        if rc != capi.IGA_OK:
            raise capi.IgaError(rc, "iga_assemble")
        return values

    def apply(self, x, kappa=None, rho=None, jac=None, alpha=1.0, beta=0.0, y=None, stream=None):
        """y = alpha K(kappa) x + beta M(rho) x, matrix-free."""
        if y is None:
            y = torch.empty_like(x)
        rc = capi.iga_apply(self.handle, _ptr(kappa), _ptr(rho), _ptr(jac), _ptr(x), alpha, beta,
                            _ptr(y), _stream(stream))
        if rc != capi.IGA_OK:
            raise capi.IgaError(rc, "iga_apply")
        return y

    def wq_points(self, patch: int = 0):
        """Parametric coordinates of the weighted-quadrature points, one array per direction."""
        out = []
        for d in range(self.patches[patch].dim):
            n = ctypes.c_int64()
            rc = capi.iga_wq_points(self.handle, patch, d, None, ctypes.byref(n))
            if rc != capi.IGA_OK:
                raise capi.IgaError(rc, "iga_wq_points")
            x = np.zeros(n.value)
            rc = capi.iga_wq_points(self.handle, patch, d, x.ctypes.data_as(ctypes.c_void_p),
                                    ctypes.byref(n))
            if rc != capi.IGA_OK:
                raise capi.IgaError(rc, "iga_wq_points")
            out.append(x)
        return out

    def wq_grid_size(self, patch: int = -1) -> int:
        n = ctypes.c_int64()
        rc = capi.iga_wq_points(self.handle, patch, -1, None, ctypes.byref(n))
        if rc != capi.IGA_OK:
            raise capi.IgaError(rc, "iga_wq_points")
        return n.value

    def wq_mass(self, c=None, values=None, stream=None):
        """CSR values of the weighted-quadrature mass matrix (c on the point grid or None = 1)."""
        if values is None:
            values = torch.empty(self.n_csr_nnz, dtype=torch.float64, device="cuda")
        rc = capi.iga_wq_mass(self.handle, _ptr(c), _ptr(values), _stream(stream))
        if rc != capi.IGA_OK:
            raise capi.IgaError(rc, "iga_wq_mass")
        return values

    def wq_stiffness(self, c=None, values=None, stream=None):
        """CSR values of the weighted-quadrature diffusion stiffness (c on the point
        grid or None = 1; 3D, 2 <= p <= 4)."""
        if values is None:
            values = torch.empty(self.n_csr_nnz, dtype=torch.float64, device="cuda")
        rc = capi.iga_wq_stiffness(self.handle, _ptr(c), _ptr(values), _stream(stream))
        if rc != capi.IGA_OK:
            raise capi.IgaError(rc, "iga_wq_stiffness")
        return values

    def profile_read(self):
        """(ms, launches) of the element-matrix kernels since the last read."""
        return capi.iga_profile_read(self.handle)

    def basis_tables(self, stream=None):
        out = torch.empty(self.info.n_table_entries, dtype=torch.float64, device="cuda")
        rc = capi.iga_basis_tables(self.handle, _ptr(out), _stream(stream))
        if rc != capi.IGA_OK:
            raise capi.IgaError(rc, "iga_basis_tables")
        return out

    def patch_view(self, flat, i: int):
        """Reshape patch i's block of a flat K/M output to [E][N][N]."""
        N = self.patches[i].N
        a, b = self.mat_offset[i], self.mat_offset[i + 1]
        return flat[a:b].view(-1, N, N)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            rc = capi.iga_destroy(self.handle)
            self.handle = None
            if rc != capi.IGA_OK:
                raise capi.IgaError(rc, "iga_destroy")

    def __del__(self):
        try:
            if getattr(self, "handle", None) is not None and self.handle.value:
                capi.iga_destroy(self.handle)
                self.handle = None
        except Exception:
            pass
