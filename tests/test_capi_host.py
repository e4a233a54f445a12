"""CPU tests of the C ABI: the library builds and loads, exports every symbol
include/iga.h declares, and rejects bad arguments and knot vectors on the host
before any CUDA call.  No kernel is launched."""
import ctypes
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_2207_00280_gb300 import build, capi as c
    if not os.path.exists(c.LIB_PATH):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc unavailable and library not built")
        build.build()
    c.lib()
    return c


def _declared_symbols():
    out = set()
    for name in os.listdir(os.path.join(ROOT, "include")):
        if name.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", name)).read()
            out |= set(re.findall(r"^\s*(?:int|const char\*)\s+(iga_\w+)\s*\(", txt, re.M))
    return out


def test_exports_every_declared_symbol(capi):
    declared = _declared_symbols()
    assert {"iga_plan", "iga_integrate", "iga_integrate_backward", "iga_destroy"} <= declared
    L = capi.lib()
    for s in sorted(declared):
        assert hasattr(L, s), s
    assert set(capi.EXPORTED) == declared


def test_status_strings(capi):
    for code in range(9):
        s = capi.iga_status_str(code)
        assert s.startswith("IGA_")
    assert "unknown" in capi.iga_status_str(99)


def _desc(capi, dim=3, p=3, q=4, knots=None):
    from paper_2207_00280_gb300 import workloads as wl
    d = capi.PatchDesc()
    p0 = p if np.ndim(p) == 0 else p[0]
    d.dim = dim
    d.set_order(p, q)
    keep = []
    for k in range(dim):
        t = np.ascontiguousarray(knots[k] if knots is not None else wl.open_uniform_knots(4, p0))
        keep.append(t)
        d.n_knots[k] = len(t)
        d.knots[k] = t.ctypes.data
    return d, keep


def _opts(capi, method=1, precision=0, matrices=3):
    o = capi.PlanOpts()
    o.method, o.precision, o.matrices, o.schedule, o.blocking = method, precision, matrices, 0, 1
    return o


def _plan_rc(capi, descs, opts):
    arr = (capi.PatchDesc * len(descs))(*descs)
    h = ctypes.c_void_p()
    info = capi.PlanInfo()
    rc = capi.lib().iga_plan(ctypes.byref(h), arr, len(descs), ctypes.byref(opts), ctypes.byref(info))
    if rc == 0:
        capi.iga_destroy(h)
    return rc


def test_argument_errors(capi):
    L = capi.lib()
    d, keep = _desc(capi)
    arr = (capi.PatchDesc * 1)(d)
    o = _opts(capi)
    assert L.iga_plan(None, arr, 1, ctypes.byref(o), None) == capi.IGA_ERR_ARG
    h = ctypes.c_void_p()
    assert L.iga_plan(ctypes.byref(h), arr, 0, ctypes.byref(o), None) == capi.IGA_ERR_ARG
    assert L.iga_plan(ctypes.byref(h), None, 1, ctypes.byref(o), None) == capi.IGA_ERR_ARG
    assert _plan_rc(capi, [d], _opts(capi, method=7)) == capi.IGA_ERR_ARG
    assert _plan_rc(capi, [d], _opts(capi, precision=9)) == capi.IGA_ERR_ARG
    assert _plan_rc(capi, [d], _opts(capi, matrices=0)) == capi.IGA_ERR_ARG
    # classical is FP64 only
    assert _plan_rc(capi, [d], _opts(capi, method=0, precision=1)) == capi.IGA_ERR_UNSUPPORTED
    assert L.iga_integrate(None, None, None, None, None, None, None, None) == capi.IGA_ERR_ARG
    assert L.iga_integrate_backward(None, None, None, None, None, None, None, None) == capi.IGA_ERR_ARG
    assert L.iga_basis_tables(None, None, None) == capi.IGA_ERR_ARG
    assert L.iga_csr_pattern(None, None, None, None) == capi.IGA_ERR_ARG
    assert L.iga_assemble(None, None, None, None) == capi.IGA_ERR_ARG
    assert L.iga_apply(None, None, None, None, None, 1.0, 0.0, None, None) == capi.IGA_ERR_ARG
    n = ctypes.c_int64()
    assert L.iga_wq_points(None, 0, 0, None, ctypes.byref(n)) == capi.IGA_ERR_ARG
    assert L.iga_wq_mass(None, None, None, None) == capi.IGA_ERR_ARG
    assert L.iga_wq_stiffness(None, None, None, None) == capi.IGA_ERR_ARG
    assert L.iga_integrate_grad(None, None, None, None, None, None, None) == capi.IGA_ERR_ARG
    assert L.iga_destroy(None) == capi.IGA_OK


def test_degree_and_gauss_limits(capi):
    """The boundary's domain: 1 <= p_k <= 8 and 1 <= q_k <= 16 per direction
    (IGA_ERR_ARG outside); FP64 takes every patch inside it, anisotropic ones
    included; FP32/BF16/FP64_DF plans only the (p, q) classes their specialised
    kernels cover."""
    from paper_2207_00280_gb300 import workloads as wl
    ok = (capi.IGA_OK, capi.IGA_ERR_CUDA)   # a valid plan stops at its first CUDA call without a GPU
    for p, q in ((0, 1), (9, 10), (3, 17), (3, 0)):
        pk = max(p, 1)
        d, keep = _desc(capi, p=p, q=q, knots=[wl.open_uniform_knots(4, pk)] * 3)
        assert _plan_rc(capi, [d], _opts(capi)) == capi.IGA_ERR_ARG, (p, q)
    # one direction out of range
    d, keep = _desc(capi, p=(2, 9, 2), q=(3, 10, 3),
                    knots=[wl.open_uniform_knots(3, 2), wl.open_uniform_knots(3, 9), wl.open_uniform_knots(3, 2)])
    assert _plan_rc(capi, [d], _opts(capi)) == capi.IGA_ERR_ARG
    # FP64, classical and sum factorization: p up to 8, q from 1 to 16, a
    # different degree and Gauss order per direction
    for p, q in ((8, 9), (6, 7), (3, 1), (3, 16), (1, 16)):
        d, keep = _desc(capi, p=p, q=q, knots=[wl.open_uniform_knots(2, p)] * 3)
        for method in (0, 1):
            assert _plan_rc(capi, [d], _opts(capi, method=method)) in ok, (p, q, method)
    ps, qs = (1, 4, 8), (2, 7, 16)
    d, keep = _desc(capi, p=ps, q=qs, knots=[wl.open_uniform_knots(2, pk) for pk in ps])
    for method in (0, 1):
        assert _plan_rc(capi, [d], _opts(capi, method=method)) in ok
    d2, keep2 = _desc(capi, dim=2, p=(8, 3), q=(16, 2),
                      knots=[wl.open_uniform_knots(3, 8), wl.open_uniform_knots(3, 3)])
    assert _plan_rc(capi, [d2], _opts(capi)) in ok
    # the low-precision and float-float forms need their specialised kernels
    for prec in (1, 2, 3):
        assert _plan_rc(capi, [d], _opts(capi, precision=prec)) == capi.IGA_ERR_UNSUPPORTED
        d6, keep6 = _desc(capi, p=6, q=7, knots=[wl.open_uniform_knots(2, 6)] * 3)
        assert _plan_rc(capi, [d6], _opts(capi, precision=prec)) == capi.IGA_ERR_UNSUPPORTED
        d3, keep3 = _desc(capi, p=3, q=7)
        assert _plan_rc(capi, [d3], _opts(capi, precision=prec)) == capi.IGA_ERR_UNSUPPORTED


@pytest.mark.parametrize("bad", ["not_open", "decreasing", "multiplicity", "short", "nan", "end_mult"])
def test_knot_errors(capi, bad):
    p = 3
    t = [0.0] * 4 + [0.25, 0.5, 0.75] + [1.0] * 4
    if bad == "not_open":
        t = [0.0, 0.0, 0.0, 0.1] + [0.25, 0.5, 0.75] + [1.0] * 4
    elif bad == "decreasing":
        t = [0.0] * 4 + [0.5, 0.25, 0.75] + [1.0] * 4
    elif bad == "multiplicity":
        t = [0.0] * 4 + [0.5] * 4 + [1.0] * 4
    elif bad == "short":
        t = [0.0] * 4 + [1.0] * 3
    elif bad == "nan":
        t = [0.0] * 4 + [float("nan")] + [1.0] * 4
    elif bad == "end_mult":
        t = [0.0] * 5 + [0.5] + [1.0] * 4
    d, keep = _desc(capi, p=p, q=4, knots=[np.array(t)] * 3)
    assert _plan_rc(capi, [d], _opts(capi)) == capi.IGA_ERR_KNOTS


def test_mixed_dimensions_rejected(capi):
    from paper_2207_00280_gb300 import workloads as wl
    d3, k3 = _desc(capi)
    d2, k2 = _desc(capi, dim=2, p=2, q=3, knots=[wl.open_uniform_knots(4, 2)] * 2)
    assert _plan_rc(capi, [d3, d2], _opts(capi)) == capi.IGA_ERR_UNSUPPORTED


def test_valid_plan_without_gpu_reports_cuda_error(capi):
    """On a machine without a GPU a valid plan stops at the first CUDA call with
    IGA_ERR_CUDA (no crash); with a GPU it succeeds."""
    d, keep = _desc(capi)
    rc = _plan_rc(capi, [d], _opts(capi))
    assert rc in (capi.IGA_OK, capi.IGA_ERR_CUDA)


def test_noalloc_size_limits_on_host(capi):
    """iga_adjoint_noalloc rejects a patch beyond its fixed scratch on the host,
    before any CUDA call: more knots per direction than the scratch holds, more
    elements (p = 1, 70^3 = 343,000 > 262,144), and more basis-table doubles.
    The pointers are never dereferenced on these paths."""
    from paper_2207_00280_gb300 import workloads as wl
    L = capi.lib()
    dummy = ctypes.c_void_p(64)
    cases = [
        ([wl.open_uniform_knots(1100, 3), wl.open_uniform_knots(2, 3), wl.open_uniform_knots(2, 3)], 3, 4),
        ([wl.open_uniform_knots(70, 1)] * 3, 1, 2),
        # 261,820 elements (under the limit) but (1007 + 260 + 1) x 304 = 385,472
        # doubles of degree-8, 16-point basis tables (over the 196,608 limit)
        ([wl.open_uniform_knots(1007, 8), wl.open_uniform_knots(260, 8), wl.open_uniform_knots(1, 8)], 8, 16),
    ]
    for knots, p, q in cases:
        d, keep = _desc(capi, p=p, q=q, knots=knots)
        rc = L.iga_adjoint_noalloc(ctypes.byref(d), dummy, None, dummy, dummy, dummy, None, None)
        assert rc == capi.IGA_ERR_TOO_LARGE, (p, q, rc)
