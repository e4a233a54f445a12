"""Per-operation timing driver: runs one library operation on a standard
workload, times it with CUDA events (L2 flushed before every step) and prints
one JSON line.  Used for profiling single kernels, e.g.

  python opbench.py --op assemble --workload 3d_p3_16 --precision fp32

Operations: integrate (element matrices), assemble (CSR values of the stiffness
from its element matrices, integrated once before timing), apply (y = K x + M x),
adjoint (J and dJ/dkappa) and grad (dL/dkappa, and dL/drho where the workload
has a mass, from random upstream gradients of the element matrices), wq_mass and
wq_stiffness (weighted-quadrature global matrices, lognormal coefficient on the
point grid, FP64).
"""
from __future__ import annotations

import argparse
import json
import statistics

import numpy as np
import torch

from paper_2207_00280_gb300 import workloads as wl
from paper_2207_00280_gb300.plan import IgaPlan, Patch

L2_FLUSH_BYTES = 2 * 129 * 1024 * 1024


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", default="integrate", choices=["integrate", "assemble", "apply", "adjoint", "grad", "wq_mass",
                                                 "wq_stiffness", "probe"])
    ap.add_argument("--workload", default="3d_p3_16")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp64_df", "fp32", "bf16"])
    ap.add_argument("--method", default="sumfact", choices=["sumfact", "classical"])
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    args = ap.parse_args(argv)

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    if args.op == "probe":
        return probe(dev)
    W = wl.WORKLOADS[args.workload]
    sp = W.spec
    G = W.jacobian()
    mass = G is None
    plan = IgaPlan(Patch(sp.knots, sp.p, sp.q), method=args.method, precision=args.precision,
                   mass=mass, stiffness=True, blocking=False)
    kappa = torch.as_tensor(W.kappa(), device=dev)
    jac = torch.as_tensor(np.ascontiguousarray(G), device=dev).reshape(-1) if G is not None else None
    stream = torch.cuda.current_stream(dev)
    K, M, D = plan.empty_outputs(device=dev)
    dt = plan.out_dtype
    if args.op == "integrate":
        def step():
            plan.integrate(kappa=kappa, jac=jac, K=K, M=M, dof=D, stream=stream)
    elif args.op == "assemble":
        plan.integrate(kappa=kappa, jac=jac, K=K, M=M, stream=stream)
        vals = torch.empty(plan.n_csr_nnz, dtype=dt, device=dev)

        def step():
            plan.assemble(K, values=vals, stream=stream)
    elif args.op == "apply":
        del K, M, D
        x = torch.as_tensor(wl.normal(plan.n_dofs, wl.SEED_ADJ_U), device=dev, dtype=dt)
        y = torch.empty_like(x)

        def step():
            plan.apply(x, kappa=kappa, jac=jac, alpha=1.0, beta=1.0, y=y, stream=stream)
    elif args.op in ("wq_mass", "wq_stiffness"):
        del K, M, D
        c = torch.as_tensor(wl.lognormal(plan.wq_grid_size(0), wl.SEED_ADJ_U), device=dev)
        vals = torch.empty(plan.n_csr_nnz, dtype=torch.float64, device=dev)
        fn = plan.wq_mass if args.op == "wq_mass" else plan.wq_stiffness

        def step():
            fn(c=c, values=vals, stream=stream)
    elif args.op == "grad":
        del D
        gen = torch.Generator(device=dev).manual_seed(wl.SEED_ADJ_U)
        GK = torch.randn(K.numel(), dtype=dt, device=dev, generator=gen)
        GM = torch.randn(M.numel(), dtype=dt, device=dev, generator=gen) if M is not None else None
        del K, M
        gk = torch.empty(plan.n_qp, dtype=dt, device=dev)
        gr = torch.empty(plan.n_qp, dtype=dt, device=dev) if GM is not None else None

        def step():
            plan.integrate_grad(GK=GK, GM=GM, jac=jac, grad_kappa=gk, grad_rho=gr, stream=stream)
    else:
        del K, M, D
        u = torch.as_tensor(wl.normal(plan.n_dofs, wl.SEED_ADJ_U), device=dev, dtype=dt)
        v = torch.as_tensor(wl.normal(plan.n_dofs, wl.SEED_ADJ_V), device=dev, dtype=dt)
        g = torch.empty(plan.n_qp, dtype=dt, device=dev)
        J = torch.empty(1, dtype=torch.float64, device=dev)

        def step():
            plan.backward(kappa, u, v, grad=g, J=J, jac=jac, stream=stream)

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(max(1, args.warmup)):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize(dev)
    ts = []
    for i in range(args.steps):
        flush.fill_(float(i))
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    print(json.dumps({"op": args.op, "workload": args.workload, "precision": args.precision,
                      "method": args.method, "elements": sp.E, "steps": args.steps,
                      "ms_median": round(statistics.median(ts), 4),
                      "ms_min": round(min(ts), 4)}), flush=True)
    plan.close()


def probe(dev):
    """Arithmetic rates of this GPU (include/iga_probe.h): DFMA, DMMA (mma.sync
    m8n8k4 f64) and FFMA throughput for 1, 2, 4 and 8 CTAs of 256 threads per
    SM, best of three CUDA-event timings each, in TFLOP/s."""
    import ctypes
    from paper_2207_00280_gb300 import capi
    st = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    out = {}
    for name, kind, iters in (("dfma", capi.IGA_PROBE_DFMA, 1 << 16),
                              ("dmma", capi.IGA_PROBE_DMMA, 1 << 14),
                              ("ffma", capi.IGA_PROBE_FFMA, 1 << 20)):
        capi.iga_probe_rate(kind, 1024, 1, st)   # warm-up
        for ctas in (1, 2, 4, 8):
            best, ms_b = 0.0, 0.0
            for _ in range(3):
                ms, fl = capi.iga_probe_rate(kind, iters, ctas, st)
                if fl / (ms * 1e-3) / 1e12 > best:
                    best, ms_b = fl / (ms * 1e-3) / 1e12, ms
            out[f"{name}_ctas{ctas}"] = {"tflops": round(best, 4), "ms": round(ms_b, 3)}
    print(json.dumps({"op": "probe", "rates": out}), flush=True)


if __name__ == "__main__":
    main()
