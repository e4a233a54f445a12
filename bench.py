#!/usr/bin/env python
"""Benchmark: batched IGA-FEM element-matrix integration on GB300.

Default workload: 3D, p=3, 32^3 elements, 4^3 Gauss points, lognormal(0,0.5)
kappa (seed 2207), identity geometry, FP64 sum factorization producing the
stiffness and mass element matrices (64x64 each) and the dof map.  A step is
one iga_integrate call (Cox--de Boor tables, dof map, element matrices) with
inputs resident in HBM.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--method sumfact|classical] [--precision fp64|fp32|bf16]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3D p=3 element matrices/s, sumfact vs classical, FP64 vs FP32/BF16 at stated err"
UNIT = "element matrices/s (one K_e and one M_e per element)"
L2_BYTES = 129 * 1024 * 1024

# FP64 issue rate of the GB300 CUDA cores used for the FP64 roofline: DFMA per
# SM per clock (2 flops each), so the peak is 152 SMs x 2 x 2 flops x the SM
# clock (1.2586 TFLOP/s at 2070 MHz).  The FP64 sum-factorization kernel keeps
# its FP64 pipe ~94% active (ncu) at this rate.
DFMA_PER_SM_CLK = 2.0
N_SM = 152
# FP32 operations of one float-float multiply-add (product with its exact
# error, two-sum, renormalisation); the float-float roofline divides the FP32
# issue rate by this count.
DF_OPS_PER_FMA = 14


def flops_per_element(dim, p, q, stiffness, mass, general_geometry):
    """Algorithmic flops of sum factorization per element (multiply-add = 2),
    last stage over the symmetric half S = N(N+1)/2.  General geometry: all d^2
    stiffness terms; identity geometry: the d diagonal terms only (the
    off-diagonal coefficients vanish identically)."""
    n, N = p + 1, (p + 1) ** dim
    S = N * (N + 1) // 2
    terms = dim * dim if general_geometry else dim
    f = 0
    if dim == 3:
        if stiffness:
            f += 2 * terms * (n * n * q ** 3 + n ** 4 * q * q) + (8 if general_geometry else 4) * q * S
        if mass:
            f += 2 * n * n * q ** 3 + 2 * n ** 4 * q * q + 2 * q * S
    else:
        if stiffness:
            f += 2 * terms * n * n * q * q + (8 if general_geometry else 4) * q * S
        if mass:
            f += 2 * n * n * q * q + 2 * q * S
    return f


def classical_flops_per_element(dim, p, q, stiffness, mass):
    N, Q = (p + 1) ** dim, q ** dim
    S = N * (N + 1) // 2
    return 2 * S * Q * ((dim if stiffness else 0) + (1 if mass else 0))


def bytes_per_element(dim, p, q, esize, stiffness, mass, general_geometry, dof=True):
    N, Q = (p + 1) ** dim, q ** dim
    b = N * N * esize * (int(stiffness) + int(mass)) + 8 * Q
    if general_geometry:
        b += 8 * Q * dim * dim
    if dof:
        b += 4 * N
    return b


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def fp_rate_probe(stream_ptr):
    """Measured arithmetic rates of this GPU (include/iga_probe.h): FP64 FMA on
    the CUDA cores, FP64 MMA (mma.sync m8n8k4) and FP32 FMA, each a ~0.1-0.3 s
    kernel over all SMs, best of three.  The FP64 kernels of this library are
    bound by the first; the second is the FP64 tensor path they do not use."""
    from paper_2207_00280_gb300 import capi
    out = {}
    for name, kind, iters in (("dfma", capi.IGA_PROBE_DFMA, 1 << 16),
                              ("dmma", capi.IGA_PROBE_DMMA, 1 << 14),
                              ("ffma", capi.IGA_PROBE_FFMA, 1 << 20)):
        best = 0.0
        for ctas in (2, 4):
            for _ in range(3):
                ms, fl = capi.iga_probe_rate(kind, iters, ctas, stream_ptr)
                best = max(best, fl / (ms * 1e-3) / 1e12)
        out[f"{name}_tflops"] = round(best, 4)
    out["how"] = ("iga_probe_rate: independent FMA chains (8 per thread) or MMA "
                  "accumulators (4 per warp), 2 and 4 CTAs of 256 threads per SM, best of 3 "
                  "CUDA-event timings each")
    return out


def cpu_model():
    """CPU model name of this host (lscpu, else /proc/cpuinfo)."""
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for ln in r.stdout.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in a thread."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_id_for_smi(local):
    """nvidia-smi -i accepts a UUID; fall back to the local index."""
    try:
        import torch
        u = torch.cuda.get_device_properties(local).uuid
        u = str(u)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(local)


def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws, device="cuda"):
    """Max of a per-rank scalar over all ranks (the timed region's duration)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(ws, units_per_rank, steps, max_ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return ws * units_per_rank * steps / (max_ms / 1e3)


def cpu_baseline_oracle(workload, budget_s=12.0, method="sumfact", max_elems=None, threads=1):
    """Time the FP64 oracle (as it stands) on a bounded sample of the workload's
    elements; returns elements/s, the elements done and the seconds taken.
    threads > 1 runs chunks of elements concurrently on that many host threads
    (the oracle has no global state and ctypes releases the GIL during its
    calls), the over-elements parallelism of the paper's OpenMP runs."""
    import concurrent.futures as cf
    import numpy as np
    import oracle
    from paper_2207_00280_gb300 import workloads as wl
    W = wl.WORKLOADS[workload]
    sp = W.spec
    P = oracle.Patch(sp.knots, sp.p, sp.q)
    kappa = W.kappa()
    G = W.jacobian()
    fn = P.sumfact if method == "sumfact" else P.classical
    rng = np.random.default_rng(2207)
    order = rng.permutation(sp.E)
    chunk = 64 if method == "sumfact" else 8
    limit = max_elems or sp.E
    done, t0 = 0, time.perf_counter()
    if threads <= 1:
        while done < limit and time.perf_counter() - t0 < budget_s:
            el = order[done:done + chunk]
            fn(el, kappa=kappa, G=G, stiffness=True, mass=G is None)
            done += len(el)
        return done / (time.perf_counter() - t0), done, time.perf_counter() - t0
    lock = threading.Lock()
    state = {"next": 0, "done": 0}

    def worker():
        while time.perf_counter() - t0 < budget_s:
            with lock:
                a = state["next"]
                if a >= limit:
                    return
                state["next"] = a + chunk
            el = order[a:a + chunk]
            fn(el, kappa=kappa, G=G, stiffness=True, mass=G is None)
            with lock:
                state["done"] += len(el)

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        futs = [ex.submit(worker) for _ in range(threads)]
        for f in futs:
            f.result()
    dt = time.perf_counter() - t0
    return state["done"] / dt, state["done"], dt


def cpu_baselines(workload, E, seconds):
    """The oracle's Algorithm 2 (sum factorization) and Algorithm 1 (classical)
    on one host thread and on every host core, each on a bounded seeded sample
    of the workload's elements."""
    cores = os.cpu_count() or 1
    res = {}
    for meth in ("sumfact", "classical"):
        for th in (1, cores):
            rate, done, dt = cpu_baseline_oracle(workload, budget_s=seconds, method=meth,
                                                 threads=th)
            res[f"{meth}_{'1_thread' if th == 1 else 'all_cores'}"] = {
                "value": round(rate, 2), "threads": th, "elements": done, "seconds": round(dt, 2)}
    return res, cores


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch
    from paper_2207_00280_gb300 import workloads as wl
    from paper_2207_00280_gb300.plan import IgaPlan, Patch

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    W = wl.WORKLOADS[args.workload]
    sp = W.spec
    G = W.jacobian()
    general = G is not None
    mass = not general   # the curved workload integrates the stiffness only
    plan = IgaPlan(Patch(sp.knots, sp.p, sp.q), method=args.method, precision=args.precision,
                   mass=mass, stiffness=True, blocking=False, profile=True)
    kappa_h = torch.from_numpy(W.kappa())
    kappa = kappa_h.to(dev)
    jac = torch.from_numpy(np.ascontiguousarray(G)).reshape(-1).to(dev) if general else None
    K, M, D = plan.empty_outputs(device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.integrate(kappa=kappa, jac=jac, K=K, M=M, dof=D, stream=stream)

    # measured FP64/FP32 rates of this GPU, before the warm-up (a few seconds)
    import ctypes
    probe = fp_rate_probe(ctypes.c_void_p(stream.cuda_stream)) if args.probe else None

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize(dev)
    plan.profile_read()  # reset the kernel counters

    sampler = ClockSampler(gpu_id_for_smi(local))
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize(dev)
    sampler.start()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))          # L2 flush, outside the step's events
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize(dev)
    barrier(ws)
    t_wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    kern_ms, launches = plan.profile_read()
    total_ms = max_over_ranks(sum(step_ms), ws)
    E = sp.E
    value = weak_scaling_value(ws, E, args.steps, total_ms)

    # roofline of the dominant kernel (the element-matrix kernel)
    esize = 8 if args.precision in ("fp64", "fp64_df") else 4
    peaks, peak_src = measured_peaks()
    launch_ms = kern_ms / max(1, launches)
    if args.method == "sumfact":
        f_el = flops_per_element(3 if len(sp.knots) == 3 else 2, sp.p, sp.q, True, mass, general)
    else:
        f_el = classical_flops_per_element(len(sp.knots), sp.p, sp.q, True, mass)
    b_el = bytes_per_element(len(sp.knots), sp.p, sp.q, esize, True, mass, general, dof=False)
    if args.precision in ("fp64", "fp64_df"):
        if args.precision == "fp64":
            peak_tf = N_SM * DFMA_PER_SM_CLK * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            src = (f"FP64 CUDA cores: {N_SM} SMs x {DFMA_PER_SM_CLK:g} DFMA/clk x 2 x "
                   f"{peaks.get('sm_max_mhz', 2070.0):g} MHz")
        else:
            # float-float: one FP64-equivalent multiply-add = DF_OPS_PER_FMA FP32 operations
            peak_tf = (N_SM * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / DF_OPS_PER_FMA * 2) / 1e12
            src = (f"FP32 pipes: {N_SM} SMs x 128 lanes x {peaks.get('sm_max_mhz', 2070.0):g} MHz / "
                   f"{DF_OPS_PER_FMA} FP32 ops per float-float multiply-add x 2 flops")
        achieved = f_el * E / (launch_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak_tf, 4),
                "unit": "TFLOP/s", "frac": round(achieved / peak_tf, 4),
                "traffic": None,
                "flop_per_element": f_el, "elements_per_launch": E,
                "launch_ms": round(launch_ms, 4),
                "peak_source": src,
                "hbm_frac": round(b_el * E / (launch_ms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4),
                "hbm_peak_gbs": peaks["hbm_gbs"], "hbm_peak_source": peak_src}
        if args.method == "sumfact" and not general:
            # the same time under the count of all d^2 stiffness terms (the
            # off-diagonal ones are identically zero for the identity map)
            f_gen = flops_per_element(len(sp.knots), sp.p, sp.q, True, mass, True)
            roof["flop_per_element_all_terms"] = f_gen
            roof["frac_all_terms"] = round(f_gen * E / (launch_ms * 1e-3) / 1e12 / peak_tf, 4)
        if probe and args.precision == "fp64":
            roof["measured_dfma_tflops"] = probe["dfma_tflops"]
            roof["frac_of_measured_dfma"] = round(achieved / probe["dfma_tflops"], 4)
            roof["measured_dmma_tflops"] = probe["dmma_tflops"]
    else:
        ach = b_el * E / (launch_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(ach / peaks["hbm_gbs"], 4), "traffic": None,
                "bytes_per_element": b_el, "elements_per_launch": E,
                "launch_ms": round(launch_ms, 4), "peak_source": peak_src}
    tr = traffic_from_profiles(args, esize)
    if tr is not None:
        roof["traffic"] = tr

    # the other forms the metric compares, on the same GPU
    forms = {}
    if args.compare and rank == 0:
        forms = measure_forms(args, W, kappa, jac, mass, flush, stream, dev,
                              total_ms / args.steps)

    # end to end through the public API with host buffers: H2D of kappa (and the
    # Jacobian), the integration, D2H of the element matrices and the dof map.
    # Serial: every step's copies follow its integration on one stream.
    # Pipelined (the reported value): two sets of device outputs and a copy
    # stream, so that step i's D2H overlaps step i+1's integration, as a serving
    # loop would run it; every step still moves all of its bytes to the host.
    e2e = None
    if args.e2e:
        kap_pin = kappa_h.pin_memory()
        jac_pin = torch.from_numpy(np.ascontiguousarray(G)).reshape(-1).pin_memory() if general else None
        h2d = kap_pin.numel() * 8 + (jac_pin.numel() * 8 if general else 0)
        d2h = sum(t.numel() * t.element_size() for t in (K, M, D) if t is not None)
        n_e2e = max(2, min(args.steps, 5))
        # two sets of device outputs, one set of pinned host buffers: the copy
        # stream serialises the D2H copies, so each step's result lands in the
        # same host memory (a second 2 GB pinned set measured as slow as 42 GB/s
        # on one box, against 186 GB/s for the first)
        dev_sets = [(K, M, D), plan.empty_outputs(device=dev)]
        host_set = [torch.empty(t.numel(), dtype=t.dtype).pin_memory() if t is not None else None
                    for t in (K, M, D)]
        host_sets = [host_set, host_set]
        copy_stream = torch.cuda.Stream(dev)
        comp_done = [torch.cuda.Event() for _ in range(2)]
        copy_done = [torch.cuda.Event() for _ in range(2)]

        def e2e_inputs():
            kappa.copy_(kap_pin, non_blocking=True)
            if general:
                jac.copy_(jac_pin, non_blocking=True)

        def e2e_serial():
            e2e_inputs()
            Ks, Ms, Ds = dev_sets[0]
            plan.integrate(kappa=kappa, jac=jac, K=Ks, M=Ms, dof=Ds, stream=stream)
            for th, td in zip(host_sets[0], dev_sets[0]):
                if td is not None:
                    th.copy_(td, non_blocking=True)

        def e2e_pipelined(i):
            j = i % 2
            stream.wait_event(copy_done[j])      # the set's previous D2H is done
            e2e_inputs()
            Ks, Ms, Ds = dev_sets[j]
            plan.integrate(kappa=kappa, jac=jac, K=Ks, M=Ms, dof=Ds, stream=stream)
            comp_done[j].record(stream)
            copy_stream.wait_event(comp_done[j])
            with torch.cuda.stream(copy_stream):
                for th, td in zip(host_sets[j], dev_sets[j]):
                    if td is not None:
                        th.copy_(td, non_blocking=True)
            copy_done[j].record(copy_stream)

        def timed(run):
            torch.cuda.synchronize(dev)
            barrier(ws)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for i in range(n_e2e):
                run(i)
            stream.wait_stream(copy_stream)
            b.record(stream)
            b.synchronize()
            barrier(ws)
            return max_over_ranks(a.elapsed_time(b), ws)

        for j in range(2):
            copy_done[j].record(copy_stream)
        e2e_serial()
        e2e_pipelined(0)
        e2e_pipelined(1)
        # three alternating repeats of each loop, the median reported: the link
        # to host memory is shared with the node's other GPUs, and one loop of a
        # pair has measured 66 GB/s while the other measured 186 GB/s
        s_rep, e_rep = [], []
        for _ in range(3):
            s_rep.append(timed(lambda i: e2e_serial()))
            e_rep.append(timed(e2e_pipelined))
        s_ms = sorted(s_rep)[1]
        e_ms = sorted(e_rep)[1]
        torch.cuda.synchronize(dev)
        ok = all(torch.equal(th[:4096], td[:4096].cpu()) for th, td in zip(host_sets[1], dev_sets[1])
                 if td is not None)
        e2e = {"value": round(ws * E * n_e2e / (e_ms * 1e-3), 1), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": n_e2e,
               "ms_per_step": round(e_ms / n_e2e, 4),
               "pipelined": "D2H of step i on a copy stream overlaps the integration of step i+1",
               "serial_ms_per_step": round(s_ms / n_e2e, 4),
               "serial_value": round(ws * E * n_e2e / (s_ms * 1e-3), 1),
               "d2h_gbs": round(d2h * n_e2e / (e_ms * 1e-3) / 1e9, 1),
               "repeats_ms_per_step": {"pipelined": [round(x / n_e2e, 3) for x in e_rep],
                                       "serial": [round(x / n_e2e, 3) for x in s_rep],
                                       "reported": "median of the three"},
               "host_copy_checked": ok}
        del dev_sets, host_sets

    cpu = None
    if args.cpu_baseline and rank == 0 and ws == 1:
        per, cores = cpu_baselines(args.workload, E, args.cpu_seconds / 4)
        key = ("sumfact" if args.method == "sumfact" else "classical") + "_all_cores"
        cpu = {"value": per[key]["value"], "unit": UNIT, "cores": cores, "kind": "oracle",
               "cpu_model": cpu_model(),
               "sample": (f"{per[key]['elements']} of {E} elements (seeded permutation), FP64 oracle "
                          f"{'Algorithm 2 sum factorization' if args.method == 'sumfact' else 'Algorithm 1 classical'}"
                          f", chunks of elements on {cores} host threads, {per[key]['seconds']} s"),
               "runs": per,
               "note": "each run: a bounded seeded sample of the workload's elements; elements/s"}

    n_kernels_per_step = 3  # basis tables, dof map, element matrices
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp64_df": "f32x2 (float-float, FP64-accurate)", "fp32": "f32",
                  "bf16": "bf16"}[args.precision],
        "data": "synthetic (seeded lognormal kappa, open uniform knots)",
        "config": {"workload": args.workload, "dim": len(sp.knots), "degree": sp.p,
                   "elements": E, "gauss_per_dir": sp.q, "method": args.method,
                   "precision": args.precision, "matrices": "stiffness+mass" if mass else "stiffness",
                   "geometry": "curved" if general else "identity",
                   "l2": "flushed before every step (256 MiB write outside the step's events)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "clocks": clocks, "e2e": e2e, "gpu_launches": n_kernels_per_step * args.steps,
        "roofline": roof, "cpu_baseline": cpu, "forms": forms or None,
        "fp_rate_probe": probe,
        "wall_s_timed_region": round(t_wall, 4),
        "kernel_ms_per_launch": round(launch_ms, 4),
    }
    plan.close()
    return line


def _time_steps(fn, steps, stream, flush):
    """Median per-step device time (ms) of fn, L2 flushed before each step."""
    import torch
    fn()
    fn()
    ts = []
    for _ in range(steps):
        flush.fill_(3.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def _graph_us_per_step(fn, dev, reps=50):
    """Device time per step of fn captured in a CUDA graph and replayed reps
    times back to back (the launch-latency form of a small workload)."""
    import torch
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        fn()
    torch.cuda.current_stream(dev).wait_stream(side)
    torch.cuda.synchronize(dev)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    g.replay()
    torch.cuda.synchronize(dev)
    st = torch.cuda.current_stream(dev)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(reps):
        g.replay()
    b.record(st)
    b.synchronize()
    return a.elapsed_time(b) * 1e3 / reps


# error levels against the FP64 oracle (per-element relative Frobenius): the
# tolerances the GPU tests enforce and the worst errors they measured
FORM_ERR = {
    "sumfact_fp64": {"tolerance": 1e-12},
    "classical_fp64": {"tolerance": 1e-12},
    "sumfact_fp32": {"tolerance": 1e-5},
    "sumfact_bf16": {"tolerance": 5e-3},
    "sumfact_fp64_df": {"tolerance": 1e-12},
}


def measure_forms(args, W, kappa, jac, mass, flush, stream, dev, main_ms):
    """Time the other forms of the metric on the same GPU: FP64 classical,
    FP32/BF16 sum factorization of the same workload, the 64-patch batch
    (persistent CUDA graph vs per-patch launches) and the adjoint."""
    import numpy as np
    import torch
    from paper_2207_00280_gb300 import capi
    from paper_2207_00280_gb300 import workloads as wl
    from paper_2207_00280_gb300.plan import IgaPlan, Patch
    sp = W.spec
    E = sp.E
    forms = {f"{args.method}_{args.precision}": {"ms_per_step": round(main_ms, 4),
                                                 "value": round(E / (main_ms * 1e-3), 1),
                                                 **FORM_ERR.get(f"{args.method}_{args.precision}", {})}}
    variants = [("classical", "fp64")]
    if args.method == "sumfact":
        variants += [("sumfact", pr) for pr in ("fp64", "fp64_df", "fp32", "bf16")
                     if pr != args.precision]
    for meth, pr in variants:
        key = f"{meth}_{pr}"
        try:
            pl = IgaPlan(Patch(sp.knots, sp.p, sp.q), method=meth, precision=pr, mass=mass,
                         stiffness=True, blocking=False)
        except capi.IgaError as ex:
            forms[key] = {"unavailable": str(ex)}
            continue
        K2, M2, _ = pl.empty_outputs(device=dev, dof=False)
        ms = _time_steps(lambda: pl.integrate(kappa=kappa, jac=jac, K=K2, M=M2, stream=stream),
                         3 if meth == "classical" else 5, stream, flush)
        forms[key] = {"ms_per_step": round(ms, 4), "value": round(E / (ms * 1e-3), 1), **FORM_ERR.get(key, {})}
        del K2, M2
        pl.close()
        torch.cuda.empty_cache()
    if "classical_fp64" in forms and "ms_per_step" in forms["classical_fp64"]:
        base = forms["classical_fp64"]["ms_per_step"]
        for k, v in forms.items():
            if "ms_per_step" in v:
                v["speedup_vs_classical_fp64"] = round(base / v["ms_per_step"], 3)
    if not args.extra_forms:
        return forms
    forms["3d_p4_48_curved"] = measure_curved_p4(stream, flush, dev)
    forms["3d_p8_8"] = measure_high_degree(stream, flush, dev)
    # 2D p=2 16x16 (256 elements, kappa = 1): launch-latency bound, reported in microseconds
    W2 = wl.WORKLOADS["2d_p2_16"]
    s2 = W2.spec
    small = {"elements": s2.E}
    for meth in ("sumfact", "classical"):
        pl = IgaPlan(Patch(s2.knots, s2.p, s2.q), method=meth, precision="fp64", blocking=False)
        K2, M2, D2 = pl.empty_outputs(device=dev)
        ms = _time_steps(lambda: pl.integrate(K=K2, M=M2, dof=D2, stream=stream), 20, stream, flush)
        small[f"{meth}_fp64_us_per_step"] = round(ms * 1e3, 2)
        small[f"{meth}_fp64_graph_us_per_step"] = round(
            _graph_us_per_step(lambda: pl.integrate(K=K2, M=M2, dof=D2), dev), 2)
        pl.close()
    small["note"] = ("us_per_step: each call through the Python binding, host launch overhead "
                     "included; graph_us_per_step: the same three launches (tables, dof map, "
                     "element kernel) captured once in a CUDA graph and replayed back to back")
    forms["2d_p2_16"] = small
    # 64-patch mixed batch, FP32 mass + stiffness: one persistent graph vs per-patch launches
    specs = wl.batch_specs()
    nqp = sum(s.E * s.Q for s in specs)
    kb = torch.as_tensor(wl.lognormal(nqp, wl.SEED_BATCH_KAPPA), device=dev)
    Eb = sum(s.E for s in specs)
    batch = {"patches": len(specs), "elements": Eb}
    for name, sched in (("per_patch", capi.IGA_SCHED_PER_PATCH),
                        ("persistent_graph_autotuned", capi.IGA_SCHED_AUTO)):
        pl = IgaPlan([Patch(s.knots, s.p, s.q) for s in specs], method="sumfact", precision="fp32",
                     schedule=sched, blocking=False)
        Kb, Mb, Db = pl.empty_outputs(device=dev)
        ms = _time_steps(lambda: pl.integrate(kappa=kb, K=Kb, M=Mb, dof=Db, stream=stream), 5,
                         stream, flush)
        batch[name] = {"ms_per_step": round(ms, 4), "value": round(Eb / (ms * 1e-3), 1)}
        out_bytes = 2 * Kb.numel() * 4 + Db.numel() * 4 + nqp * 8
        batch[name]["hbm_frac"] = round(out_bytes / (ms * 1e-3) / 1e9 / measured_peaks()[0]["hbm_gbs"], 4)
        del Kb, Mb, Db
        pl.close()
        torch.cuda.empty_cache()
    batch["speedup_graph_vs_per_patch"] = round(batch["per_patch"]["ms_per_step"] /
                                                batch["persistent_graph_autotuned"]["ms_per_step"], 3)
    batch["autotuned_schedules"] = autotune_table()
    forms["batch_64_patches_fp32"] = batch
    # adjoint: J = u^T K(kappa) v and dJ/dkappa, 40^3 p=3
    A = wl.WORKLOADS["3d_p3_40_adjoint"]
    sa = A.spec
    ka = torch.as_tensor(A.kappa(), device=dev)
    adj = {"elements": sa.E, "qp": sa.E * sa.Q}
    for pr, dt in (("fp64", torch.float64), ("fp64_df", torch.float64), ("fp32", torch.float32)):
        pl = IgaPlan(Patch(sa.knots, sa.p, sa.q), method="sumfact", precision=pr, blocking=False)
        u = torch.as_tensor(wl.normal(sa.n_dofs, wl.SEED_ADJ_U), device=dev, dtype=dt)
        v = torch.as_tensor(wl.normal(sa.n_dofs, wl.SEED_ADJ_V), device=dev, dtype=dt)
        g = torch.empty(pl.n_qp, dtype=dt, device=dev)
        J = torch.empty(1, dtype=torch.float64, device=dev)
        ms = _time_steps(lambda: pl.backward(ka, u, v, grad=g, J=J, stream=stream), 5, stream, flush)
        adj[pr] = {"ms_per_step": round(ms, 4), "qp_per_s": round(sa.E * sa.Q / (ms * 1e-3), 1)}
        pl.close()
    forms["adjoint_3d_p3_40"] = adj
    forms["apply_3d_p3_40"] = measure_apply(A, ka, stream, flush, dev)
    forms["assembly_3d_p3_32"] = measure_assembly(W, kappa, stream, flush, dev)
    forms["wq_mass_3d_p3_32"] = measure_wq(W, stream, flush, dev)
    forms["grad_3d_p3_32"] = measure_grad(W, stream, flush, dev)
    return forms


def measure_curved_p4(stream, flush, dev):
    """3D p=4, 48^3 elements, 5^3 Gauss points, the curved map, seeded lognormal
    kappa: the stiffness by sum factorization in FP64, float-float (FP64_DF
    plan), FP32 and BF16, and by FP64 classical integration.  Each form gets its
    step time, the element kernel's own time (CUDA events around it), its
    roofline fraction (FP64 issue rate for FP64 and classical, the float-float
    rate for FP64_DF, HBM for FP32/BF16, whose bytes are the output) and its
    speed-up over FP64 classical."""
    import numpy as np
    import torch
    from paper_2207_00280_gb300 import workloads as wl
    from paper_2207_00280_gb300.plan import IgaPlan, Patch
    W3 = wl.WORKLOADS["3d_p4_48_curved"]
    sp = W3.spec
    E = sp.E
    kappa = torch.as_tensor(W3.kappa(), device=dev)
    jac = torch.as_tensor(np.ascontiguousarray(W3.jacobian()), device=dev).reshape(-1)
    peaks = measured_peaks()[0]
    mhz = peaks.get("sm_max_mhz", 2070.0)
    fp64_peak = N_SM * DFMA_PER_SM_CLK * 2 * mhz * 1e6
    df_peak = N_SM * 128 * mhz * 1e6 / DF_OPS_PER_FMA * 2
    f_sf = flops_per_element(3, sp.p, sp.q, True, False, True)
    f_cl = classical_flops_per_element(3, sp.p, sp.q, True, False)
    out = {"elements": E, "degree": sp.p, "gauss_per_dir": sp.q, "geometry": "curved",
           "matrices": "stiffness", "flop_per_element_sumfact": f_sf,
           "flop_per_element_classical": f_cl}
    for meth, pr in (("classical", "fp64"), ("sumfact", "fp64"), ("sumfact", "fp64_df"),
                     ("sumfact", "fp32"), ("sumfact", "bf16")):
        key = f"{meth}_{pr}"
        pl = IgaPlan(Patch(sp.knots, sp.p, sp.q), method=meth, precision=pr, mass=False,
                     stiffness=True, blocking=False, profile=True)
        K, _, _ = pl.empty_outputs(device=dev, dof=False)
        pl.integrate(kappa=kappa, jac=jac, K=K, stream=stream)
        torch.cuda.synchronize(dev)
        pl.profile_read()
        ms = _time_steps(lambda: pl.integrate(kappa=kappa, jac=jac, K=K, stream=stream),
                         3 if meth == "classical" else 5, stream, flush)
        kern_ms, launches = pl.profile_read()
        kms = kern_ms / max(1, launches)
        esz = 8 if pr in ("fp64", "fp64_df") else 4
        b_el = bytes_per_element(3, sp.p, sp.q, esz, True, False, True, dof=False)
        ent = {"ms_per_step": round(ms, 4), "kernel_ms": round(kms, 4),
               "value": round(E / (ms * 1e-3), 1),
               "hbm_frac": round(b_el * E / (kms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4),
               "bytes_per_element": b_el, **FORM_ERR.get(key, {})}
        f_el = f_cl if meth == "classical" else f_sf
        if pr == "fp64":
            ent["fp64_frac"] = round(f_el * E / (kms * 1e-3) / fp64_peak, 4)
        elif pr == "fp64_df":
            ent["float_float_frac"] = round(f_el * E / (kms * 1e-3) / df_peak, 4)
        ent["roofline_frac"] = ent.get("fp64_frac", ent.get("float_float_frac", ent["hbm_frac"]))
        out[key] = ent
        del K
        pl.close()
        torch.cuda.empty_cache()
    base = out["classical_fp64"]["ms_per_step"]
    for k, v in out.items():
        if isinstance(v, dict) and "ms_per_step" in v:
            v["speedup_vs_classical_fp64"] = round(base / v["ms_per_step"], 3)
    return out


def measure_high_degree(stream, flush, dev):
    """3D p=8, 8^3 elements, 9^3 Gauss points, lognormal kappa, identity map:
    mass and stiffness (729 x 729 per element) by sum factorization and by
    classical integration, FP64, on the runtime-sized kernels.  Each form with
    its FP64 fraction (algorithmic flops over the element kernel's time) and
    the speed-up of sum factorization over the classical loop."""
    import torch
    from paper_2207_00280_gb300 import workloads as wl
    from paper_2207_00280_gb300.plan import IgaPlan, Patch
    W8 = wl.WORKLOADS["3d_p8_8"]
    sp = W8.spec
    E = sp.E
    kappa = torch.as_tensor(W8.kappa(), device=dev)
    peaks = measured_peaks()[0]
    fp64_peak = N_SM * DFMA_PER_SM_CLK * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6
    out = {"elements": E, "degree": sp.p, "gauss_per_dir": sp.q, "matrices": "stiffness+mass",
           "geometry": "identity"}
    for meth in ("sumfact", "classical"):
        pl = IgaPlan(Patch(sp.knots, sp.p, sp.q), method=meth, precision="fp64", blocking=False,
                     profile=True)
        K, M, _ = pl.empty_outputs(device=dev, dof=False)
        pl.integrate(kappa=kappa, K=K, M=M, stream=stream)
        torch.cuda.synchronize(dev)
        pl.profile_read()
        ms = _time_steps(lambda: pl.integrate(kappa=kappa, K=K, M=M, stream=stream),
                         1 if meth == "classical" else 3, stream, flush)
        kern_ms, launches = pl.profile_read()
        kms = kern_ms / max(1, launches)
        f_el = (flops_per_element(3, sp.p, sp.q, True, True, False) if meth == "sumfact"
                else classical_flops_per_element(3, sp.p, sp.q, True, True))
        out[f"{meth}_fp64"] = {"ms_per_step": round(ms, 4), "kernel_ms": round(kms, 4),
                               "value": round(E / (ms * 1e-3), 1), "flop_per_element": f_el,
                               "fp64_frac": round(f_el * E / (kms * 1e-3) / fp64_peak, 4),
                               **FORM_ERR.get(f"{meth}_fp64", {})}
        del K, M
        pl.close()
        torch.cuda.empty_cache()
    out["speedup_sumfact_vs_classical"] = round(out["classical_fp64"]["ms_per_step"] /
                                                out["sumfact_fp64"]["ms_per_step"], 2)
    return out


SCHED_NAMES = {0: "cta", 4: "cta_other_stage3_form", 8: "cta_other_size", 16: "warp_per_element"}


def autotune_table():
    """The batch autotuner's choices, read back from its cache file: per (p, q)
    class the schedule and the elements per work item."""
    path = os.environ.get("IGA_AUTOTUNE_CACHE")
    try:
        with open(path) as f:
            tab = json.load(f)
    except Exception:
        return None
    out = {}
    for k, v in tab.items():
        parts = k.split("/")
        try:
            i = parts.index("sf3v2")
        except ValueError:
            continue
        cls = "/".join(parts[i + 1:])
        out[cls] = {"schedule": SCHED_NAMES.get(v // 100, str(v // 100)), "elements_per_item": v % 100}
    return out


def wq_flops(knots, p, xs, stiffness=False):
    """Algorithmic flops of the weighted-quadrature mass, row by row: for row
    i with n_k support points and w_k coupled functions per direction,
    2 (w3 n1 n2 n3 + w2 w3 n1 n2 + w1 w2 w3 n1); the stiffness contracts two
    tables in z, three products in y and two in x:
    2 (2 w3 n1 n2 n3 + 3 w2 w3 n1 n2 + 2 w1 w2 w3 n1)."""
    import numpy as np
    per_dir = []
    for t, x in zip(knots, xs):
        nf = len(t) - p - 1
        n = np.array([np.count_nonzero((x >= t[i]) & (x <= t[i + p + 1])) for i in range(nf)])
        lo = np.array([max(0, i - p) for i in range(nf)])
        hi = np.array([min(nf - 1, i + p) for i in range(nf)])
        per_dir.append((n.astype(float), (hi - lo + 1).astype(float)))
    (n1, w1), (n2, w2), (n3, w3) = per_dir
    N1, N2, N3 = np.meshgrid(n1, n2, n3, indexing="ij")
    W1, W2, W3 = np.meshgrid(w1, w2, w3, indexing="ij")
    a, b = (2, 3) if stiffness else (1, 1)
    return float(2 * (a * W3 * N1 * N2 * N3 + b * W2 * W3 * N1 * N2 + a * W1 * W2 * W3 * N1).sum())


def measure_wq(W, stream, flush, dev):
    """Weighted-quadrature mass and diffusion stiffness (FP64, lognormal
    coefficient on the point grid) on the 32^3 p=3 mesh, each next to the Gauss
    form of the same matrix: element matrices by sum factorization plus their
    CSR assembly."""
    import torch
    from paper_2207_00280_gb300 import workloads as wl
    from paper_2207_00280_gb300.plan import IgaPlan, Patch
    sp = W.spec
    peaks = measured_peaks()[0]
    pl = IgaPlan(Patch(sp.knots, sp.p, sp.q), method="sumfact", precision="fp64", mass=True,
                 stiffness=False, blocking=False)
    c = torch.as_tensor(wl.lognormal(pl.wq_grid_size(0), 93), device=dev)
    vals = torch.empty(pl.n_csr_nnz, dtype=torch.float64, device=dev)
    ms = _time_steps(lambda: pl.wq_mass(c=c, values=vals, stream=stream), 10, stream, flush)
    fl = wq_flops(sp.knots, sp.p, pl.wq_points(0))
    peak = N_SM * DFMA_PER_SM_CLK * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6
    out = {"rows": pl.n_dofs, "nnz": pl.n_csr_nnz, "ms_per_matrix": round(ms, 4),
           "rows_per_s": round(pl.n_dofs / (ms * 1e-3), 1), "flop_per_matrix": fl,
           "fp64_frac": round(fl / (ms * 1e-3) / peak, 4)}
    # the Gauss route to the same global matrix
    _, M, _ = pl.empty_outputs(device=dev, dof=False)
    rho = torch.as_tensor(wl.lognormal(pl.n_qp, 94), device=dev)

    def gauss():
        pl.integrate(rho=rho, M=M, stream=stream)
        pl.assemble(M, values=vals, stream=stream)
    out["gauss_sumfact_plus_assembly_ms"] = round(_time_steps(gauss, 10, stream, flush), 4)
    pl.close()
    # the diffusion stiffness by weighted quadrature, next to its Gauss route
    pl = IgaPlan(Patch(sp.knots, sp.p, sp.q), method="sumfact", precision="fp64", mass=False,
                 stiffness=True, blocking=False)
    ms = _time_steps(lambda: pl.wq_stiffness(c=c, values=vals, stream=stream), 10, stream, flush)
    fl = wq_flops(sp.knots, sp.p, pl.wq_points(0), stiffness=True)
    st = {"ms_per_matrix": round(ms, 4), "rows_per_s": round(pl.n_dofs / (ms * 1e-3), 1),
          "flop_per_matrix": fl, "fp64_frac": round(fl / (ms * 1e-3) / peak, 4)}
    K, _, _ = pl.empty_outputs(device=dev, dof=False)
    kap = torch.as_tensor(wl.lognormal(pl.n_qp, 95), device=dev)

    def gauss_k():
        pl.integrate(kappa=kap, K=K, stream=stream)
        pl.assemble(K, values=vals, stream=stream)
    st["gauss_sumfact_plus_assembly_ms"] = round(_time_steps(gauss_k, 10, stream, flush), 4)
    out["stiffness"] = st
    del K
    pl.close()
    # the same two matrices in float-float arithmetic (FP64_DF plan)
    pl = IgaPlan(Patch(sp.knots, sp.p, sp.q), method="sumfact", precision="fp64_df", blocking=False)
    out["fp64_df_ms_per_matrix"] = {
        "mass": round(_time_steps(lambda: pl.wq_mass(c=c, values=vals, stream=stream), 10, stream,
                                  flush), 4),
        "stiffness": round(_time_steps(lambda: pl.wq_stiffness(c=c, values=vals, stream=stream), 10,
                                       stream, flush), 4)}
    pl.close()
    return out


def apply_flops_per_element(p, q):
    """Algorithmic flops of the matrix-free operator per element (3D, identity
    geometry, multiply-add = 2): interpolation a1, a2, a3 (value and gradient),
    the flux, then the transposed contractions q3, q2, q1."""
    n = p + 1
    fma = 2 * n ** 3 * q + 3 * n * n * q * q + 4 * n * q ** 3   # interpolation
    fma += 4 * q ** 3                                          # flux and mass weight
    fma += 4 * n * q ** 3 + 3 * n * n * q * q + 2 * n ** 3 * q   # test side
    return 2 * fma


def measure_apply(A, kappa, stream, flush, dev):
    """Matrix-free y = K(kappa) x + M x on the 40^3 p=3 workload, FP64, float-float
    (FP64_DF plan) and FP32."""
    import torch
    from paper_2207_00280_gb300 import workloads as wl
    from paper_2207_00280_gb300.plan import IgaPlan, Patch
    sa = A.spec
    peaks = measured_peaks()[0]
    f_el = apply_flops_per_element(sa.p, sa.q)
    out = {"elements": sa.E, "dofs": sa.n_dofs, "flop_per_element": f_el}
    for pr, dt in (("fp64", torch.float64), ("fp64_df", torch.float64), ("fp32", torch.float32)):
        pl = IgaPlan(Patch(sa.knots, sa.p, sa.q), method="sumfact", precision=pr, blocking=False)
        x = torch.as_tensor(wl.normal(sa.n_dofs, wl.SEED_ADJ_U), device=dev, dtype=dt)
        y = torch.empty_like(x)
        ms = _time_steps(lambda: pl.apply(x, kappa=kappa, alpha=1.0, beta=1.0, y=y, stream=stream),
                         10, stream, flush)
        esz = 4 if pr == "fp32" else 8
        # kappa, the per-element results written and read back, x gathered, y written
        bytes_ = sa.E * sa.Q * 8 + 2 * sa.E * (sa.p + 1) ** 3 * esz + 2 * sa.n_dofs * esz
        ent = {"ms_per_step": round(ms, 4), "elements_per_s": round(sa.E / (ms * 1e-3), 1),
               "gflops": round(f_el * sa.E / (ms * 1e-3) / 1e9, 1),
               "hbm_frac": round(bytes_ / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4)}
        if pr == "fp64":
            peak = N_SM * DFMA_PER_SM_CLK * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6
            ent["fp64_frac"] = round(f_el * sa.E / (ms * 1e-3) / peak, 4)
        out[pr] = ent
        pl.close()
    return out


def grad_flops_per_element(p, q):
    """Operations of the element-matrix backward per element (3D, identity
    geometry, multiply-add = 2, FP64 form): S = G + G^T on the triangle of x
    blocks, then for the stiffness (3 terms, x pairs (d, d) and (v, v)) and the
    mass (1 term) the x stage on the triangle, the y stage on the (a3 <= b3)
    triangle and the z stage."""
    n = p + 1
    n2 = n * n
    tx, t3 = n2 * (n2 + 1) // 2, n * (n + 1) // 2
    adds = 2 * tx * n2
    fma_k = q * tx * (2 * n2 + 2 * n) + q * 3 * t3 * q * (n2 + n) + q * 3 * q * q * (n2 + n)
    fma_m = q * tx * (n2 + n) + q * t3 * q * (n2 + n) + q * q * q * (n2 + n)
    return adds + 2 * (fma_k + fma_m)


def measure_grad(W, stream, flush, dev):
    """Backward of the 32^3 p=3 element matrices (dL/dkappa and dL/drho from
    dL/dK_e and dL/dM_e), FP64, float-float (FP64_DF plan) and FP32: bytes =
    both upstream blocks read and both gradients written."""
    import torch
    from paper_2207_00280_gb300.plan import IgaPlan, Patch
    sp = W.spec
    peaks = measured_peaks()[0]
    f_el = grad_flops_per_element(sp.p, sp.q)
    out = {"elements": sp.E, "flop_per_element": f_el}
    for pr in ("fp64", "fp64_df", "fp32"):
        pl = IgaPlan(Patch(sp.knots, sp.p, sp.q), method="sumfact", precision=pr, blocking=False)
        dt = pl.out_dtype
        gen = torch.Generator(device=dev).manual_seed(20220701)
        GK = torch.randn(pl.info.n_mat_entries, dtype=dt, device=dev, generator=gen)
        GM = torch.randn(pl.info.n_mat_entries, dtype=dt, device=dev, generator=gen)
        gk = torch.empty(pl.n_qp, dtype=dt, device=dev)
        gr = torch.empty(pl.n_qp, dtype=dt, device=dev)
        ms = _time_steps(lambda: pl.integrate_grad(GK=GK, GM=GM, grad_kappa=gk, grad_rho=gr,
                                                   stream=stream), 10, stream, flush)
        esz = 4 if pr == "fp32" else 8
        bytes_ = 2 * (GK.numel() + pl.n_qp) * esz
        ent = {"ms_per_step": round(ms, 4), "elements_per_s": round(sp.E / (ms * 1e-3), 1),
               "gflops": round(f_el * sp.E / (ms * 1e-3) / 1e9, 1),
               "hbm_frac": round(bytes_ / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4)}
        if pr == "fp64":
            peak = N_SM * DFMA_PER_SM_CLK * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6
            ent["fp64_frac"] = round(f_el * sp.E / (ms * 1e-3) / peak, 4)
        out[pr] = ent
        del GK, GM, gk, gr
        pl.close()
        torch.cuda.empty_cache()
    return out


def measure_assembly(W, kappa, stream, flush, dev):
    """Global CSR assembly of the 32^3 p=3 element matrices (FP64 K and M, and
    FP32 K): HBM-bound gather, bytes = element matrices read + values written."""
    import torch
    from paper_2207_00280_gb300.plan import IgaPlan, Patch
    sp = W.spec
    peaks = measured_peaks()[0]
    out = {"elements": sp.E, "dofs": sp.n_dofs}
    for pr in ("fp64", "fp32"):
        pl = IgaPlan(Patch(sp.knots, sp.p, sp.q), method="sumfact", precision=pr, blocking=False)
        K, M, _ = pl.empty_outputs(device=dev, dof=False)
        pl.integrate(kappa=kappa, K=K, M=M, stream=stream)
        vals = torch.empty(pl.n_csr_nnz, dtype=pl.out_dtype, device=dev)
        ms = _time_steps(lambda: pl.assemble(K, values=vals, stream=stream), 10, stream, flush)
        esz = 8 if pr == "fp64" else 4
        bytes_ = (K.numel() + pl.n_csr_nnz) * esz
        out[pr] = {"nnz": pl.n_csr_nnz, "ms_per_matrix": round(ms, 4),
                   "achieved_gbs": round(bytes_ / (ms * 1e-3) / 1e9, 1),
                   "hbm_frac": round(bytes_ / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4),
                   "bytes_per_launch": bytes_}
        del K, M, vals
        pl.close()
        torch.cuda.empty_cache()
    return out


def traffic_from_profiles(args, esize):
    """DRAM bytes per launch of the element kernel from a committed ncu summary,
    if its recorded source hash matches the current kernel source."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        with open(path) as f:
            tab = json.load(f)
    except Exception:
        return None
    key = f"{args.workload}:{args.method}:{args.precision}"
    ent = tab.get(key)
    if not ent:
        return None
    src = os.path.join(ROOT, "paper_2207_00280_gb300", "csrc", ent["source"])
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except Exception:
        return None
    if h != ent.get("sha"):
        return None
    return ent["dram_bytes_per_launch"]


def run_reference(args, ws, rank):
    """Reference arm: the FP64 oracle timed on the host cores, each step a
    bounded sample of the workload's elements."""
    if rank != 0:
        return None
    import numpy as np
    import oracle
    from paper_2207_00280_gb300 import workloads as wl
    W = wl.WORKLOADS[args.workload]
    sp = W.spec
    P = oracle.Patch(sp.knots, sp.p, sp.q)
    kappa = W.kappa()
    G = W.jacobian()
    mass = G is None
    fn = P.sumfact if args.method == "sumfact" else P.classical
    per_step = args.ref_elements
    rng = np.random.default_rng(7)
    for _ in range(args.warmup):
        fn(rng.choice(sp.E, size=min(8, sp.E), replace=False), kappa=kappa, G=G, mass=mass)
    times = []
    for _ in range(args.steps):
        el = rng.choice(sp.E, size=min(per_step, sp.E), replace=False)
        t0 = time.perf_counter()
        fn(el, kappa=kappa, G=G, mass=mass)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    rate = per_step * args.steps / tot
    return {
        "impl": "reference", "metric": METRIC, "value": round(rate, 2), "unit": UNIT,
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(tot / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded lognormal kappa, open uniform knots)",
        "config": {"workload": args.workload, "method": args.method, "precision": "fp64",
                   "sample_elements_per_step": per_step, "elements": sp.E},
        "cpu_baseline": {"value": round(rate, 2), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} random elements per step of {sp.E}, FP64 oracle "
                                   f"({'Algorithm 2' if args.method == 'sumfact' else 'Algorithm 1'}), one thread"},
        "e2e": {"value": round(rate, 2), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="3d_p3_32")
    ap.add_argument("--method", default="sumfact", choices=["sumfact", "classical"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp64_df", "fp32", "bf16"])
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-compare", dest="compare", action="store_false")
    ap.add_argument("--no-extra-forms", dest="extra_forms", action="store_false")
    ap.add_argument("--no-probe", dest="probe", action="store_false")
    ap.add_argument("--cpu-seconds", type=float, default=24.0)
    ap.add_argument("--ref-elements", type=int, default=512)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    if args.impl == "reference":
        ws = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        line = run_reference(args, ws, rank)
        if line is not None:
            print(json.dumps(line), flush=True)
        return 0

    # the batch autotuner's choices go to a file the line reports (a fresh one
    # per run, so that every run tunes)
    os.environ.setdefault("IGA_AUTOTUNE_CACHE",
                          os.path.join("/tmp", f"iga_autotune_{os.getpid()}.json"))
    ws, rank, local = dist_setup()
    line = run_ours(args, ws, rank, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
