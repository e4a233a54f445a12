"""GPU tests of the batched schedules: many patches of mixed degree and size in
one persistent launch (optionally a CUDA graph) against per-patch launches
(bit-exact: the same device function runs in the same order) and against the
oracle; the queue's watchdog and item checks report errors without faults."""
import json
import os

import numpy as np
import pytest
import torch

from gpu_util import BF16_TOL, FP32_TOL, rel_frob
from paper_2207_00280_gb300 import capi
from paper_2207_00280_gb300 import workloads as wl
from paper_2207_00280_gb300.plan import IgaPlan, Patch

pytestmark = pytest.mark.gpu
dev = torch.device("cuda")

SCHED = {"per_patch": capi.IGA_SCHED_PER_PATCH, "persistent": capi.IGA_SCHED_PERSISTENT,
         "graph": capi.IGA_SCHED_PERSISTENT_GRAPH, "auto": capi.IGA_SCHED_AUTO}


def _batch(specs, kappa, schedule, prec="fp32", mass=True, G=None):
    patches = [Patch(s.knots, s.p, s.q) for s in specs]
    plan = IgaPlan(patches, method="sumfact", precision=prec, mass=mass, schedule=SCHED[schedule])
    K, M, D = plan.empty_outputs()
    K.fill_(float("nan"))
    if M is not None:
        M.fill_(float("nan"))
    plan.integrate(kappa=kappa, jac=G, K=K, M=M, dof=D)
    torch.cuda.synchronize()
    return plan, K, M, D


def _specs_small():
    # every degree 1..5, uneven sizes, q = p+1 (and one q = p+2 patch)
    return [wl.PatchSpec(3, 3, 3, 4), wl.PatchSpec(3, 1, 5, 2), wl.PatchSpec(3, 5, 2, 6),
            wl.PatchSpec(3, 2, 4, 3), wl.PatchSpec(3, 4, 2, 5), wl.PatchSpec(3, 1, 3, 2),
            wl.PatchSpec(3, 2, 2, 4), wl.PatchSpec(3, 3, 2, 4)]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_persistent_equals_per_patch_and_oracle(oracle_mod, prec):
    specs = _specs_small()
    nqp = sum(s.E * s.Q for s in specs)
    kappa = torch.as_tensor(wl.lognormal(nqp, 2210), device=dev)
    ref = _batch(specs, kappa, "per_patch", prec)
    tol = FP32_TOL if prec == "fp32" else BF16_TOL
    for sched in ("persistent", "graph", "auto"):
        plan, K, M, D = _batch(specs, kappa, sched, prec)
        if sched == "auto":
            # the autotuner may pick another schedule (warp-per-element, the
            # other stage-3 form or CTA size): same sums, another rounding order
            assert torch.equal(D, ref[3])
            for i in range(len(specs)):
                assert rel_frob(plan.patch_view(K, i).cpu().numpy(),
                                ref[0].patch_view(ref[1], i).cpu().numpy()) <= tol
                assert rel_frob(plan.patch_view(M, i).cpu().numpy(),
                                ref[0].patch_view(ref[2], i).cpu().numpy()) <= tol
            continue
        assert torch.equal(K, ref[1]) and torch.equal(M, ref[2]) and torch.equal(D, ref[3]), sched
        # the graph is replayed for the same pointers: same result again
        plan.integrate(kappa=kappa, K=K, M=M, dof=D)
        torch.cuda.synchronize()
        assert torch.equal(K, ref[1]) and torch.equal(M, ref[2])
    plan, K, M, D = ref
    kh = kappa.cpu().numpy()
    for i, s in enumerate(specs):
        P = oracle_mod.Patch(s.knots, s.p, s.q)
        q0, q1 = plan.qp_offset[i], plan.qp_offset[i + 1]
        el = np.arange(min(P.E, 6))
        Kr, Mr = P.sumfact(el, kappa=kh[q0:q1])
        Kg = plan.patch_view(K, i).cpu().numpy()[el]
        Mg = plan.patch_view(M, i).cpu().numpy()[el]
        tol = FP32_TOL if prec == "fp32" else BF16_TOL
        assert rel_frob(Kg, Kr) <= tol and rel_frob(Mg, Mr) <= tol
        d0, d1 = plan.dofmap_offset[i], plan.dofmap_offset[i + 1]
        dof = D[d0:d1].view(-1, P.N).cpu().numpy()[el]
        np.testing.assert_array_equal(dof, P.dofmap(el) + plan.dof_offset[i])


def test_64_patch_batch_full(oracle_mod):
    """64 patches, p ~ U{1..5}, elements per side ~ U{4..24} (seeded), q = p+1,
    lognormal kappa, FP32 mass + stiffness (the benchmark's batch): one
    persistent CUDA-graph launch equals the 64 per-patch launches bit for bit,
    and a seeded sample of every patch's elements (its 8 corners and 4 random
    elements; every patch of every degree, so each p = 5 patch) matches the
    oracle within the FP32 tolerance, dof maps bit-exact with the patch offset."""
    specs = wl.batch_specs()
    nqp = sum(s.E * s.Q for s in specs)
    kappa = torch.as_tensor(wl.lognormal(nqp, wl.SEED_BATCH_KAPPA), device=dev)
    a = _batch(specs, kappa, "per_patch")
    b = _batch(specs, kappa, "graph")
    assert torch.equal(a[1], b[1]) and torch.equal(a[2], b[2]) and torch.equal(a[3], b[3])
    del a
    plan, K, M, D = b
    assert torch.isfinite(K).all() and torch.isfinite(M).all()
    assert sum(1 for s in specs if s.p == 5) > 0
    kh = kappa.cpu().numpy()
    rng = np.random.default_rng(2209)
    worst = {}
    for i, s in enumerate(specs):
        P = oracle_mod.Patch(s.knots, s.p, s.q)
        Kk = s.K
        corners = {c0 + Kk * (c1 + Kk * c2) for c0 in (0, Kk - 1) for c1 in (0, Kk - 1)
                   for c2 in (0, Kk - 1)}
        el = np.array(sorted(corners | set(rng.choice(P.E, size=4, replace=False).tolist())),
                      dtype=np.int64)
        q0, q1 = plan.qp_offset[i], plan.qp_offset[i + 1]
        Kr, Mr = P.sumfact(el, kappa=kh[q0:q1])
        idx = torch.as_tensor(el, device=dev)
        Kg = plan.patch_view(K, i)[idx].cpu().numpy()
        Mg = plan.patch_view(M, i)[idx].cpu().numpy()
        ek, em = rel_frob(Kg, Kr), rel_frob(Mg, Mr)
        worst[s.p] = max(worst.get(s.p, 0.0), ek, em)
        assert ek <= FP32_TOL and em <= FP32_TOL, (i, s, ek, em)
        d0, d1 = plan.dofmap_offset[i], plan.dofmap_offset[i + 1]
        dof = D[d0:d1].view(-1, P.N)[idx].cpu().numpy()
        np.testing.assert_array_equal(dof, P.dofmap(el) + plan.dof_offset[i])
    print("64-patch batch, worst FP32 error per degree:", worst)


def test_curved_batch_stiffness_only(oracle_mod):
    specs = [wl.PatchSpec(3, 2, 3, 3), wl.PatchSpec(3, 3, 2, 4), wl.PatchSpec(3, 4, 2, 5)]
    nqp = sum(s.E * s.Q for s in specs)
    kappa = torch.as_tensor(wl.lognormal(nqp, 77), device=dev)
    G = np.concatenate([wl.curved_map_jacobian(s.knots, s.q).reshape(-1) for s in specs])
    Gt = torch.as_tensor(G, device=dev)
    a = _batch(specs, kappa, "per_patch", mass=False, G=Gt)
    b = _batch(specs, kappa, "graph", mass=False, G=Gt)
    assert torch.equal(a[1], b[1])
    plan, K = b[0], b[1]
    off = 0
    for i, s in enumerate(specs):
        P = oracle_mod.Patch(s.knots, s.p, s.q)
        n = s.E * s.Q
        Kr, _ = P.sumfact(kappa=kappa[plan.qp_offset[i]:plan.qp_offset[i + 1]].cpu().numpy(),
                          G=G[off * 9:(off + n) * 9].reshape(s.E, s.Q, 3, 3), mass=False)
        off += n
        assert rel_frob(plan.patch_view(K, i).cpu().numpy(), Kr) <= FP32_TOL


def _fresh_plan_with_env(env, specs):
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        patches = [Patch(s.knots, s.p, s.q) for s in specs]
        return IgaPlan(patches, method="sumfact", precision="fp32",
                       schedule=capi.IGA_SCHED_PERSISTENT)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def test_queue_watchdog_timeout_is_reported():
    """A time budget of 1 ns (host flag) makes every CTA stop before its first
    item: the call returns IGA_ERR_TIMEOUT and the error stays with the plan."""
    specs = _specs_small()[:3]
    plan = _fresh_plan_with_env({"IGA_QUEUE_BUDGET_NS": "1"}, specs)
    K, M, D = plan.empty_outputs()
    kappa = torch.ones(plan.n_qp, dtype=torch.float64, device=dev)
    with pytest.raises(capi.IgaError) as ei:
        plan.integrate(kappa=kappa, K=K, M=M, dof=D)
    assert ei.value.code == capi.IGA_ERR_TIMEOUT
    with pytest.raises(capi.IgaError) as ei:  # sticky
        plan.integrate(kappa=kappa, K=K, M=M, dof=D)
    assert ei.value.code == capi.IGA_ERR_TIMEOUT
    # the context is still usable
    x = torch.ones(4, device=dev).sum()
    assert float(x) == 4.0


def test_corrupted_work_item_is_reported():
    """A work item naming a patch that does not exist (written on the host) is
    detected by the kernel, skipped, and reported as IGA_ERR_DEVICE."""
    specs = _specs_small()[:3]
    plan = _fresh_plan_with_env({"IGA_TEST_CORRUPT_QUEUE": "1"}, specs)
    K, M, D = plan.empty_outputs()
    kappa = torch.ones(plan.n_qp, dtype=torch.float64, device=dev)
    with pytest.raises(capi.IgaError) as ei:
        plan.integrate(kappa=kappa, K=K, M=M, dof=D)
    assert ei.value.code == capi.IGA_ERR_DEVICE


def test_autotune_cache_file(tmp_path):
    path = tmp_path / "tune.json"
    old = os.environ.get("IGA_AUTOTUNE_CACHE")
    os.environ["IGA_AUTOTUNE_CACHE"] = str(path)
    try:
        specs = [wl.PatchSpec(3, 2, 9, 3), wl.PatchSpec(3, 1, 12, 2)]
        nqp = sum(s.E * s.Q for s in specs)
        kappa = torch.as_tensor(wl.lognormal(nqp, 5), device=dev)
        _batch(specs, kappa, "auto")
    finally:
        if old is None:
            os.environ.pop("IGA_AUTOTUNE_CACHE", None)
        else:
            os.environ["IGA_AUTOTUNE_CACHE"] = old
    if path.exists():  # the cache is process-wide: an earlier test may have tuned these classes
        tab = json.loads(path.read_text())
        assert all(v % 100 in (1, 2, 4, 8) and v // 100 in (0, 4, 8, 16) for v in tab.values())


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("forced", [4, 8, 16])
@pytest.mark.parametrize("curved", [False, True])
def test_forced_schedules_match_oracle(oracle_mod, prec, forced, curved):
    """Every schedule the autotuner can pick, forced through IGA_BATCH_SCHED on a
    batch of every degree 1..5: the mma.sync stage-3 form (4; p = 3, BF16
    p = 4), the other CTA size (8; p = 4, 5, identity map), the warp-per-element
    kernel (16; p <= 2).  Each patch against the oracle within the plan's
    tolerance, dof maps bit-exact."""
    specs = _specs_small()
    nqp = sum(s.E * s.Q for s in specs)
    kappa = torch.as_tensor(wl.lognormal(nqp, 2211), device=dev)
    G = None
    if curved:
        G = torch.as_tensor(np.concatenate([wl.curved_map_jacobian(s.knots, s.q).reshape(-1)
                                            for s in specs]), device=dev)
    old = os.environ.get("IGA_BATCH_SCHED")
    os.environ["IGA_BATCH_SCHED"] = str(forced)
    try:
        plan, K, M, D = _batch(specs, kappa, "graph", prec, G=G)
    finally:
        if old is None:
            os.environ.pop("IGA_BATCH_SCHED", None)
        else:
            os.environ["IGA_BATCH_SCHED"] = old
    kh = kappa.cpu().numpy()
    Gh = G.cpu().numpy() if curved else None
    tol = FP32_TOL if prec == "fp32" else BF16_TOL
    g0 = 0
    for i, s in enumerate(specs):
        P = oracle_mod.Patch(s.knots, s.p, s.q)
        q0, q1 = plan.qp_offset[i], plan.qp_offset[i + 1]
        Gi = Gh[g0 * 9:(g0 + P.E * P.Q) * 9].reshape(P.E, P.Q, 3, 3) if curved else None
        g0 += P.E * P.Q
        Kr, Mr = P.sumfact(kappa=kh[q0:q1], G=Gi)
        assert rel_frob(plan.patch_view(K, i).cpu().numpy(), Kr) <= tol, (i, s)
        assert rel_frob(plan.patch_view(M, i).cpu().numpy(), Mr) <= tol, (i, s)
        d0, d1 = plan.dofmap_offset[i], plan.dofmap_offset[i + 1]
        np.testing.assert_array_equal(D[d0:d1].view(-1, P.N).cpu().numpy(), P.dofmap() + plan.dof_offset[i])
