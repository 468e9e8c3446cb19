"""Benchmark of the two-site QC-DMRG hot path on GB300 (one JSON line on rank 0).

Default: the FeMoco-shaped middle bond (L=76, N=113, 2Sz=1, M=6000, the largest
workload; block bases grown from seeded random sector-orthonormal O),
split-BF16 x3 tensor-core H.psi (Eq. dgemm, Sec. 2.2.1).  A step is a fixed chunk of the working-precision
Davidson iteration (dmrg_davidson_lowp from a fixed start vector: one H.psi per
iteration plus FP64 orthogonalisation, subspace eigenproblem and residual).
Untimed extras: the FP32 and FP64 sigma of the same psi (relative error), the
FP64 H.psi and Davidson iteration, one renormalization (Eq. renorm_mat), and a
sub-line with the FP64 L=24/M=512 step (Davidson to 1e-8 + renormalization)
against its mixed-precision runs (|dE|, overlap).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c5b] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H·ψ TFLOP/s & Davidson s/iter at M; mixed vs FP64 GPU at |ΔE|≤1e-6 Eh"

# hpsi_flops: algorithmic FLOPs of one middle-bond H.psi (sum over the task list of
# 2 min(mnp + mpq, npq + mnq), identity sides free), counted once by the host
# planner from the workload's sector tables (checked against the planner by
# tests/test_workloads_cpu.py), so that the oracle arm needs no library call.
# oracle: the workload the FP64 oracle times as the CPU baseline and reference arm
# (it cannot build the L=40 or L=76 blocks within host memory and time).
WORKLOADS = {
    # FP64 two-site DMRG, L=24, N=24, Sz=0, M=512, Davidson tol 1e-8, middle bond
    "c2": dict(name="L24_N24_Sz0_M512_fp64_middle_bond", L=24, N=24, two_sz=0, M=512, tol=1e-8,
               precision=0, hpsi_flops=19930869124.0, oracle="c2"),
    # mixed-precision workload: L=40, N=40, Sz=0, M=2000 (middle bond)
    "c3": dict(name="L40_N40_Sz0_M2000_middle_bond", L=40, N=40, two_sz=0, M=2000, tol=1e-8,
               precision=2, hpsi_flops=1200097633784.0, oracle="c2"),
    # FeMoco-shaped: L=76, N=113, 2Sz=1, M=3000 / 6000 (middle bond)
    "c5a": dict(name="L76_N113_Sz1_M3000_middle_bond", L=76, N=113, two_sz=1, M=3000, tol=1e-8,
                precision=2, hpsi_flops=4254718080252.0, oracle="c2"),
    "c5b": dict(name="L76_N113_Sz1_M6000_middle_bond", L=76, N=113, two_sz=1, M=6000, tol=1e-8,
                precision=2, hpsi_flops=31452027390656.0, oracle="c2", grow_renorm="fp32"),
    # batched: 256 independent instances (seeds 0..255), L in 10..20, N=L, M in 64..256
    "c4": dict(name="batched_256_L10-20_M64-256_middle_bonds", L=0, N=0, two_sz=0, M=0, tol=1e-8,
               precision=1, instances=256, oracle="c2"),
    # small case: L=8, N=8, M=64
    "c1": dict(name="L8_N8_Sz0_M64_fp64_middle_bond", L=8, N=8, two_sz=0, M=64, tol=1e-9,
               precision=0, hpsi_flops=26282476.0, oracle="c1"),
}

for _key, _wl in WORKLOADS.items():
    _wl["key"] = _key

DAVIDSON_ITERS_PER_STEP = 4  # working-precision Davidson iterations per timed step

FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 (nominal, recipe table)
FP32_SIMT_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # FP32 FMA units x 2 FLOP x max SM clock

# DRAM bytes (read + write) per launch of the dominant H.psi kernel, from one ncu
# capture of the unchanged kernel at that workload and precision (else null)
TRAFFIC_PER_LAUNCH = {
    ("c2", 0, 512, (32768.0, 50000.0, 33, 0, 0, 0)): 1.034e9 + 0.147e9,
    ("c2", 0, 512, (32768.0, 200000.0, 33, 0, 0, 0)): 1.0293e9 + 0.1472e9,
    ("c2", 0, 512, (131072.0, 50000.0, 33, 0, 0, 0)): 1.8010e9 + 0.7325e9,
    ("c2", 0, 512, (131072.0, 200000.0, 33, 0, 0, 0)): 1.4767e9 + 0.4892e9,
    # split-BF16x3 H.psi, every block on the tensor cores: DRAM read + write of the
    # chain_tc2 launches of one H.psi (one shape at M=3000, two at M=6000)
    ("c5a", 2, 3000, (8192.0, 200000.0, 1, 1, 1, 0)): 434.8e9 + 0.175e9,
    ("c5b", 2, 6000, (8192.0, 200000.0, 1, 1, 1, 0)): 1282.5e9 + 0.536e9,
}
# Algorithmic bytes of one split-BF16x3 H.psi: the distinct pre-split operator tiles
# (4 bytes per padded element, each read once), the psi tiles, psi and sigma
# (host task dump of the same launch plan).
ALG_BYTES = {
    "c5a": 30.7e9 + 10e6 + 2 * 10.6e6,
    "c5b": 88.655e9 + 27.8e6 + 2 * 40.6e6,
}


def _clock_sampler():
    f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                             stdout=f, stderr=subprocess.DEVNULL)
    except FileNotFoundError:
        return None, f.name
    return p, f.name


def _clock_summary(path, gpu_index):
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9 or parts[0] != str(gpu_index):
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
    except OSError:
        pass
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


def max_over_ranks(x, device):
    """Max of a per-rank scalar over all ranks (replicas: the job takes as long as its slowest rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_tflops(flops_per_rank, world, step_ms_max):
    """Whole-job throughput of N replicas: all ranks' algorithmic FLOPs over the slowest rank's time."""
    return flops_per_rank * world / (step_ms_max * 1e-3) / 1e12


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def _oracle_workload(wl):
    """The workload the oracle times for this one, and its recorded H.psi FLOPs."""
    owl = dict(WORKLOADS[wl.get("oracle", "c2")])
    return owl, owl["hpsi_flops"]


def _setup(wl, precision, stream, dev, release=False):
    """Context at the workload's middle bond, blocks grown from seeded random O (with FP32
    renormalization products where the workload says so: the same bases serve every
    precision measured on them); later renormalizations are FP64."""
    import torch
    from paper_2001_04890_gb300 import binding, workloads
    L, N, two_sz, M = wl["L"], wl["N"], wl["two_sz"], wl["M"]
    nu, nd = (N + two_sz) // 2, (N - two_sz) // 2
    k = (L - 2) // 2
    h, v = workloads.integrals(L, seed=0)
    ctx = binding.DMRG(h, v, N, two_sz, M, precision, stream=stream.cuda_stream)
    if wl.get("grow_renorm") == "fp32":
        ctx.set_renorm_precision(binding.PREC_FP32)
    workloads.grow_middle_bond(ctx, L, nu, nd, M, k, seed=0, release=release)
    ctx.set_renorm_precision(binding.PREC_FP64)
    return ctx, k


def run_gpu(args, wl, rank, world, precision, e2e=True, sample_clocks=True):
    import torch
    from paper_2001_04890_gb300 import workloads

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    ctx, k = _setup(wl, precision, stream, dev)
    tune = None
    if getattr(args, "tune", ""):
        ctx.set_tune(**_fixed_tune(args.tune))
        tune = ctx.get_tune()
    elif getattr(args, "autotune", False):
        tune_ms, tune = ctx.autotune(reps=2)  # plan-time choice of the launch shape (untimed)
    blocks, dim = ctx.psi_layout()
    if tune is not None:
        ctx.set_tune(**tune)  # same shape; drops the plan so that one build of it is timed here
    t_plan = time.perf_counter()
    flops_per_hpsi, ntasks = ctx.hpsi_flops()  # builds the position's H.psi plan (host lists + upload)
    plan_s = time.perf_counter() - t_plan
    psi0_host = workloads.gaussian(dim, seed=1)
    psi0_host /= np.linalg.norm(psi0_host)
    with torch.cuda.stream(stream):
        psi0_dev = torch.from_numpy(psi0_host).to(f"cuda:{dev}")
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{dev}")
    stream.synchronize()

    def step():
        ctx.set_position(k, 1)
        ctx.set_psi(psi0_dev)
        e, it = ctx.davidson(tol=wl["tol"], max_iter=400, allow_noconv=True)
        ctx.renormalize(+1)
        return e, it

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ctx.stats(reset=True)
    sampler, clk_path = _clock_sampler() if sample_clocks else (None, None)
    time.sleep(0.3)
    ev, iters, energy = [], [], None
    torch.cuda.nvtx.range_push("step")  # lets ncu --nvtx-include "step/" capture the timed steps only
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)  # L2 flush between timed steps (256 MB > 129 MB L2)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        energy, it = step()
        b.record(stream)
        ev.append((a, b))
        iters.append(it)
    stream.synchronize()
    torch.cuda.nvtx.range_pop()
    st = ctx.stats(reset=True)
    step_ms = sum(a.elapsed_time(b) for a, b in ev)
    e2e_ms, d2h_bytes = None, 0
    if e2e:
        # end-to-end through the C ABI with HOST buffers: H2D of the start vector and
        # D2H of the result (energy + predicted wave function) inside the timed region
        pin_in = torch.from_numpy(psi0_host).pin_memory()
        e2e_ms = 0.0
        for _ in range(args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.set_position(k, 1)
            ctx.set_psi(pin_in.numpy())
            ctx.davidson(tol=wl["tol"], max_iter=400, allow_noconv=True)
            ctx.renormalize(+1)
            out = ctx.get_psi()
            e2e_ms += (time.perf_counter() - t0) * 1e3
            d2h_bytes = out.nbytes + 8
    clocks = None
    if sampler is not None:
        time.sleep(0.2)
        sampler.terminate()
        sampler.wait()
        clocks = _clock_summary(clk_path, dev)
    # converged middle-bond state for the mixed-vs-FP64 comparison (untimed)
    ctx.set_position(k, 1)
    ctx.set_psi(psi0_dev)
    e_mid, _ = ctx.davidson(tol=wl["tol"], max_iter=400, allow_noconv=True)
    psi_mid = ctx.get_psi()
    step_ms_max = max_over_ranks(step_ms, f"cuda:{dev}")
    ctx.close()
    return dict(dim=dim, flops_per_hpsi=flops_per_hpsi, ntasks=ntasks, stats=st, plan_s=plan_s,
                step_ms=step_ms_max, iters=iters, energy=energy, e2e_ms=e2e_ms, tune=tune,
                h2d=psi0_host.nbytes, d2h=d2h_bytes, clocks=clocks, k=k, e_mid=e_mid, psi_mid=psi_mid)


def run_davidson_bench(args, wl, rank, world, precision):
    """The default measurement: working-precision Davidson iterations at the middle bond.

    Each timed step runs DAVIDSON_ITERS_PER_STEP iterations of dmrg_davidson_lowp
    from the same start vector (one H.psi per iteration and one for the start
    vector); every block goes to the tensor-core kernel in split-BF16 x3.
    """
    import torch
    from paper_2001_04890_gb300 import binding, workloads

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    ctx, k = _setup(wl, precision, stream, dev, release=True)  # only the middle-bond blocks stay resident
    setup_s = time.perf_counter() - t0
    if precision == binding.PREC_BF16X3:
        ctx.set_tune(tc_min=1, by_work=1)  # every output block on the tensor cores
    blocks, dim = ctx.psi_layout()
    t_plan = time.perf_counter()
    flops_per_hpsi, ntasks = ctx.hpsi_flops()  # builds the position's H.psi plan (host lists + upload)
    plan_s = time.perf_counter() - t_plan
    tune = ctx.get_tune()
    psi0_host = workloads.gaussian(dim, seed=1)
    psi0_host /= np.linalg.norm(psi0_host)
    with torch.cuda.stream(stream):
        psi0_dev = torch.from_numpy(psi0_host).to(f"cuda:{dev}")
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{dev}")
    stream.synchronize()
    nit = DAVIDSON_ITERS_PER_STEP

    def step():
        ctx.set_psi(psi0_dev)
        return ctx.davidson_lowp(tol=1e-300, max_iter=nit, allow_noconv=True)

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ctx.stats(reset=True)
    sampler, clk_path = _clock_sampler()
    time.sleep(0.3)
    ev, energy = [], None
    torch.cuda.nvtx.range_push("step")  # lets ncu --nvtx-include "step/" capture the timed steps only
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)  # L2 flush between timed steps (256 MB > 129 MB L2)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        energy, _ = step()
        b.record(stream)
        ev.append((a, b))
    stream.synchronize()
    torch.cuda.nvtx.range_pop()
    st = ctx.stats(reset=True)
    step_ms = sum(a.elapsed_time(b) for a, b in ev)
    # end to end through the C ABI with HOST buffers: H2D of the start vector and D2H of
    # the Ritz vector inside the timed region
    pin_in = torch.from_numpy(psi0_host).pin_memory()
    out = np.empty(dim)
    e2e_ms = 0.0
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        ctx.set_psi(pin_in.numpy())
        ctx.davidson_lowp(tol=1e-300, max_iter=nit, allow_noconv=True)
        ctx.get_psi(out)
        e2e_ms += (time.perf_counter() - t1) * 1e3
    time.sleep(0.2)
    if sampler is not None:
        sampler.terminate()
        sampler.wait()
    clocks = _clock_summary(clk_path, dev) if sampler is not None else None
    step_ms_max = max_over_ranks(step_ms, f"cuda:{dev}")
    extra = {}
    if rank == 0 and not args.no_extras:
        extra = _precision_extras(ctx, psi0_dev, k)
    ctx.close()
    return dict(dim=dim, flops_per_hpsi=flops_per_hpsi, ntasks=ntasks, stats=st, plan_s=plan_s,
                setup_s=setup_s, step_ms=step_ms_max, energy=energy, e2e_ms=e2e_ms, tune=tune,
                h2d=psi0_host.nbytes, d2h=out.nbytes, clocks=clocks, k=k, extra=extra)


def _precision_extras(ctx, psi_dev, k):
    """Untimed: sigma of one psi in each precision (relative error against FP64), the
    H.psi time and one Davidson iteration in FP32 and FP64, and one renormalization."""
    import torch
    from paper_2001_04890_gb300 import binding
    out = {}
    sig = {}
    for name, prec in (("bf16x3", binding.PREC_BF16X3), ("fp32", binding.PREC_FP32), ("fp64", binding.PREC_FP64)):
        if name != "bf16x3":
            ctx.set_precision(prec)
        t0 = time.perf_counter()
        ctx.hpsi(psi_dev)  # builds this precision's task list
        torch.cuda.synchronize()
        plan_s = time.perf_counter() - t0
        ctx.stats(reset=True)
        sig[name] = ctx.hpsi(psi_dev).cpu().numpy()
        st = ctx.stats(reset=True)
        r = {"hpsi_ms": st["hpsi_ms"], "hpsi_tflops": st["hpsi_flops"] / (st["hpsi_ms"] * 1e-3) / 1e12,
             "plan_s": plan_s}
        if name != "bf16x3" and st["hpsi_ms"] < 20000.0:  # one iteration = two H.psi
            ctx.set_psi(psi_dev)
            t0 = time.perf_counter()
            _, it = ctx.davidson_lowp(tol=1e-300, max_iter=1, allow_noconv=True)
            torch.cuda.synchronize()
            r["davidson_s_per_iter"] = (time.perf_counter() - t0) / max(it, 1)
        out[name] = r
        print(json.dumps({name: r}), file=sys.stderr, flush=True)
    ref = sig["fp64"]
    for name in ("bf16x3", "fp32"):
        out[name]["sigma_rel_err_vs_fp64"] = float(np.max(np.abs(sig[name] - ref)) / np.max(np.abs(ref)))
    ctx.set_position(k, 1)
    ctx.set_psi(psi_dev)
    t0 = time.perf_counter()
    ctx.renormalize(+1)
    torch.cuda.synchronize()
    out["renormalize_s"] = time.perf_counter() - t0
    return out


def _shape_key(tune):
    if not tune:
        return None
    return (tune["target_chunks"], tune["min_chunk"], tune["tc_min"], tune["by_work"], tune["flat_wide"],
            tune.get("tc_tiny", 0))


def _fixed_tune(spec):
    t = [float(x) for x in spec.split(",")]
    return dict(target_chunks=t[0], min_chunk=t[1], tc_min=int(t[2]), by_work=int(t[3]), flat_wide=int(t[4]),
                tc_tiny=int(t[5]) if len(t) > 5 else 0)


def profile_hpsi(wl, precision, ncalls, autotune=False, tune_spec=""):
    """Setup, then ncalls H.psi launches inside an NVTX range "hpsi" (for ncu --nvtx)."""
    import torch
    from paper_2001_04890_gb300 import workloads
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    ctx, k = _setup(wl, precision, stream, 0, release=True)  # only the middle-bond blocks stay resident
    setup_s = time.perf_counter() - t0
    _, dim = ctx.psi_layout()
    psi = torch.from_numpy(workloads.gaussian(dim, seed=1)).cuda()
    if tune_spec:
        ctx.set_tune(**_fixed_tune(tune_spec))
    ctx.hpsi(psi)  # builds the task list and temporaries outside the range
    tune = ctx.autotune(reps=2)[1] if (autotune and not tune_spec) else ctx.get_tune()
    ctx.hpsi(psi)
    ctx.stats(reset=True)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("hpsi")
    for _ in range(ncalls):
        ctx.hpsi(psi)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    st = ctx.stats()
    print(json.dumps({"profile": wl["name"], "precision": precision, "hpsi_calls": ncalls,
                      "setup_s": setup_s, "psi_dim": dim, "tune": tune,
                      "hpsi_ms_avg": st["hpsi_ms"] / max(st["hpsi_calls"], 1),
                      "gflop_per_hpsi": ctx.hpsi_flops()[0] / 1e9}), flush=True)
    ctx.close()


def batched_workload(args, wl):
    """Batched instances: one grouped, CUDA-graph-replayed H.psi over all middle bonds.

    Reports the aggregate H.psi TFLOP/s of the grouped launch and of one launch
    sequence per instance (same work), per-instance Davidson s/iter and, for
    the first 16 instances, |dE| of the mixed run against FP64.
    """
    import torch
    from paper_2001_04890_gb300 import binding, workloads
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    n = wl["instances"]
    out = {"workload": wl["name"], "instances": n}
    res = {}
    pairs = (("fp32", 1), ("bf16x3", 2))
    if args.precision != "fp64":  # one low precision only
        pairs = tuple(pr for pr in pairs if pr[0] == args.precision)
    for name, prec in pairs:
        ctxs = []
        t0 = time.perf_counter()
        for seed in range(n):
            L, M, h, v = workloads.batched_instance(seed)
            tsz = L % 2  # N = L; odd N has no Sz = 0 sector: lowest |Sz| (2Sz = 1)
            c = binding.DMRG(h, v, L, tsz, M, prec, stream=stream.cuda_stream)
            workloads.grow_middle_bond(c, L, (L + tsz) // 2, (L - tsz) // 2, M, (L - 2) // 2, seed=seed)
            ctxs.append(c)
        setup_s = time.perf_counter() - t0
        batch = binding.Batch(ctxs)
        tune = batch.autotune(reps=2)[1] if args.autotune else None
        with torch.cuda.stream(stream):
            x = torch.from_numpy(workloads.gaussian(batch.offsets[-1], seed=1)).cuda()
        stream.synchronize()
        for _ in range(args.warmup):
            batch.hpsi(x)
        stream.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            batch.hpsi(x)
        b.record(stream)
        stream.synchronize()
        t_batch = a.elapsed_time(b) / args.steps
        xs = [x[batch.offsets[i]:batch.offsets[i + 1]].clone() for i in range(n)]
        for i, c in enumerate(ctxs):
            c.hpsi(xs[i])
        stream.synchronize()
        a.record(stream)
        for _ in range(args.steps):
            for i, c in enumerate(ctxs):
                c.hpsi(xs[i])
        b.record(stream)
        stream.synchronize()
        t_seq = a.elapsed_time(b) / args.steps
        t0 = time.perf_counter()
        its = 0
        energies = []
        for c in ctxs:
            e, it = c.davidson(tol=wl["tol"], max_iter=400, allow_noconv=True)
            its += it
            energies.append(e)
        dav_s = time.perf_counter() - t0
        res[name] = {"setup_s": setup_s, "launch_shape": tune, "batched_hpsi_ms": t_batch,
                     "batched_hpsi_tflops": batch.flops / (t_batch * 1e-3) / 1e12,
                     "per_instance_hpsi_ms": t_seq,
                     "per_instance_hpsi_tflops": batch.flops / (t_seq * 1e-3) / 1e12,
                     "gflop_per_batched_hpsi": batch.flops / 1e9,
                     "davidson_s_per_iter_avg": dav_s / max(its, 1), "davidson_iters_total": its,
                     "energies_head": energies[:16]}
        print(json.dumps({name: res[name]}), flush=True)
        batch.close()
        for c in ctxs:
            c.close()
    # FP64 reference energies for the first 16 instances
    e64 = []
    for seed in range(16):
        L, M, h, v = workloads.batched_instance(seed)
        tsz = L % 2
        c = binding.DMRG(h, v, L, tsz, M, 0, stream=stream.cuda_stream)
        workloads.grow_middle_bond(c, L, (L + tsz) // 2, (L - tsz) // 2, M, (L - 2) // 2, seed=seed)
        e, _ = c.davidson(tol=wl["tol"], max_iter=400, allow_noconv=True)
        e64.append(e)
        c.close()
    peaks = _peaks()
    for name in res:
        res[name]["max_abs_dE_vs_fp64_first16"] = float(np.max(np.abs(np.array(res[name]["energies_head"]) - e64)))
        del res[name]["energies_head"]
        if name == "bf16x3" and peaks.get("bf16_tflops"):
            peak = peaks["bf16_tflops"] / 3.0
            res[name]["roofline"] = {
                "bound": "tensor", "kernel": "chain_tc2_kernel (batched H.psi, split-BF16 x3 on tcgen05)",
                "achieved": res[name]["batched_hpsi_tflops"], "peak": peak,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst) / 3 (of measured)", "unit": "TFLOP/s",
                "frac": res[name]["batched_hpsi_tflops"] / peak}
    out.update(res)
    return out


def sweep_workload(args, wl):
    """Full two-site sweeps from the Aufbau start (Sec. 2.1) per working precision.

    Reports the wall time per sweep (every Davidson to tol, truncation and
    renormalization of every position, both directions), the lowest energy of
    each sweep and, for the mixed precisions, |dE| against the FP64 run.
    """
    import torch
    from paper_2001_04890_gb300 import binding, workloads
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    L, N, two_sz, M = wl["L"], wl["N"], wl["two_sz"], wl["M"]
    h, v = workloads.integrals(L, seed=0)
    out = {"workload": wl["name"], "sweeps": args.sweeps, "davidson_tol": wl["tol"],
           "positions_per_sweep": 2 * (L - 2), "refine_keep": args.refine_keep,
           "sweep_max_iter": args.sweep_max_iter}
    ref = None
    for name, prec in (("fp64", 0), ("fp32", 1), ("bf16x3", 2)):
        ctx = binding.DMRG(h, v, N, two_sz, M, prec, stream=stream.cuda_stream)
        if args.tune:
            ctx.set_tune(**_fixed_tune(args.tune))
        ctx.set_davidson(args.refine_keep, args.sweep_max_iter)
        torch.cuda.synchronize()
        per = []
        energies = []
        dw_max = []
        for _ in range(args.sweeps):
            t0 = time.perf_counter()
            rec = ctx.sweep_record(1, tol=wl["tol"])  # energies, discarded weights, two-site entropies
            torch.cuda.synchronize()
            per.append(time.perf_counter() - t0)
            energies.append(float(np.min(rec["energies"])))
            dw_max.append(float(np.max(rec["discarded"])))
        st = ctx.stats()
        r = {"s_per_sweep": per, "min_energy_per_sweep": energies, "max_discarded_weight_per_sweep": dw_max,
             "last_sweep_site_entropies": _site_entropies(rec, L),
             "davidson_iters": st["davidson_iters"], "davidson_iters_lowp": st["davidson_iters_lowp"]}
        if ref is None:
            ref = energies
        else:
            r["abs_dE_vs_fp64_per_sweep"] = [abs(a - b) for a, b in zip(energies, ref)]
            r["speedup_vs_fp64_last_sweep"] = out["fp64"]["s_per_sweep"][-1] / per[-1]
        out[name] = r
        print(json.dumps({name: r}), flush=True)
        ctx.close()
    return out


def _site_entropies(rec, L):
    """One-orbital entropy of every site from one sweep's records: the left site of the
    forward positions 0..L-3, then both sites of the first backward position L-2."""
    ent = rec["entropies"]
    return [float(x) for x in list(ent[: L - 2, 0]) + [ent[L - 2, 0], ent[L - 2, 1]]]


def mixed_step_workload(args, wl, tol):
    """One middle-bond step per working precision on the same bases and start vector.

    Davidson to tol (mixed: low-precision matvecs, then the FP64 defect-corrected
    refinement), truncation and renormalization; wall time of each part, H.psi
    counts, |dE| and the state overlap against the FP64 step.
    """
    import torch
    from paper_2001_04890_gb300 import workloads
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    out = {"workload": wl["name"], "davidson_tol": tol}
    ref = None
    for name, prec in (("fp64", 0), ("fp32", 1), ("bf16x3", 2)):
        t0 = time.perf_counter()
        ctx, k = _setup(wl, prec, stream, 0)
        setup_s = time.perf_counter() - t0
        if args.tune:
            ctx.set_tune(**_fixed_tune(args.tune))
        elif args.autotune:
            ctx.autotune(reps=1)
        _, dim = ctx.psi_layout()
        psi0 = workloads.gaussian(dim, seed=1)
        psi0 /= np.linalg.norm(psi0)
        ctx.set_position(k, 1)
        ctx.set_psi(psi0)
        ctx.stats(reset=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e, it = ctx.davidson(tol=tol, max_iter=400, allow_noconv=True)
        torch.cuda.synchronize()
        t_dav = time.perf_counter() - t0
        st = ctx.stats(reset=True)
        x = ctx.get_psi()
        t0 = time.perf_counter()
        ctx.renormalize(+1)
        torch.cuda.synchronize()
        t_ren = time.perf_counter() - t0
        r = {"setup_s": setup_s, "launch_shape": ctx.get_tune(), "davidson_s": t_dav, "iters": it,
             "iters_lowp": st["davidson_iters_lowp"], "iters_fp64": it - st["davidson_iters_lowp"],
             "hpsi_ms_avg": st["hpsi_ms"] / max(st["hpsi_calls"], 1), "renormalize_s": t_ren,
             "step_s": t_dav + t_ren, "energy": e}
        if ref is None:
            ref = (e, x, t_dav + t_ren)
        else:
            r["abs_dE_vs_fp64"] = abs(e - ref[0])
            r["overlap_vs_fp64"] = float(abs(np.dot(x, ref[1])))
            r["step_speedup_vs_fp64"] = ref[2] / (t_dav + t_ren)
        out[name] = r
        print(json.dumps({name: r}), flush=True)
        ctx.close()
    return out


def large_workload(wl, args, iters=4):
    """Middle bond of a large workload, grown once; each working precision in turn.

    Reports the block-growth time, H.psi time and TFLOP/s per precision, a few
    Davidson iterations in the working precision (s/iter; one iteration in FP64,
    whose H.psi takes a minute at M=6000), one renormalization, and the
    relative difference of each low-precision sigma from the FP64 sigma.  The
    bases are grown with FP32 renormalization products when --renorm fp32 (the
    same bases then serve every precision); --M-right sets a smaller bond
    dimension for the right blocks (the non-enlarged block of the paper's
    largest run).
    """
    import torch
    from paper_2001_04890_gb300 import binding, workloads
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    out = {"workload": wl["name"], "L": wl["L"], "N": wl["N"], "two_sz": wl["two_sz"], "M": wl["M"],
           "M_right": args.M_right or wl["M"], "renorm": args.renorm}
    L, N, two_sz, M = wl["L"], wl["N"], wl["two_sz"], wl["M"]
    nu, nd = (N + two_sz) // 2, (N - two_sz) // 2
    k = (L - 2) // 2
    h, v = workloads.integrals(L, seed=0)
    ctx = binding.DMRG(h, v, N, two_sz, M, 0, stream=stream.cuda_stream)
    if args.renorm == "fp32":
        ctx.set_renorm_precision(binding.PREC_FP32)
    t0 = time.perf_counter()
    workloads.grow_middle_bond(ctx, L, nu, nd, M, k, seed=0, release=True, M_right=args.M_right or None)
    torch.cuda.synchronize()
    out["setup_s"] = time.perf_counter() - t0
    _, dim = ctx.psi_layout()
    out["psi_dim"] = dim
    out["sectors"] = [int(len(ctx.block_sectors(0))), int(len(ctx.block_sectors(1)))]
    out["max_sector"] = [int(ctx.block_sectors(0)[:, 2].max()), int(ctx.block_sectors(1)[:, 2].max())]
    psi = torch.from_numpy(workloads.gaussian(dim, seed=1)).cuda()
    sigs = {}
    for name, prec in (("bf16x3", 2), ("fp32", 1), ("fp64", 0)):
        ctx.set_precision(prec)
        if prec == 2:
            ctx.set_tune(tc_min=1, by_work=1)
        t0 = time.perf_counter()
        sig = ctx.hpsi(psi)  # builds task list + temporaries
        torch.cuda.synchronize()
        plan_s = time.perf_counter() - t0
        ctx.stats(reset=True)
        for _ in range(1 if prec == 0 else 3):
            sig = ctx.hpsi(psi)
        st = ctx.stats(reset=True)
        fl, tasks = ctx.hpsi_flops()
        ms = st["hpsi_ms"] / max(st["hpsi_calls"], 1)
        r = {"plan_s": plan_s, "launch_shape": ctx.get_tune(), "hpsi_ms": ms,
             "hpsi_tflops": fl / (ms * 1e-3) / 1e12, "gflop_per_hpsi": fl / 1e9, "tasks": tasks}
        sigs[name] = sig.double().cpu().numpy()
        ctx.set_position(k, 1)
        ctx.set_psi(psi)
        t0 = time.perf_counter()
        e, it = ctx.davidson_lowp(tol=1e-300, max_iter=1 if prec == 0 else iters, allow_noconv=True)
        torch.cuda.synchronize()
        r["davidson_s_per_iter"] = (time.perf_counter() - t0) / max(it, 1)
        r["davidson_hpsi"] = it
        out[name] = r
        print(json.dumps({name: r}), flush=True)
    for name in ("bf16x3", "fp32"):
        out[name]["rel_diff_vs_fp64"] = float(np.max(np.abs(sigs[name] - sigs["fp64"])) /
                                              np.max(np.abs(sigs["fp64"])))
    ctx.set_position(k, 1)
    ctx.set_psi(psi)
    t0 = time.perf_counter()
    ctx.renormalize(+1)
    torch.cuda.synchronize()
    out["renormalize_s"] = time.perf_counter() - t0
    ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="c5b", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the untimed FP32 / FP64 comparisons, the renormalization and the sub-line")
    ap.add_argument("--no-mixed", action="store_true", help="FP64 step mode: skip the mixed-precision runs")
    ap.add_argument("--fp64-step", action="store_true",
                    help="the FP64 step mode (Davidson to tol + renormalization, mixed runs beside it)")
    ap.add_argument("--profile-hpsi", type=int, default=0, metavar="N",
                    help="setup, then N H.psi calls in an NVTX range 'hpsi' (for ncu); no JSON line")
    ap.add_argument("--precision", default="bf16x3", choices=["fp64", "fp32", "bf16x3"])
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the default launch shape instead of timing candidates at plan time")
    ap.add_argument("--mixed-step", type=float, default=0.0, metavar="TOL",
                    help="one middle-bond step per precision to Davidson tolerance TOL (FP64 vs mixed)")
    ap.add_argument("--sweeps", type=int, default=0, metavar="S",
                    help="time S full sweeps from the start state per precision (instead of the step)")
    ap.add_argument("--tune", default="", metavar="T,MIN,TC,ORDER,WIDE",
                    help="fixed launch shape (target_chunks,min_chunk,tc_min,by_work,flat_wide[,tc_tiny]); no autotuning")
    ap.add_argument("--M", type=int, default=0, help="override the workload's bond dimension (profiling)")
    ap.add_argument("--refine-keep", type=int, default=0,
                    help="sweeps: Ritz vectors carried between mixed-precision refinement steps")
    ap.add_argument("--sweep-max-iter", type=int, default=200, help="sweeps: matvec cap of each Davidson step")
    ap.add_argument("--large", action="store_true",
                    help="middle-bond measurement of a large workload in every precision (JSON lines)")
    ap.add_argument("--renorm", default="fp64", choices=["fp64", "fp32"],
                    help="--large: arithmetic of the renormalizations that grow the bases")
    ap.add_argument("--M-right", type=int, default=0, help="--large: bond dimension of the right blocks")
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.M:
        wl["M"] = args.M
        wl["name"] = wl["name"].replace(f"M{WORKLOADS[args.workload]['M']}", f"M{args.M}")
        wl.pop("hpsi_flops", None)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        from oracle import baseline
        owl, oflops = _oracle_workload(wl)
        note = "" if owl["name"] == wl["name"] else (
            f"; the oracle cannot build the {wl['name']} blocks within host memory and time, so it is timed "
            f"on {owl['name']}")
        line = baseline.reference_line(owl, args.steps, args.warmup, METRIC, oflops, note)
        print(json.dumps(line))
        return 0
    prec = {"fp64": 0, "fp32": 1, "bf16x3": 2}[args.precision]
    if args.workload == "c4":
        print(json.dumps(batched_workload(args, wl)))
        return 0
    if args.large:
        print(json.dumps(large_workload(wl, args)))
        return 0
    if args.sweeps:
        print(json.dumps(sweep_workload(args, wl)))
        return 0
    if args.mixed_step:
        print(json.dumps(mixed_step_workload(args, wl, args.mixed_step)))
        return 0
    if args.profile_hpsi:
        profile_hpsi(wl, prec, args.profile_hpsi, args.autotune, args.tune)
        return 0
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    if args.fp64_step:
        line = fp64_step_line(args, wl, rank, world)
    else:
        line = davidson_line(args, wl, rank, world, prec)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:  # the oracle baseline at N = 1 only
        try:
            from oracle import baseline
            owl, oflops = _oracle_workload(wl)
            note = "" if owl["name"] == wl["name"] else (
                f"; the oracle cannot build the {wl['name']} blocks within host memory and time, so its "
                f"H.psi rate is measured on {owl['name']}")
            line["cpu_baseline"] = baseline.cpu_baseline(owl, oflops, note=note)
        except Exception as exc:  # reported, never silently replaced
            line["cpu_baseline"] = {"error": str(exc)}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()
    return 0


def davidson_line(args, wl, rank, world, prec):
    """The default JSON line: working-precision Davidson iterations at the middle bond."""
    r = run_davidson_bench(args, wl, rank, world, prec)
    st = r["stats"]
    K = args.steps
    value = whole_job_tflops(st["hpsi_flops"], world, r["step_ms"])
    kernel_tflops = st["hpsi_flops"] / (st["hpsi_ms"] * 1e-3) / 1e12 if st["hpsi_ms"] > 0 else None
    peaks = _peaks()
    if prec == 2:
        peak = peaks.get("bf16_tflops")
        roof = {"bound": "tensor", "kernel": "chain_tc2_kernel (H.psi, split-BF16 x3 on tcgen05)",
                "achieved": kernel_tflops, "peak": peak / 3.0 if peak else None,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst) / 3: three bf16 passes per product"
                               " (of measured)",
                "unit": "TFLOP/s"}
    else:
        roof = {"bound": "alu", "kernel": "chain kernels (SIMT)", "achieved": kernel_tflops,
                "peak": FP64_NOMINAL_TFLOPS if prec == 0 else FP32_SIMT_TFLOPS,
                "peak_source": "unit counts x 2.07 GHz (no measured SIMT peak)", "unit": "TFLOP/s"}
    roof["frac"] = (kernel_tflops / roof["peak"]) if (kernel_tflops and roof["peak"]) else None
    roof["traffic"] = TRAFFIC_PER_LAUNCH.get((args.workload, prec, wl["M"], _shape_key(r["tune"])))
    if prec == 2 and args.workload in ALG_BYTES and wl["M"] == WORKLOADS[args.workload]["M"]:
        roof["traffic_scope"] = "DRAM bytes of the chain_tc2 launches of one H.psi (ncu, one capture)"
        roof["algorithmic_bytes"] = ALG_BYTES[args.workload]
    hps = st["hpsi_calls"] / K
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "TFLOP/s",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": r["step_ms"] / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {0: "f64", 1: "f32", 2: "bf16x3"}[prec],
        "data": "synthetic",
        "config": {"workload": wl["name"], "L": wl["L"], "N": wl["N"], "two_sz": wl["two_sz"],
                   "M": wl["M"], "position": r["k"], "psi_dim": r["dim"], "hpsi_tasks": r["ntasks"],
                   "step": f"{DAVIDSON_ITERS_PER_STEP} working-precision Davidson iterations from a fixed "
                           f"start vector ({hps:g} H.psi per step)",
                   "l2": "flushed between timed steps (256 MB write)", "launch_shape": r["tune"],
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "davidson_s_per_iter": (r["step_ms"] * 1e-3) / max(st["hpsi_calls"], 1),
        "hpsi_per_step": hps,
        "hpsi_kernel_tflops": kernel_tflops,
        "hpsi_ms": st["hpsi_ms"] / max(st["hpsi_calls"], 1),
        "hpsi_gflop_per_call": r["flops_per_hpsi"] / 1e9,
        "hpsi_plan_s": r["plan_s"],
        "setup_s": r["setup_s"],
        "energy": r["energy"],
        "roofline": roof,
        "e2e": {"value": st["hpsi_flops"] / (r["e2e_ms"] * 1e-3) / 1e12, "unit": "TFLOP/s",
                "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"]},
        "gpu_launches": st["kernel_launches"],
        "clocks": r["clocks"],
        "cpu_baseline": None,
    }
    if r["extra"]:
        line["precisions"] = r["extra"]
    if rank == 0 and world == 1 and not args.no_extras:
        sub = argparse.Namespace(**vars(args))
        sub.steps, sub.warmup, sub.autotune, sub.tune = 2, 1, True, ""
        sl = fp64_step_line(sub, dict(WORKLOADS["c2"]), rank, world)
        line["c2_fp64_step"] = {k: sl[k] for k in ("value", "ms_per_step", "davidson_s_per_iter",
                                                   "davidson_iters_per_step", "hpsi_kernel_tflops",
                                                   "roofline", "energy", "mixed_fp32", "mixed_bf16x3", "config")
                                if k in sl}
    return line


def fp64_step_line(args, wl, rank, world):
    """The FP64 step: Davidson to tol from a fixed start + one renormalization, with the
    same step in the mixed precisions beside it (|dE| and overlap of the refined state)."""
    r = run_gpu(args, wl, rank, world, 0)
    st = r["stats"]
    K = args.steps
    hpsi_flops = st["hpsi_flops"]
    value = whole_job_tflops(hpsi_flops, world, r["step_ms"])
    kernel_tflops = st["hpsi_flops"] / (st["hpsi_ms"] * 1e-3) / 1e12 if st["hpsi_ms"] > 0 else None
    dav_iters = st["davidson_iters"]
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "TFLOP/s",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": r["step_ms"] / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl["name"], "L": wl["L"], "N": wl["N"], "two_sz": wl["two_sz"],
                   "M": wl["M"], "position": r["k"], "psi_dim": r["dim"], "hpsi_tasks": r["ntasks"],
                   "davidson_tol": wl["tol"], "l2": "flushed between timed steps (256 MB write)",
                   "launch_shape": r["tune"],
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "davidson_s_per_iter": (r["step_ms"] * 1e-3) / max(dav_iters, 1),
        "davidson_iters_per_step": dav_iters / K,
        "hpsi_kernel_tflops": kernel_tflops,
        "hpsi_gflop_per_call": r["flops_per_hpsi"] / 1e9,
        "hpsi_plan_s": r["plan_s"],
        "energy": r["energy"],
        "roofline": {
            "bound": "alu",
            "kernel": "chain_flat_kernel<double> (H.psi)",
            "achieved": kernel_tflops,
            "peak": FP64_NOMINAL_TFLOPS,
            "peak_source": "nominal GB300 FP64 from the recipe table (no measured FP64 peak in MEASURED_PEAKS.json)",
            "unit": "TFLOP/s",
            "frac": (kernel_tflops / FP64_NOMINAL_TFLOPS) if kernel_tflops else None,
            "traffic": TRAFFIC_PER_LAUNCH.get((wl.get("key", ""), 0, wl["M"], _shape_key(r["tune"]))),
        },
        "e2e": {"value": hpsi_flops / (r["e2e_ms"] * 1e-3) / 1e12, "unit": "TFLOP/s",
                "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"]},
        "gpu_launches": st["kernel_launches"],
        "clocks": r["clocks"],
        "cpu_baseline": None,
    }
    if not args.no_mixed:
        for key, lp, what in (
                ("mixed_fp32", 1, "FP32 operator copies for the Davidson matvecs"),
                ("mixed_bf16x3", 2, "split-BF16x3 tensor-core matvecs (FP32 SIMT below the routing threshold)")):
            m = run_gpu(args, wl, rank, world, lp, e2e=False, sample_clocks=False)
            ms = m["stats"]
            line[key] = {
                "what": f"same step with {what}, then the FP64 defect-corrected refinement to the same "
                        "tolerance; FP64 renormalization and density matrix",
                "value": ms["hpsi_flops"] / (m["step_ms"] * 1e-3) / 1e12,
                "ms_per_step": m["step_ms"] / K,
                "speedup_vs_fp64_step": r["step_ms"] / m["step_ms"],
                "davidson_iters_per_step": ms["davidson_iters"] / K,
                "lowp_matvec_iters_per_step": ms["davidson_iters_lowp"] / K,
                "launch_shape": m["tune"],
                "hpsi_plan_s": m["plan_s"],
                "abs_dE_vs_fp64": abs(m["e_mid"] - r["e_mid"]),
                "overlap_vs_fp64": float(abs(np.dot(m["psi_mid"], r["psi_mid"]))),
                "energy": m["e_mid"],
            }
    return line


if __name__ == "__main__":
    sys.exit(main())
