#!/usr/bin/env python
"""PnP-ADMM reconstruction throughput on GB300 (voxel-iterations per second).

Workload (one "step"): 64 independent coded measurements of uneven size
(H = W in {256, 512, 768, 1024}, Z in {8, 16, 32} slices, drawn with seed
4000; 614 M voxels in all) reconstructed by 60 iterations of Algorithm 1 with
the TV prior and the z-smoothness Gauss-Seidel sweep (rho = 1, lambda = 0.05,
gamma = 0.2, 20 Chambolle steps per prox), all of them in ONE persistent
launch replayed from a CUDA graph (the batched solver), iterates u, d, w
stored in BF16 with FP32 arithmetic.  A step re-packs every item's DMD
patterns and runs the batch through the C ABI.  Inputs are seeded synthetic
data (drifting Gaussian blobs, Bernoulli(0.3) patterns, Poisson peak 50 +
Gaussian 0.02).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME]

N > 1 runs under torchrun, one independent batch per rank (weak scaling, no
data-path collective).  --impl reference times the FP64 CPU oracle on a
stratified 8-item sample of the batch (bounded iterations) on the host cores.
--workload runs one of the other configurations instead (one JSON line).
"""
from __future__ import annotations

import argparse
import atexit
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "batched_64"
PARAMS = dict(rho=1.0, lam=0.05, gamma=0.2, iters=60, denoiser="tv", tv_inner=20,
              tv_tau=0.125, storage="bf16")
# the single-volume 512 x 512 x 16 configuration (a secondary workload)
PARAMS_TVZ = dict(rho=1.0, lam=0.05, gamma=0.2, iters=100, denoiser="tv", tv_inner=20,
                  tv_tau=0.125)
METRIC = "PnP-ADMM voxel-iterations/s"
UNIT = "voxel-it/s"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2
DOMINANT = "batch_persistent"  # one launch = the whole 60-iteration batch
BATCH_PROFILE_K = 7  # steps per phase of the 8-item profiling case (see batched_8x6)
DOMINANT_SOURCES = ("kernels_batch.cu", "tv_body.cuh", "storage.cuh")
TVZ_DOMINANT = "tvz_sweep"  # the single-volume configuration's dominant kernel
TVZ_SOURCES = ("kernels_tvz.cu", "tv_body.cuh", "storage.cuh")
TIMING_PERIOD = 1  # every launch of each kernel timed with CUDA events
ORACLE_SAMPLE_ITERS = 2  # bounded CPU sample: ADMM iterations per sampled item


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def _config(world: int, voxels: int) -> dict:
    return {"workload": f"{WORKLOAD}: 64 independent measurements, H = W in "
                        "{256,512,768,1024} x Z in {8,16,32} (seed 4000), TV + z-smoothness "
                        f"PnP-ADMM, {PARAMS['iters']} iterations, {PARAMS['tv_inner']} TV steps, "
                        "one persistent launch under a CUDA graph",
            "items": 64, "voxels": voxels, "iterations": PARAMS["iters"],
            "tv_inner": PARAMS["tv_inner"], "rho": PARAMS["rho"], "lambda": PARAMS["lam"],
            "gamma": PARAMS["gamma"], "storage": "bf16 iterates (u, d, w), fp32 arithmetic",
            "l2": "inputs larger than L2 (2.5 GB per field) and L2 flushed between steps",
            "parallelism": f"replicas x{world}"}


def _config_tvz(world: int) -> dict:
    return {"workload": "tvz_512x512x16: TV + z-smoothness PnP-ADMM, 512x512x16, "
                        f"{PARAMS_TVZ['iters']} iterations, {PARAMS_TVZ['tv_inner']} TV steps",
            "volume": [16, 512, 512], "iterations": PARAMS_TVZ["iters"],
            "tv_inner": PARAMS_TVZ["tv_inner"], "rho": PARAMS_TVZ["rho"],
            "lambda": PARAMS_TVZ["lam"], "gamma": PARAMS_TVZ["gamma"],
            "l2": "flushed between steps (512 MiB write)", "parallelism": f"replicas x{world}"}


def tv_flops_per_launch(H: int, W: int, T: int) -> float:
    """Algorithmic FP32 operations of one single-slice TV-prox launch.

    Per pixel and Chambolle step: q = div p - g/theta (5), grad q (2),
    |grad q| (3 + sqrt = 4), 1 + tau|.| (2), two p updates (2 x 3) = 19;
    per pixel once: g from w and the two z neighbours (5) and
    u = g - theta div p with d = w - u (6) = 11.
    """
    return float(H * W) * (19.0 * T + 11.0)


def tv_stream_bytes(R: int, T: int, z_term: bool) -> float:
    """Bytes per voxel and ADMM iteration of the TV path executed as streaming
    HBM passes (one pass per Chambolle step, FP32, R slices per shot): the
    x-update reads u, d, b, the pattern word and writes w (12.125 + 4 / R), the
    first prox pass reads w and writes p (12), every later pass reads p and
    writes it (20), the final pass forms u and d (20); with the z term the prox
    input also reads u_{n-1} and u_{n+1} (8)."""
    return 44.125 + 4.0 / R + 20.0 * (T - 1) + (8.0 if z_term else 0.0)


def alu_peak_tflops(sm_mhz: float) -> float:
    """FP32 FMA peak: 152 SMs x 128 lanes x 2 flops x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def _kernel_hash(sources=DOMINANT_SOURCES) -> str:
    h = hashlib.sha256()
    for f in sources:
        h.update(open(os.path.join(ROOT, "paper_2511_03093_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def _record(kernel: str, workload: str, sources) -> dict:
    """A kernel's committed ncu record, if it was taken on the kernel's sources
    as they are now; else an empty record."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.json")
    try:
        rec = json.load(open(p))
    except (OSError, ValueError):
        return {}
    if rec.get("sources_sha256_16") != _kernel_hash(sources):
        return {}
    return rec


def _traffic(kernel: str, workload: str, sources) -> float | None:
    """DRAM bytes per launch of a kernel from its committed ncu record."""
    return _record(kernel, workload, sources).get("dram_bytes_per_launch")


def _l2(kernel: str, workload: str, sources, avg_launch_s: float) -> dict | None:
    """L2 throughput of a kernel whose working set is L2-resident: the L2 bytes
    per launch of its ncu record over the launch time measured in this run,
    against the L2 sector peak of the same record."""
    rec = _record(kernel, workload, sources)
    if "l2_bytes_per_launch" not in rec or avg_launch_s <= 0:
        return None
    gbs = rec["l2_bytes_per_launch"] / avg_launch_s / 1e9
    return {"bytes_per_launch": rec["l2_bytes_per_launch"], "achieved": gbs, "unit": "GB/s",
            "peak": rec["l2_peak_GBs"], "frac": gbs / rec["l2_peak_GBs"],
            "hit_rate_pct": rec.get("l2_sector_hit_rate_pct"),
            "source": "L2 bytes from ncu (lts__t_sectors x 32 B), launch time from this run"}


def _quality(cs, v, data, dev):
    """PSNR and 3-D SSIM (Sec. IV) of the last solve's v^K against the synthetic
    ground truth, both computed by the library's kernels outside the timed region."""
    import torch

    x = torch.from_numpy(data["x"].astype("float32")).to(dev)
    return {"psnr_db": float(cs.psnr(v, x)), "ssim3d": float(cs.ssim3d(v, x))}


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.proc = None
        # raw samples: BENCH_CLOCKS_DIR if set, else the system temporary directory
        out_dir = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"cslsm_clocks_{os.getpid()}.csv")
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "50"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        if self.proc is not None:
            atexit.register(self._end)  # no sampler outlives the bench, even on an error

    def _end(self) -> None:
        if self.proc is not None and self.proc.poll() is None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def window(self, t0: float, t1: float) -> None:
        """Host wall-clock bounds (time.time()) of the timed region."""
        self.t0, self.t1 = t0, t1

    def stop(self):
        if self.proc is None:
            return None
        self._end()
        self.f.close()
        return summarize_clocks(open(self.path).read().splitlines(),
                                getattr(self, "t0", None), getattr(self, "t1", None))


def start_clocks(dev):
    """A clock sampler on the GPU of `dev`.  Callers start it early (before the
    inputs are built): the first nvidia-smi start on a box can take seconds,
    and only the samples inside the timed region are summarised."""
    import torch

    gpu_id = None
    try:
        gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
        if gpu_id and not gpu_id.startswith("GPU-"):
            gpu_id = "GPU-" + gpu_id
    except Exception:
        gpu_id = None
    return ClockSampler(gpu_id)


def summarize_clocks(lines, t0=None, t1=None):
    """Median SM clock, max clock and the throttle reasons seen, over the samples
    taken inside [t0, t1] (host wall clock; every sample if none falls inside)."""
    import datetime

    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    rows = []
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm, sm_max = float(parts[1]), float(parts[2])
        except ValueError:
            continue
        try:
            ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            ts = None  # unknown timestamp format: the sample still counts overall
        rows.append((ts, sm, sm_max, parts[5:9]))
    if not rows:
        return None
    inside = [r for r in rows if t0 is not None and r[0] is not None and t0 <= r[0] <= t1]
    use = inside or rows
    reasons = sorted({names[i] for _, _, _, r in use for i, x in enumerate(r)
                      if x.lower() == "active"})
    return {"sm_mhz": statistics.median(s for _, s, _, _ in use),
            "sm_max_mhz": max(m for _, _, m, _ in use), "reasons": reasons,
            "samples": len(use), "samples_in_timed_region": len(inside)}


def rank_workload(rank: int):
    """The single-volume configuration: each rank its own measurement."""
    import dataclasses

    import synth

    w = synth.WORKLOADS["tvz_512x512x16"]
    return dataclasses.replace(w, seed=w.seed + 100 * rank) if rank else w


def rank_workloads(rank: int):
    """Each rank reconstructs its own independent batch (replicas): seed 4000
    for rank 0, 4000 + 1000 r for rank r."""
    import synth

    return synth.batch_workloads(seed=4000 + 1000 * rank)


def _gen_compact(w):
    """One batch item's inputs, as the bench keeps them (float32 ground truth)."""
    import synth

    d = synth.generate(w)
    return {"x": d["x"].astype("float32"), "masks": d["masks"], "b": d["b"]}


def _gen_items(ws):
    """Generates the items in a process pool started with spawn (independent of
    any CUDA state of this process)."""
    import multiprocessing as mp

    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 4)) as pool:
        return pool.map(_gen_compact, ws)


def oracle_sample(ws) -> list[int]:
    """8 items stratified by size: the items are ordered by voxel count (then
    index) and the middle item of each eighth is taken."""
    order = sorted(range(len(ws)), key=lambda i: (ws[i].Z * ws[i].H * ws[i].W, i))
    n = len(order)
    return [order[(2 * k + 1) * n // 16] for k in range(8)]


def max_over_ranks(values, world: int, device=None):
    """Element-wise max of per-rank timings (the slowest rank sets the job time)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def job_throughput(units_per_rank: float, world: int, max_ms: float) -> float:
    """Whole-job voxel-iterations per second: all ranks' units over the slowest time."""
    return units_per_rank * world / (max_ms / 1e3)


def cpu_baseline_tvz(data, iters: int) -> dict:
    import oracle

    t0 = time.perf_counter()
    oracle.admm(data["b64"], data["masks"], 16, rho=PARAMS_TVZ["rho"], lam=PARAMS_TVZ["lam"],
                gamma=PARAMS_TVZ["gamma"], iters=iters, denoiser="tv",
                tv_inner=PARAMS_TVZ["tv_inner"], tv_tau=PARAMS_TVZ["tv_tau"])
    dt = time.perf_counter() - t0
    vox = data["masks"].size
    return {"value": vox * iters / dt, "unit": UNIT, "cores": _omp_threads(), "kind": "oracle",
            "sample": f"FP64 oracle, {iters} ADMM iterations of the 512x512x16 TV + z solve "
                      f"({dt:.1f} s)"}


def oracle_batch_sample(ws, datas, idx, iters: int) -> tuple[float, int]:
    """Runs the FP64 oracle (Algorithm 1, TV + z) for `iters` iterations on each
    sampled item; returns (seconds, voxel-iterations)."""
    import numpy as np

    import oracle

    t0 = time.perf_counter()
    units = 0
    for i, d in zip(idx, datas):
        w = ws[i]
        oracle.admm(d["b"].astype(np.float64), d["masks"], w.Z, rho=PARAMS["rho"],
                    lam=PARAMS["lam"], gamma=PARAMS["gamma"], iters=iters, denoiser="tv",
                    tv_inner=PARAMS["tv_inner"], tv_tau=PARAMS["tv_tau"])
        units += w.Z * w.H * w.W * iters
    return time.perf_counter() - t0, units


def cpu_baseline(ws, datas) -> dict:
    """The oracle on the stratified 8-item sample (datas: all items)."""
    idx = oracle_sample(ws)
    dt, units = oracle_batch_sample(ws, [datas[i] for i in idx], idx, ORACLE_SAMPLE_ITERS)
    return {"value": units / dt, "unit": UNIT, "cores": _omp_threads(), "kind": "oracle",
            "sample": f"FP64 oracle, {ORACLE_SAMPLE_ITERS} of {PARAMS['iters']} ADMM iterations "
                      f"(FP64 state) of 8 items stratified by size (items {idx}, "
                      f"{units / ORACLE_SAMPLE_ITERS / 1e6:.1f} M voxels; {dt:.1f} s)"}


def _omp_threads() -> int:
    return int(os.environ.get("OMP_NUM_THREADS", len(os.sched_getaffinity(0))))


def run_reference(args) -> None:
    """The FP64 CPU oracle as the reference arm (rank 0 only): each step runs the
    oracle on the batch's stratified 8-item sample for a bounded number of
    iterations."""
    if _env_int("RANK", 0) != 0:
        return
    ws = rank_workloads(0)
    idx = oracle_sample(ws)
    datas = _gen_items([ws[i] for i in idx])
    import oracle

    oracle.lib()

    def step():
        return oracle_batch_sample(ws, datas, idx, ORACLE_SAMPLE_ITERS)

    for _ in range(args.warmup):
        step()
    runs = [step() for _ in range(args.steps)]
    total = sum(t for t, _ in runs)
    units = sum(u for _, u in runs)
    value = units / total
    sample = (f"FP64 oracle, {ORACLE_SAMPLE_ITERS} of {PARAMS['iters']} ADMM iterations of 8 "
              f"items stratified by size (items {idx}) per step")
    vox = sum(w.Z * w.H * w.W for w in ws)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": _config(1, vox),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": _omp_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def run_ours(args) -> None:
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    ws = rank_workloads(rank)
    datas = _gen_items(ws)  # host-side generation before any CUDA call

    import paper_2511_03093_gb300 as cs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    cs.lib()
    clocks = start_clocks(dev) if rank == 0 else None

    n = len(ws)
    vox = sum(w.Z * w.H * w.W for w in ws)
    masks_h = [torch.from_numpy(d["masks"]).pin_memory() for d in datas]
    b_h = [torch.from_numpy(d["b"]).pin_memory() for d in datas]
    v_h = [torch.empty((w.Z, w.H, w.W), dtype=torch.float32).pin_memory() for w in ws]
    masks_d = [m.to(dev) for m in masks_h]
    b_d = [b.to(dev) for b in b_h]
    v_d = [torch.empty((w.Z, w.H, w.W), dtype=torch.float32, device=dev) for w in ws]
    plans = [cs.Plan(w.H, w.W, 1, w.Z, m) for w, m in zip(ws, masks_d)]
    items = list(zip(plans, b_d, v_d))
    cs.set_autotune(1)  # steps per phase timed on the batch itself at creation
    prm = cs.Params(**PARAMS)
    batch = cs.Batch(items, prm)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        for plan, m in zip(plans, masks_d):
            plan.set_masks(m)
        batch.run()

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(max(args.warmup, 0)):
        step()
    batch.wait()
    # first touch of the pinned output buffers (page allocation, once) belongs to
    # setup, not to a step: one read-back of the warm-up result
    for i in range(n):
        v_h[i].copy_(v_d[i], non_blocking=True)
    torch.cuda.synchronize()

    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    cs.timing_read(DOMINANT, reset=True)
    barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    n0 = cs.launch_count()
    cs.timing_enable(TIMING_PERIOD)
    for k in range(args.steps):
        flush.zero_()
        ev_s[k].record(stream)
        step()
        ev_e[k].record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    barrier()
    cs.timing_enable(0)
    launches = cs.launch_count() - n0
    batch.wait()  # raises if a device-side wait ran out
    if clocks:
        clocks.window(t_wall0, t_wall1)
    clk = clocks.stop() if clocks else None
    step_ms = [ev_s[k].elapsed_time(ev_e[k]) for k in range(args.steps)]
    total_ms = sum(step_ms)
    n_dom, ms_dom = cs.timing_read(DOMINANT, reset=True)

    # end to end through the public API: every item's patterns and measurement
    # copied in from pinned host memory, every reconstruction copied back
    e2e_ms = []
    for k in range(args.steps):
        flush.zero_()
        s_ev, e_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s_ev.record(stream)
        for i in range(n):
            masks_d[i].copy_(masks_h[i], non_blocking=True)
            b_d[i].copy_(b_h[i], non_blocking=True)
        step()
        for i in range(n):
            v_h[i].copy_(v_d[i], non_blocking=True)
        e_ev.record(stream)
        e_ev.synchronize()
        e2e_ms.append(s_ev.elapsed_time(e_ev))
    batch.wait()
    e2e_total = sum(e2e_ms)

    total_ms, e2e_total = max_over_ranks([total_ms, e2e_total], world, dev)
    units = vox * PARAMS["iters"] * args.steps
    value = job_throughput(units, world, total_ms)
    e2e_value = job_throughput(units, world, e2e_total)

    if rank == 0:
        peaks = _peaks()
        roof = None
        if n_dom:
            avg_s = ms_dom / n_dom / 1e3
            bytes_launch = PARAMS["iters"] * sum(
                w.Z * w.H * w.W * tv_stream_bytes(w.Z, PARAMS["tv_inner"], True) for w in ws)
            achieved = bytes_launch / avg_s / 1e9
            tr = _traffic(DOMINANT, WORKLOAD, DOMINANT_SOURCES)
            roof = {"bound": "hbm", "kernel": DOMINANT, "achieved": achieved,
                    "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                    "traffic": tr, "bytes_per_launch": bytes_launch,
                    "avg_launch_us": avg_s * 1e6, "launches_timed": n_dom,
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy, burst)",
                    "model": "streaming TV + z prox (one HBM pass per Chambolle step, FP32): "
                             "44.125 + 4/R + 20 (T - 1) + 8 B per voxel-iteration, per item",
                    "share_of_step": ms_dom / total_ms}
            if tr:
                roof["traffic_per_voxel_it_B"] = tr / (vox * PARAMS["iters"])
                roof["traffic_GBs"] = tr / avg_s / 1e9
            # the same launch against the FP32 ALU: the algorithmic operations of the
            # x-update-free TV + z prox (19 per pixel and step + 11 per pixel), the
            # view for a kernel whose data stays on chip
            fl = PARAMS["iters"] * sum(w.Z * tv_flops_per_launch(w.H, w.W, PARAMS["tv_inner"])
                                       for w in ws)
            alu_peak = alu_peak_tflops((clk or {}).get("sm_max_mhz") or 2070.0)
            roof["alu_view"] = {"achieved": fl / avg_s / 1e12, "peak": alu_peak,
                                "unit": "TFLOP/s", "frac": fl / avg_s / 1e12 / alu_peak,
                                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock"}
        # the comparison the metric names: plain per-volume FP32 solves of the same
        # items, and the batch with FP32 state, each run once (not in the timed region)
        x_d = [torch.from_numpy(d["x"]).to(dev) for d in datas]
        ps_batch = [float(cs.psnr(v, x)) for v, x in zip(v_d, x_d)]
        plain = cs.Params(**dict(PARAMS, storage="fp32"))
        v_p = [torch.empty_like(v) for v in v_d]
        for plan, b, v in zip(plans, b_d, v_p):  # warm-up of the per-volume path
            plan.solve(b, plain, v_out=v)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for plan, b, v in zip(plans, b_d, v_p):
            plan.solve(b, plain, v_out=v)
        e1.record(stream)
        e1.synchronize()
        plain_ms = e0.elapsed_time(e1)
        ps_plain = [float(cs.psnr(v, x)) for v, x in zip(v_p, x_d)]
        batch32 = cs.Batch(list(zip(plans, b_d, v_p)), plain)
        batch32.run()
        batch32.wait()
        e0.record(stream)
        batch32.run()
        e1.record(stream)
        e1.synchronize()
        b32_ms = e0.elapsed_time(e1)
        batch32.wait()
        ps_b32 = [float(cs.psnr(v, x)) for v, x in zip(v_p, x_d)]
        sched32 = batch32.info()
        batch32.close()
        cpu = cpu_baseline(ws, datas) if world == 1 else None
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded Gaussian-blob volumes, Bernoulli DMD masks)",
            "config": _config(world, vox), "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(sum(m.numel() + b.numel() * 4
                                                  for m, b in zip(masks_h, b_h))),
                    "d2h_bytes_per_step": int(sum(v.numel() * 4 for v in v_h))},
            "gpu_launches": int(launches), "clocks": clk,
            "step_ms": [round(x, 3) for x in step_ms],
            "e2e_step_ms": [round(x, 3) for x in e2e_ms],
            "vs_plain": {"plain_fp32_ms": plain_ms,
                         "plain_fp32_value": vox * PARAMS["iters"] / (plain_ms / 1e3),
                         "batched_fp32_ms": b32_ms,
                         "batched_fp32_value": vox * PARAMS["iters"] / (b32_ms / 1e3),
                         "speedup_bf16_vs_plain_fp32": plain_ms / (total_ms / args.steps),
                         "max_dpsnr_bf16_vs_plain_fp32_db": max(abs(a - b) for a, b in
                                                                zip(ps_batch, ps_plain)),
                         "max_dpsnr_fp32_batched_vs_plain_db": max(abs(a - b) for a, b in
                                                                   zip(ps_b32, ps_plain)),
                         "batched_fp32_schedule": sched32},
            "schedule": batch.info(),
            "quality": {"psnr_db_mean": float(np.mean(ps_batch)),
                        "psnr_db_min": float(np.min(ps_batch))},
        }
        bm = statistics.fmean(tv_stream_bytes(w.Z, PARAMS["tv_inner"], True) for w in ws)
        out["hbm_roofline_model"] = {
            "bytes_per_voxel_it": bm, "equivalent_GBs": value / world * bm / 1e9,
            "peak_GBs": peaks["hbm_gbs"], "frac": value / world * bm / 1e9 / peaks["hbm_gbs"],
            "model": "streaming TV + z prox, one HBM pass per Chambolle step (mean over items)"}
        print(json.dumps(out), flush=True)
    batch.close()
    for plan in plans:
        plan.close()
    if world > 1:
        dist.destroy_process_group()


def run_tvz(args) -> None:
    """The single-volume configuration (512 x 512 x 16, 100 iterations) with the
    same line layout as the default bench."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    import paper_2511_03093_gb300 as cs

    rank, world = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    cs.lib()
    clocks = start_clocks(dev) if rank == 0 else None

    w = rank_workload(rank)
    data = synth.generate(w)
    prm = cs.Params(**PARAMS_TVZ)
    vox = w.Z * w.H * w.W
    masks_h = torch.from_numpy(data["masks"]).pin_memory()
    b_h = torch.from_numpy(data["b"]).pin_memory()
    v_h = torch.empty((w.Z, w.H, w.W), dtype=torch.float32).pin_memory()
    masks_d = masks_h.to(dev)
    b_d = b_h.to(dev)
    v_d = torch.empty((w.Z, w.H, w.W), dtype=torch.float32, device=dev)
    plan = cs.Plan(w.H, w.W, 1, w.Z, masks_d)
    cs.set_autotune(1)  # the warm-up steps time the TV kernel variants once
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        plan.set_masks(masks_d)
        plan.solve(b_d, prm, v_out=v_d)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(max(args.warmup, 0)):
        step()
    v_h.copy_(v_d, non_blocking=True)  # first touch of the pinned output: setup
    torch.cuda.synchronize()

    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    cs.timing_read(TVZ_DOMINANT, reset=True)

    barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    n0 = cs.launch_count()
    cs.timing_enable(4)
    for k in range(args.steps):
        flush.zero_()
        ev_s[k].record(stream)
        step()
        ev_e[k].record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    barrier()
    cs.timing_enable(0)
    launches = cs.launch_count() - n0
    if clocks:
        clocks.window(t_wall0, t_wall1)
    clk = clocks.stop() if clocks else None
    step_ms = [ev_s[k].elapsed_time(ev_e[k]) for k in range(args.steps)]
    total_ms = sum(step_ms)
    n_dom, ms_dom = cs.timing_read(TVZ_DOMINANT, reset=True)

    # end to end through the public API: host inputs in, host result out
    e2e_ms = []
    for k in range(args.steps):
        flush.zero_()
        s_ev, e_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s_ev.record(stream)
        masks_d.copy_(masks_h, non_blocking=True)
        b_d.copy_(b_h, non_blocking=True)
        step()
        v_h.copy_(v_d, non_blocking=True)
        e_ev.record(stream)
        e_ev.synchronize()
        e2e_ms.append(s_ev.elapsed_time(e_ev))
    e2e_total = sum(e2e_ms)

    total_ms, e2e_total = max_over_ranks([total_ms, e2e_total], world, dev)
    units = vox * PARAMS_TVZ["iters"] * args.steps
    value = job_throughput(units, world, total_ms)
    e2e_value = job_throughput(units, world, e2e_total)

    if rank == 0:
        sm_max = (clk or {}).get("sm_max_mhz") or 2070.0
        roof = None
        if n_dom:
            avg_s = ms_dom / n_dom / 1e3
            # the dominant kernel's launches per solve: one per iteration, or one
            # for the whole solve; its TV work per launch follows
            per_step = n_dom * 4 / args.steps
            achieved = (PARAMS_TVZ["iters"] * w.Z * tv_flops_per_launch(w.H, w.W, PARAMS_TVZ["tv_inner"])
                        / per_step / avg_s / 1e12)
            peak = alu_peak_tflops(sm_max)
            roof = {"bound": "alu", "kernel": TVZ_DOMINANT, "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak, "traffic": _traffic(TVZ_DOMINANT, "tvz_512x512x16", TVZ_SOURCES),
                    "avg_launch_us": avg_s * 1e6, "launches_timed": n_dom,
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock",
                    "share_of_step": ms_dom * 4 / total_ms}
            # the working set (16.8 MB per field) is L2-resident: report L2 throughput
            roof["l2"] = _l2(TVZ_DOMINANT, "tvz_512x512x16", TVZ_SOURCES, avg_s)
        cpu = cpu_baseline_tvz(data, PARAMS_TVZ["iters"]) if world == 1 or rank == 0 else None
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded Gaussian-blob volumes, Bernoulli DMD masks)",
            "config": _config_tvz(world), "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(masks_h.numel() + b_h.numel() * 4),
                    "d2h_bytes_per_step": int(v_h.numel() * 4)},
            "gpu_launches": int(launches), "clocks": clk,
            "zsweep_shape": cs.zsweep_shape(w.H, w.W, w.Z, PARAMS_TVZ["tv_inner"]),
            "step_ms": [round(x, 3) for x in step_ms],
            "e2e_step_ms": [round(x, 3) for x in e2e_ms],
            "quality": _quality(cs, v_d, data, dev),
        }
        # the metric's "% HBM roofline": voxel-iterations/s times the bytes the
        # TV path would move as streaming passes, over the measured HBM peak.
        # This solver keeps the prox on chip (its kernel roofline is "roofline");
        # the figure says how far the whole step runs ahead of an unfused one.
        peaks = _peaks()
        bm = tv_stream_bytes(w.Z, PARAMS_TVZ["tv_inner"], True)
        out["hbm_roofline_model"] = {
            "bytes_per_voxel_it": bm, "equivalent_GBs": value / world * bm / 1e9,
            "peak_GBs": peaks["hbm_gbs"], "frac": value / world * bm / 1e9 / peaks["hbm_gbs"],
            "model": "streaming TV prox, one HBM pass per Chambolle step"}
        print(json.dumps(out), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


# ---- secondary workloads (the other configurations of the method) -------------
# Not the default line: `python bench.py --workload NAME` prints one JSON line.

def _timed(fn, steps, warmup, flush):
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return ms


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "source": "fallback"}


def _gen(args):
    import synth

    return synth.generate(synth.Workload(*args[:4], **args[4]))


def run_secondary(args) -> None:
    import numpy as np
    import torch

    import oracle
    import paper_2511_03093_gb300 as cs
    import synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    name = args.workload
    out = {"workload": name, "steps": args.steps, "warmup": args.warmup}
    peaks = _peaks()
    if name == "tvz_512x512x16":
        run_tvz(args)
        return
    known = ("batched_8x6", "tikhonov_1024x1024x32", "tikhonovz_1024x1024x32", "tv_1024x1024x32",
             "tv_tiles_1024x1024x32",
             "bm3d_1024x1024x32", "tv_128x128x8", "unrolled_b8", "unrolled_b1",
             "wnnm_512x512x16", "tol_caps_512x512x16", "cr_sweep_256x256x40")
    if name not in known:
        raise SystemExit(f"unknown workload {name}")
    # clocks and throttle reasons over the whole workload (the warm-up included)
    clocks = start_clocks(dev)
    t_start = time.time()
    if name in ("tikhonov_1024x1024x32", "tikhonovz_1024x1024x32", "tv_1024x1024x32",
                "tv_tiles_1024x1024x32", "bm3d_1024x1024x32", "tv_128x128x8"):
        # tv_tiles_*: the same TV solve held on the per-launch tile kernel
        cs.set_tv_route(1 if name.startswith("tv_tiles") else 0)
        wk = synth.WORKLOADS["tv_128x128x8" if name == "tv_128x128x8" else "bm3d_1024x1024x32"]
        data = synth.generate(wk)
        den = name.split("_")[0]
        if name.startswith("tv_tiles"):
            out["path"] = "per-launch TV tiles (cslsm_set_tv_route(1))"
        gam = 0.2 if den == "tikhonovz" else 0.0  # Tikhonov with the z term (Sec. III-C)
        den = "tikhonov" if den == "tikhonovz" else den
        iters = 50 if name == "tv_128x128x8" else 30
        prm = cs.Params(rho=1.0, lam=0.0 if den == "bm3d" else 0.05, gamma=gam, iters=iters,
                        denoiser=den, tv_inner=20, bm3d_sigma=0.05)
        plan = cs.Plan(wk.H, wk.W, 1, wk.Z, torch.from_numpy(data["masks"]).to(dev))
        b = torch.from_numpy(data["b"]).to(dev)
        v = torch.empty((wk.Z, wk.H, wk.W), dtype=torch.float32, device=dev)
        cs.set_autotune(1)
        # TV: large slice-independent solves run as a one-item persistent batch
        # (the library's route), the others as per-launch tiles
        doms = {"tikhonov": ("tikhonov_iter",), "tv": ("tv_tile", DOMINANT),
                "bm3d": ("bm3d_match",)}[den]
        cs.timing_read(doms[0], reset=True)
        steps = max(1, args.steps if den != "bm3d" else min(args.steps, 2))
        warm = max(1, args.warmup if den != "bm3d" else 1)
        ms_w = _timed(lambda: plan.solve(b, prm, v_out=v), warm, 0, flush)
        cs.timing_read(doms[0], reset=True)
        cs.timing_enable(1)
        ms = _timed(lambda: plan.solve(b, prm, v_out=v), steps, 0, flush)
        cs.timing_enable(0)
        # read every candidate first: a read with reset clears all kernels' records
        reads = {d_: cs.timing_read(d_, reset=False) for d_ in doms}
        cs.timing_read(doms[0], reset=True)
        dom = max(doms, key=lambda d_: reads[d_][1])
        n_dom, ms_dom = reads[dom]
        vox = wk.Z * wk.H * wk.W
        out.update(metric=METRIC, unit=UNIT, value=vox * iters / (sum(ms) / steps / 1e3),
                   ms_per_step=sum(ms) / steps, iterations=iters, dominant=dom,
                   dominant_share=ms_dom / sum(ms), psnr_db=oracle.psnr(v.double().cpu().numpy(),
                                                                        data["x"]))
        if den == "tikhonov":
            R = wk.Z
            bytes_launch = vox * (16.0 + 8.0 / R)
            avg = ms_dom / n_dom / 1e3
            out["roofline"] = {"bound": "hbm", "kernel": dom, "achieved": bytes_launch / avg / 1e9,
                               "peak": peaks["hbm_gbs"], "unit": "GB/s",
                               "frac": bytes_launch / avg / 1e9 / peaks["hbm_gbs"],
                               "bytes_per_launch": bytes_launch, "avg_launch_us": avg * 1e6}
        elif den == "tv" and dom == DOMINANT:
            # one launch = the whole solve; the streaming model of the prox as the
            # headline counts it, against the measured HBM copy bandwidth
            avg = ms_dom / n_dom / 1e3
            bytes_launch = vox * iters * tv_stream_bytes(wk.Z, 20, False)
            out["roofline"] = {"bound": "hbm", "kernel": dom, "achieved": bytes_launch / avg / 1e9,
                               "peak": peaks["hbm_gbs"], "unit": "GB/s",
                               "frac": bytes_launch / avg / 1e9 / peaks["hbm_gbs"],
                               "bytes_per_launch": bytes_launch, "avg_launch_us": avg * 1e6,
                               "model": "streaming TV prox, one HBM pass per Chambolle step"}
            out["path"] = "one-item persistent batch (cslsm_set_tv_route)"
        elif den == "tv":
            avg = ms_dom / n_dom / 1e3
            fl = tv_flops_per_launch(wk.H, wk.W, 20) * wk.Z
            out["roofline"] = {"bound": "alu", "kernel": dom, "achieved": fl / avg / 1e12,
                               "peak": alu_peak_tflops(2070.0), "unit": "TFLOP/s",
                               "frac": fl / avg / 1e12 / alu_peak_tflops(2070.0),
                               "avg_launch_us": avg * 1e6,
                               "streaming_model_GBs": vox * tv_stream_bytes(wk.Z, 20, False)
                               / (sum(ms) / steps / iters / 1e3) / 1e9}
        plan.close()
    elif name == "batched_8x6":
        # a small case of the batched solver for profiler captures: the batch's
        # stratified 8-item sample (77 M voxels), 6 iterations, BF16 state
        ws = rank_workloads(0)
        idx = oracle_sample(ws)
        sub = [ws[i] for i in idx]
        datas = _gen_items(sub)
        items = []
        for w, d in zip(sub, datas):
            plan = cs.Plan(w.H, w.W, 1, w.Z, torch.from_numpy(d["masks"]).to(dev))
            items.append((plan, torch.from_numpy(d["b"]).to(dev),
                          torch.empty((w.Z, w.H, w.W), dtype=torch.float32, device=dev)))
        iters = 6
        # the phase length the 64-item batch's timing chooses (its line reports it
        # as `schedule`): 8 items alone would time fewer, longer phases as faster
        cs.set_batch_steps_per_phase(BATCH_PROFILE_K)
        batch = cs.Batch(items, cs.Params(**dict(PARAMS, iters=iters)))
        cs.set_batch_steps_per_phase(0)
        ms = _timed(lambda: (batch.run(), batch.wait()), max(1, args.steps), args.warmup, flush)
        vox = sum(w.Z * w.H * w.W for w in sub)
        out.update(metric=METRIC, unit=UNIT, value=vox * iters / (sum(ms) / len(ms) / 1e3),
                   ms_per_step=sum(ms) / len(ms), iterations=iters, items=idx, voxels=vox,
                   schedule=batch.info())
        batch.close()
    elif name in ("unrolled_b8", "unrolled_b1"):
        # batch 8 with the dual iterates kept (29 GB of workspace); batch 1 with
        # them recomputed (a few hundred MB: the case for full profiler captures)
        B, Z, H, W = (8 if name == "unrolled_b8" else 1), 16, 512, 512
        keep_default = name == "unrolled_b8"
        g = torch.Generator(device="cuda").manual_seed(11)
        logits = torch.randn(B, Z, H, W, generator=g, device=dev)
        x = torch.rand(B, Z, H, W, generator=g, device=dev)
        b = (torch.sigmoid(logits) * x).sum(1)
        sc = [torch.tensor(v, device=dev, requires_grad=True) for v in (1.0, 0.05, 0.2)]
        lg = logits.clone().requires_grad_(True)
        def run(keep, n):
            fw, bw = [], []
            for it in range(n + 1):
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record()
                v = cs.unrolled_admm(lg, b, *sc, iters=30, tv_steps=20, ckpt_every=5,
                                     keep_duals=keep)
                loss = 0.5 * ((v - x) ** 2).mean()
                e1.record()
                loss.backward()
                e2.record()
                e2.synchronize()
                if it:
                    fw.append(e0.elapsed_time(e1))
                    bw.append(e1.elapsed_time(e2))
            return float(np.mean(fw)), float(np.mean(bw))

        # dual iterates kept by the segment recompute (batch 8), then recomputed
        # per slice in the reverse sweep
        fwk, bwk = run(keep_default, max(1, args.steps))
        vox = B * Z * H * W
        out.update(metric="unrolled PnP-ADMM voxel-iterations/s (forward + backward)", unit=UNIT,
                   value=vox * 30 / ((fwk + bwk) / 1e3), forward_ms=fwk, backward_ms=bwk,
                   keep_duals=keep_default, batch=B, volume=[Z, H, W], iterations=30)
        if keep_default:
            fwr, bwr = run(False, 1)
            out.update(backward_ms_recompute_duals=bwr, forward_ms_recompute_run=fwr)
    elif name == "wnnm_512x512x16":
        # the WNNM prior (listed in Sec. III-B) on the benchmark volume, z term on
        wk = synth.WORKLOADS["tvz_512x512x16"]
        data = synth.generate(wk)
        plan = cs.Plan(wk.H, wk.W, 1, wk.Z, torch.from_numpy(data["masks"]).to(dev))
        b = torch.from_numpy(data["b"]).to(dev)
        v = torch.empty((wk.Z, wk.H, wk.W), dtype=torch.float32, device=dev)
        iters = 10
        prm = cs.Params(rho=1.0, lam=0.0, gamma=0.2, iters=iters, denoiser="wnnm",
                        bm3d_sigma=0.05)
        cs.timing_read("wnnm_filter", reset=True)
        cs.timing_enable(1)
        ms = _timed(lambda: plan.solve(b, prm, v_out=v), max(1, min(args.steps, 3)), 1, flush)
        cs.timing_enable(0)
        n_f, ms_f = cs.timing_read("wnnm_filter", reset=True)
        x = torch.from_numpy(data["x"].astype(np.float32)).to(dev)
        vox = wk.Z * wk.H * wk.W
        out.update(metric=METRIC, unit=UNIT, value=vox * iters / (sum(ms) / len(ms) / 1e3),
                   ms_per_step=sum(ms) / len(ms), iterations=iters,
                   wnnm_filter_ms_per_launch=ms_f / max(n_f, 1),
                   psnr_db=float(cs.psnr(v, x)), ssim3d=float(cs.ssim3d(v, x)))
        plan.close()
    elif name == "tol_caps_512x512x16":
        # the paper's stopping caps (Sec. IV-B): 100 iterations / 1e-3, 200 / 1e-2,
        # checked on the device every iteration, TV + z on the benchmark volume
        wk = synth.WORKLOADS["tvz_512x512x16"]
        data = synth.generate(wk)
        plan = cs.Plan(wk.H, wk.W, 1, wk.Z, torch.from_numpy(data["masks"]).to(dev))
        b = torch.from_numpy(data["b"]).to(dev)
        v = torch.empty((wk.Z, wk.H, wk.W), dtype=torch.float32, device=dev)
        x = torch.from_numpy(data["x"].astype(np.float32)).to(dev)
        cs.set_autotune(1)
        rows = []
        for iters, tol in ((100, 1e-3), (200, 1e-2)):
            prm = cs.Params(rho=1.0, lam=0.05, gamma=0.2, iters=iters, tol=tol, check_every=1,
                            denoiser="tv", tv_inner=20)
            st = {}

            def run():
                st.update(plan.solve(b, prm, v_out=v, stats=True)[1])

            ms = _timed(run, max(1, args.steps), 1, flush)
            rows.append({"iters_cap": iters, "tol": tol, "iters_done": st["iters_done"],
                         "rel_change": st["rel_change"], "ms_per_solve": sum(ms) / len(ms),
                         "psnr_db": float(cs.psnr(v, x)), "ssim3d": float(cs.ssim3d(v, x))})
        plan.close()
        vox = wk.Z * wk.H * wk.W
        out.update(metric=METRIC, unit=UNIT, iterations=[r["iters_done"] for r in rows],
                   value=vox * rows[0]["iters_done"] / (rows[0]["ms_per_solve"] / 1e3),
                   caps=rows)
    elif name == "cr_sweep_256x256x40":
        # compression-ratio sweep: the same 40-slice volume seen through N shots of
        # R planes each (R = Z / N in {5, 10, 20}), patterns shared by all shots
        Z, H, W = 40, 256, 256
        cs.set_autotune(1)
        rows = []
        for R in (5, 10, 20):
            N = Z // R
            wk = synth.Workload(f"cr{R}", Z, H, W, n_shots=N, per_slice_masks=False, drift=True,
                                mask_p=0.5, peak=200.0, sigma_g=0.01, seed=5000 + R)
            data = synth.generate(wk)
            plan = cs.Plan(H, W, N, R, torch.from_numpy(data["masks"]).to(dev), per_slice=False)
            b = torch.from_numpy(data["b"]).to(dev)
            v = torch.empty((Z, H, W), dtype=torch.float32, device=dev)
            prm = cs.Params(rho=1.0, lam=0.05, gamma=0.2, iters=100, denoiser="tv", tv_inner=20)
            ms = _timed(lambda: plan.solve(b, prm, v_out=v), max(1, args.steps), 1, flush)
            x = torch.from_numpy(data["x"].astype(np.float32)).to(dev)
            rows.append({"R": R, "shots": N, "ms_per_solve": sum(ms) / len(ms),
                         "voxel_it_per_s": Z * H * W * 100 / (sum(ms) / len(ms) / 1e3),
                         "psnr_db": float(cs.psnr(v, x)), "ssim3d": float(cs.ssim3d(v, x))})
            plan.close()
        out.update(metric=METRIC, unit=UNIT, value=rows[0]["voxel_it_per_s"], iterations=100,
                   volume=[Z, H, W], sweep=rows)
    else:
        raise SystemExit(f"unknown workload {name}")
    clocks.window(t_start, time.time())
    out["clocks"] = clocks.stop()
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=None,
                    help="secondary workload: tvz_512x512x16, batched_8x6, tikhonov_1024x1024x32, "
                         "tikhonovz_1024x1024x32, "
                         "tv_1024x1024x32, tv_tiles_1024x1024x32, bm3d_1024x1024x32, tv_128x128x8, "
                         "unrolled_b8, unrolled_b1, "
                         "cr_sweep_256x256x40, tol_caps_512x512x16, wnnm_512x512x16")
    args = ap.parse_args()
    if args.workload:
        run_secondary(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
