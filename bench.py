#!/usr/bin/env python
"""Benchmark of the FFT-based Zernike moment path on one or more GB300s.

Workload: 3840x2160 float32 frames of 32 random anisotropic Gaussian blobs
(centres area-uniform in the disk, sigma 5-40 px, amplitude 0.2-1) plus noise
of standard deviation 0.01, the disk of diameter 2160 centred; moments up to
n_max = 100 on a 1024 x 1024 polar grid.  A step is one zm_moments call on a
batch of B frames already resident in HBM: bilinear polar resampling
(Sec. 2.5), the real FFT of every ring and the radial projection of Eq. 1 with
the bf16 hi + lo split on the tensor cores.  The FP64 radial-polynomial table
(Eq. 7) is built once at plan time, outside the timed region (plan_ms).

The line carries the step time's median and p99 over 200 steps with warm and
with flushed L2, and one roofline per stage, each timed over its own loop of
100 launches: K-b (resampling + ring FFT: zm_stage_spectra), K-c (projection:
zm_stage_project), K-d (reconstruction on the polar nodes: zm_reconstruct);
algorithmic bytes count only what the method must move (the image sectors the
stencils touch, the spectra, tables and results), never an intermediate.

Several GPUs run independent replicas (no collective); the value is the images
of all ranks divided by the slowest rank's time.  ``--impl reference`` times
the FP64 CPU oracle instead, on bounded ring samples of the same workload.

Without ``--quick`` the line also carries: the FP32 and fp16x3 forms' rates
and every form's error against the FP64 oracle, the reconstruction step,
one-frame latency, end to end from pinned host frames, two concurrent
pipelines, an uneven batch in one graph launch, serving swept over arrival
rates with per-request errors against the oracle, reconstruction error vs
order up to 500, a colour frame, the Cartesian-summation route (Eq. 3-6) and
the oracle timed on the host cores.  ``--profile-pass`` runs every kernel path
once, for a profiler's launch list, and measures nothing.
"""

import argparse
import functools
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ZM images/s at 4K n<=100 + p99 latency, mixed-prec vs FP32, err<=1e-4"
H, W, N_BLOBS = 2160, 3840, 32
N_MAX, N_RHO, N_THETA = 100, 1024, 1024
WORKLOAD = "4K blob frames 3840x2160, disk d=2160 centred, n_max=100, N_rho=N_theta=1024, bilinear, midpoint rho"
SYNTH_WORKLOAD_ID = 2


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--prec", default="auto", choices=["auto", "fp32", "bf16x3", "fp16x3"])
    ap.add_argument("--quick", action="store_true", help="skip latency / e2e / cpu-baseline extras")
    ap.add_argument("--profile-pass", action="store_true",
                    help="run every kernel path once at bench sizes (for a launch-list capture); no timing")
    return ap.parse_args()


from paper_2304_14492_gb300.replicas import dist_env, job_throughput, max_over_ranks, shard  # noqa: E402


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "note": "nvidia-smi unavailable"}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) == len(self.FIELDS):
                    rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, val in zip(names, r[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}


# ---------------------------------------------------------------- workload facts
def geometry():
    return (W - 1) / 2.0, (H - 1) / 2.0, min(H, W) / 2.0


def touched_sector_bytes():
    """Distinct 32-byte image sectors that the bilinear stencil of all
    N_rho x N_theta samples touches (row-major float32 frame, row pitch W)."""
    cx, cy, r = geometry()
    rho = (np.arange(N_RHO) + 0.5) / N_RHO
    th = 2 * np.pi * np.arange(N_THETA) / N_THETA
    X = cx + r * rho[:, None] * np.cos(th)[None, :]
    Y = cy - r * rho[:, None] * np.sin(th)[None, :]
    x0 = np.floor(X).astype(np.int64).ravel()
    y0 = np.floor(Y).astype(np.int64).ravel()
    secs = []
    for dy in (0, 1):
        for dx in (0, 1):
            x, y = x0 + dx, y0 + dy
            ok = (x >= 0) & (x < W) & (y >= 0) & (y < H)
            secs.append(((y[ok] * W + x[ok]) * 4) // 32)
    return int(np.unique(np.concatenate(secs)).size) * 32


def disk_box_bytes():
    return min(H, W) * min(H, W) * 4


def make_frames(n, start=0):
    from paper_2304_14492_gb300 import synth
    return [synth.blob_image(H, W, N_BLOBS, workload=SYNTH_WORKLOAD_ID, index=start + b) for b in range(n)]


def read_profile_traffic(name):
    """Per-image DRAM bytes of a stage from the committed ncu summary
    profiles/<name>.md, if the summary was taken on the current sources of the
    kernels it names (a line "source_sha: <file> <sha12> ..." per file)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", name + ".md")
    if not os.path.exists(path):
        return None, "no ncu summary"
    traffic, shas = None, []
    for line in open(path):
        if line.startswith("traffic_bytes_per_image:"):
            traffic = float(line.split(":")[1].split()[0])
        if line.startswith("source_sha:"):
            parts = line.split(":", 1)[1].split()
            shas += list(zip(parts[0::2], parts[1::2]))
    for fname, sha in shas:
        src = os.path.join(ROOT, "paper_2304_14492_gb300", "csrc", fname)
        if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest()[:12] != sha:
            return None, "%s changed since the ncu capture" % fname
    return traffic, None


# ---------------------------------------------------------------- oracle timing
def oracle_pass(img, ring_idx):
    """The FP64 oracle's moments restricted to the rings `ring_idx` of one
    frame: bilinear resampling, angular DFT and the partial radial projection
    (the whole step's work scales with the rings)."""
    import oracle
    rho_all, wr_all = oracle.grid.radial_nodes(N_RHO)
    rho, wr = rho_all[ring_idx], wr_all[ring_idx]
    fhat = oracle.resample.polar_resample(img, rho, N_THETA, geometry())
    F = oracle.moments.angular_dft(fhat, N_MAX)
    table = oracle.zernike.zrp_table(N_MAX, rho)
    return oracle.moments.project(F, wr, N_THETA, N_MAX, table=table)


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count()


def cpu_baseline(img, budget_s=12.0):
    """Whole frames (the frame `img`, repeated) through the oracle on the host
    cores for about budget_s.  Returns the line's cpu_baseline object and the
    oracle's moments of `img`."""
    rings = np.arange(N_RHO)
    t0 = time.perf_counter()
    n = 0
    Zref = None
    while True:
        Z = oracle_pass(img, rings)
        if Zref is None:
            Zref = Z
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or n >= 64:
            break
    return {"value": n / el, "unit": "images/s", "cores": blas_threads(), "kind": "oracle",
            "sample": "%d whole 4K frame(s) through the FP64 oracle (moments: resampling, angular DFT, "
                      "projection), "
                      "%.1f s of CPU time, numpy/BLAS on %d host cores" % (n, el, os.cpu_count())}, Zref


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    img = make_frames(1, start=2000)[0].astype(np.float64)
    # size the per-step ring sample so that warmup + steps take ~2 minutes
    t0 = time.perf_counter()
    oracle_pass(img, np.arange(0, N_RHO, 16))
    t_per_ring = (time.perf_counter() - t0) / (N_RHO // 16)
    budget = 120.0 / max(1, args.steps + args.warmup)
    n_rings = int(max(1, min(N_RHO, budget / max(t_per_ring, 1e-9))))
    rng = np.random.default_rng(0)
    samples = [np.sort(rng.choice(N_RHO, n_rings, replace=False)) for _ in range(args.steps + args.warmup)]
    for s in samples[:args.warmup]:
        oracle_pass(img, s)
    t0 = time.perf_counter()
    for s in samples[args.warmup:]:
        oracle_pass(img, s)
    el = time.perf_counter() - t0
    frac = args.steps * n_rings / N_RHO            # frames' worth of work done
    value = frac / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "images/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "batch": 1, "sample_rings_per_step": n_rings},
            "cpu_baseline": {"value": value, "unit": "images/s", "cores": blas_threads(), "kind": "oracle",
                             "sample": "%d random rings of 1024 per step (1/%0.1f frame), scaled to frames"
                                       % (n_rings, N_RHO / n_rings)},
            "e2e": {"value": value, "unit": "images/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def event_loop(torch, st, fn, reps):
    """Mean device time (ms) of `fn` over `reps` back-to-back calls on stream st."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        fn()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def step_distribution(torch, dev, st, step, steps=200):
    """Per-step device time (events around each step), warm L2 and with L2
    flushed (a 256 MB write) before every step: median and p99 in ms."""
    flush = torch.empty(64 * 2**20, device=dev, dtype=torch.float32)
    out = {}
    for name, cold in (("warm_l2", False), ("cold_l2", True)):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            if cold:
                flush.fill_(float(k))
            ev[k][0].record(st)
            step()
            ev[k][1].record(st)
        torch.cuda.synchronize(dev)
        t = sorted(a.elapsed_time(b) for a, b in ev)
        out[name] = {"median_ms": statistics.median(t), "p99_ms": t[min(steps - 1, int(0.99 * steps))],
                     "steps": steps}
    del flush
    return out


def stage_rooflines(zm, torch, dev, st, plan, descs, B, P, hbm, peaks, reps=100):
    """One roofline per stage of the step, each over its own loop of `reps`
    launches: K-b = zm_stage_spectra (resampling + ring FFT), K-c =
    zm_stage_project (radial projection), K-d = zm_reconstruct (radial
    reconstruction + inverse ring FFT on the polar nodes, Neumann).
    Algorithmic bytes per image: K-b the distinct 32-byte image sectors the
    bilinear stencils touch plus the spectra written; K-c the split table
    once per batch, the spectra and the moments; K-d the split table once per
    batch, the moments and the polar reconstruction written."""
    sectors = touched_sector_bytes()
    f_bytes = (N_MAX + 1) * N_RHO * 8                      # F_m(rho_i), complex64 (bf16 hi + lo: same bytes)
    table = 2 * 2 * P * N_RHO                              # hi + lo bf16 halves
    z_bytes = P * 8
    polar = N_RHO * N_THETA * 4
    out = torch.empty((B, P, 2), device=dev)
    frec = torch.empty((B, N_RHO, N_THETA), device=dev)
    zm.zm_stage_spectra(plan, descs, st)
    zm.zm_stage_project(plan, B, out, 0, st)
    l0 = zm.zm_launch_count()
    zm.zm_stage_spectra(plan, descs, st)
    kb_launches = zm.zm_launch_count() - l0
    torch.cuda.synchronize(dev)
    res = {}
    t = event_loop(torch, st, lambda: zm.zm_stage_spectra(plan, descs, st), reps)
    kb = B * (sectors + f_bytes)
    res["K-b"] = {"bound": "hbm", "launch_ms": t, "algorithmic_bytes_per_launch": kb,
                  "achieved": kb / (t / 1000.0) / 1e9, "peak": hbm, "unit": "GB/s", "frac": kb / (t / 1000.0) / 1e9 / hbm,
                  "kernels_per_call": kb_launches,
                  "path": "fused resampling + ring FFT" if kb_launches == 1 else "tile resampler, then ring FFT",
                  "per_image_bytes": {"touched_sectors": sectors, "spectra_out": f_bytes, "disk_box": disk_box_bytes()}}
    zm.zm_stage_spectra(plan, descs, st)
    t = event_loop(torch, st, lambda: zm.zm_stage_project(plan, B, out, 0, st), reps)
    kc = table + B * (f_bytes + z_bytes)
    flops = 4.0 * P * N_RHO * B
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    res["K-c"] = {"bound": "hbm", "launch_ms": t, "algorithmic_bytes_per_launch": kc,
                  "achieved": kc / (t / 1000.0) / 1e9, "peak": hbm, "unit": "GB/s",
                  "frac": kc / (t / 1000.0) / 1e9 / hbm, "algorithmic_tflops": flops / (t / 1000.0) / 1e12,
                  "executed_tflops": 3 * flops / (t / 1000.0) / 1e12, "bf16_peak_tflops": bf16,
                  "tensor_frac_executed": 3 * flops / (t / 1000.0) / 1e12 / bf16,
                  "note": "B=%d is below the bf16 ridge (%.0f flop/B), so the table and spectra traffic bounds it"
                          % (B, bf16 * 1e12 / (hbm * 1e9))}
    t = event_loop(torch, st, lambda: zm.zm_reconstruct(plan, out, B, frec, zm.ZM_NEUMANN, st), reps)
    kd = table + B * (z_bytes + polar)
    res["K-d"] = {"bound": "hbm", "launch_ms": t, "algorithmic_bytes_per_launch": kd,
                  "achieved": kd / (t / 1000.0) / 1e9, "peak": hbm, "unit": "GB/s",
                  "frac": kd / (t / 1000.0) / 1e9 / hbm, "algorithmic_tflops": flops / (t / 1000.0) / 1e12}
    # the fused kernel on the same frames (a plan made with ZM_FUSED=1), for
    # its DRAM traffic and time beside the tile path
    old = os.environ.get("ZM_FUSED")
    os.environ["ZM_FUSED"] = "1"
    try:
        pf = zm.zm_plan(N_MAX, N_RHO, N_THETA, zm.ZM_PREC_BF16X3)
    finally:
        if old is None:
            del os.environ["ZM_FUSED"]
        else:
            os.environ["ZM_FUSED"] = old
    try:
        zm.zm_plan_reserve(pf, B)
        zm.zm_stage_spectra(pf, descs, st)
        t = event_loop(torch, st, lambda: zm.zm_stage_spectra(pf, descs, st), reps)
        res["K-b_fused"] = {"launch_ms": t, "achieved": kb / (t / 1000.0) / 1e9, "frac": kb / (t / 1000.0) / 1e9 / hbm,
                            "note": "the fused resampling + ring FFT kernel forced on this grid (ZM_FUSED=1); "
                                    "zm_moments fuses up to 2^17 polar samples per image"}
    finally:
        zm.zm_plan_destroy(pf)
    for key, name in (("K-b", "kb_tile_4k_b16" if kb_launches > 1 else "kb_fused_4k_b16"),
                      ("K-b_fused", "kb_fused_4k_b16")):
        traffic, note = read_profile_traffic(name)
        res[key]["traffic"] = traffic * B if traffic else None
        if note:
            res[key]["traffic_note"] = note
        elif traffic:
            res[key]["traffic_over_algorithmic"] = traffic / (sectors + f_bytes)
    return res


def run_gb300(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2304_14492_gb300 import native as zm

    B = args.batch
    prec = args.prec
    if prec == "auto":
        prec = "bf16x3"
    pflag = {"fp32": zm.ZM_PREC_FP32, "bf16x3": zm.ZM_PREC_BF16X3, "fp16x3": zm.ZM_PREC_FP16X3}
    P = zm.zm_num_moments(N_MAX)
    frames = make_frames(B, start=shard(rank, B).start)
    imgs = torch.from_numpy(np.stack(frames)).to(dev)
    views = [imgs[b] for b in range(B)]
    del frames

    t0 = time.perf_counter()
    try:
        plan = zm.zm_plan(N_MAX, N_RHO, N_THETA, pflag[prec])
    except zm.ZmError as e:
        if e.status != zm.ZM_EUNSUPPORTED:
            raise
        prec = "fp32"
        plan = zm.zm_plan(N_MAX, N_RHO, N_THETA, pflag[prec])
    plan_ms = 1000 * (time.perf_counter() - t0)
    zm.zm_plan_reserve(plan, B)

    st = torch.cuda.current_stream(dev)
    out = torch.empty((B, P, 2), device=dev)
    descs = zm.image_array(views)            # the frames' descriptors, built once like a caller would

    def step():
        zm.zm_moments(plan, descs, out, 0, st)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()

    try:
        gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
        gpu_id = gpu_id if gpu_id.startswith("GPU-") else "GPU-" + gpu_id
    except Exception:
        gpu_id = str(local)
    sampler = ClockSampler(gpu_id)
    sampler.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    l0 = zm.zm_launch_count()
    ev0.record(st)
    for _ in range(args.steps):
        step()
    ev1.record(st)
    torch.cuda.synchronize(dev)
    l1 = zm.zm_launch_count()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    ms = max_over_ranks(ms, dev)
    value = job_throughput(world, B, args.steps, ms)

    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    dist_t = step_distribution(torch, dev, st, step)
    stages = stage_rooflines(zm, torch, dev, st, plan, descs, B, P, hbm, peaks)
    kb = stages["K-b"]
    roofline = {"bound": "hbm", "stage": "K-b (resampling + ring FFT)", "path": kb["path"],
                "achieved": kb["achieved"], "peak": hbm, "unit": "GB/s", "frac": kb["achieved"] / hbm,
                "traffic": kb.get("traffic"), "algorithmic_bytes_per_launch": kb["algorithmic_bytes_per_launch"],
                "launch_ms": kb["launch_ms"],
                "launch_timing": "CUDA events around 100 back-to-back zm_stage_spectra calls (the stage alone)",
                "peak_source": "measured copy (MEASURED_PEAKS.json)" if peaks else "fallback",
                "per_image_bytes": kb["per_image_bytes"]}
    if "traffic_note" in kb:
        roofline["traffic_note"] = kb["traffic_note"]
    sectors = kb["per_image_bytes"]["touched_sectors"]
    f_bytes = kb["per_image_bytes"]["spectra_out"]
    step_ms = ms / args.steps
    line = {"metric": METRIC, "value": value, "unit": "images/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == "fp32" else prec.replace("x3", "x3+f32acc"), "data": "synthetic",
            "config": {"workload": WORKLOAD, "batch_per_gpu": B, "global_batch": B * world,
                       "precision": prec, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (%d MB of frames per step)" % (B * H * W * 4 // 2**20),
                       "step": "zm_moments: resampling + ring FFT + radial projection (bf16 hi+lo split, "
                               "FP32 accumulate)"},
            "step_time": dist_t,
            "whole_step_hbm": {"algorithmic_bytes_per_image": sectors + 2 * f_bytes,
                               "achieved_gbs": B * (sectors + 2 * f_bytes) / (step_ms / 1000.0) / 1e9,
                               "frac": B * (sectors + 2 * f_bytes) / (step_ms / 1000.0) / 1e9 / hbm,
                               "note": "touched sectors + spectra written and read back, per image, over the "
                                       "whole step time (the split table, 10.65 MB per batch, stays in L2)"},
            "roofline": roofline, "stages": stages, "gpu_launches": l1 - l0, "clocks": clocks, "plan_ms": plan_ms}

    if rank == 0 and not args.quick:
        line.update(extras(args, zm, torch, dev, st, plan, prec, views, descs, out, B, P))
        line["pipelined"] = bench_pipelined(zm, torch, dev, descs, B, P)
        line["colour"] = bench_colour(zm, torch, dev, plan, P)
        del views, imgs
        torch.cuda.empty_cache()
        img0, frame0 = line.pop("_frame0")
        line["uneven_batch"] = bench_uneven(zm, torch, dev)
        line["stability"] = bench_stability(zm, torch, dev)
        line["cartesian"] = bench_cartesian(zm, torch, dev)
        line["serving"] = bench_serving(zm)
        line["cpu_baseline"], Zref = cpu_baseline(img0)
        line["err_vs_fp64"] = {k: float(np.max(np.abs(z - Zref)) / np.max(np.abs(Zref))) for k, z in frame0.items()}
        line["err_bars"] = {"fp32": 1e-4, "bf16x3": 2e-5, "fp16x3": 2e-5,
                            "note": "max|Z - Z_fp64| / max|Z_fp64| per frame; the split forms' per-moment bound "
                                    "3 u^2 sum_i |a_i f_i| is asserted in the tests"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
    zm.zm_plan_destroy(plan)


def extras(args, zm, torch, dev, st, plan, prec, views, descs, out, B, P):
    res = {}
    pflag = {"fp32": zm.ZM_PREC_FP32, "bf16x3": zm.ZM_PREC_BF16X3, "fp16x3": zm.ZM_PREC_FP16X3}
    plans = {prec: plan}
    for name in ("fp32", "bf16x3", "fp16x3"):
        if name not in plans:
            plans[name] = zm.zm_plan(N_MAX, N_RHO, N_THETA, pflag[name])
            zm.zm_plan_reserve(plans[name], B)

    # moments per precision on the same frames: the mixed forms against FP32
    rates = {}
    for name, p in plans.items():
        for _ in range(5):
            zm.zm_moments(p, descs, out, 0, st)
        t = event_loop(torch, st, lambda: zm.zm_moments(p, descs, out, 0, st), 100)
        rates[name] = B / (t / 1000.0)
    res["moments_images_per_s"] = rates
    res["mixed_over_fp32"] = {k: v / rates["fp32"] for k, v in rates.items() if k != "fp32"}

    # frame 0 through every precision; compared with the FP64 oracle's moments
    # of the same frame, which the cpu_baseline leg computes while it is timed
    frame0 = {}
    for name, p in plans.items():
        o1 = torch.empty((1, P, 2), device=dev)
        zm.zm_moments(p, [views[0]], o1, 0, st)
        torch.cuda.synchronize(dev)
        z = o1[0].double().cpu().numpy()
        frame0[name] = z[:, 0] + 1j * z[:, 1]
    res["_frame0"] = (views[0].double().cpu().numpy(), frame0)

    # the reconstruction step beside the moments: moments with the polar
    # samples kept, Neumann reconstruction on the polar nodes, Eq. 10 / Eq. 13
    fh = torch.empty((B, N_RHO, N_THETA), device=dev)
    fr = torch.empty((B, N_RHO, N_THETA), device=dev)
    er = torch.empty((B, 4), device=dev, dtype=torch.float64)

    def rec_step():
        zm.zm_moments_ex(plan, descs, out, fh, 0, st)
        zm.zm_reconstruct_errors(plan, out, B, fr, fh, er, zm.ZM_NEUMANN, st)

    for _ in range(3):
        rec_step()
    t = event_loop(torch, st, rec_step, 50)
    res["reconstruction_step"] = {"ms_per_batch": t, "images_per_s": B / (t / 1000.0),
                                  "step": "zm_moments_ex + zm_reconstruct_errors (Neumann, polar nodes)"}
    del fh, fr, er

    # single-frame latency (L2 flushed between calls)
    flush = torch.empty(64 * 2**20, device=dev, dtype=torch.float32)     # 256 MB > L2
    o1 = torch.empty((1, P, 2), device=dev)
    lat = []
    for k in range(120):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        zm.zm_moments(plan, [views[k % B]], o1, 0, st)
        e1.record(st)
        torch.cuda.synchronize(dev)
        if k >= 20:
            lat.append(e0.elapsed_time(e1))
    lat.sort()
    res["latency_b1_ms"] = {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                            "calls": len(lat), "note": "device time of one zm_moments call, cold L2"}
    del flush

    # end to end through the public API: pinned host frames -> disk spans on
    # the device (zm_upload_disk, a kernel reading the pinned frames) ->
    # zm_moments -> moments back to the host.  Two device buffers: the upload
    # of step k + 1 runs on its own stream while step k computes (the host
    # link, not the GPU, bounds this path)
    host = torch.empty((B, H, W), dtype=torch.float32, pin_memory=True)
    host.copy_(torch.stack([v for v in views]).cpu())
    hviews = [host[b] for b in range(B)]
    box_bytes = zm.zm_upload_disk_bytes(hviews)
    h2d_bytes = zm.zm_upload_disk_traffic(hviews)
    dbufs = [torch.empty(box_bytes // 4 + 4, device=dev) for _ in range(2)]
    hout = torch.empty((B, P, 2), dtype=torch.float32, pin_memory=True)
    s_up = torch.cuda.Stream(dev)
    up_done = [torch.cuda.Event() for _ in range(2)]
    read_done = [torch.cuda.Event() for _ in range(2)]
    boxes = [None, None]

    def upload(k):
        j = k % 2
        s_up.wait_event(read_done[j])                # the step that read this buffer is past its moments
        boxes[j] = zm.zm_upload_disk(hviews, dbufs[j], s_up)
        up_done[j].record(s_up)

    def compute(k):
        j = k % 2
        st.wait_event(up_done[j])
        zm.zm_moments(plan, boxes[j], out, 0, st)
        read_done[j].record(st)
        hout.copy_(out, non_blocking=True)

    def run(n):
        upload(0)
        for k in range(n):
            if k + 1 < n:
                upload(k + 1)
            compute(k)

    run(3)
    torch.cuda.synchronize(dev)
    reps = max(5, min(args.steps, 40))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    s_up.wait_event(e0)
    run(reps)
    e1.record(st)
    torch.cuda.synchronize(dev)
    res["e2e"] = {"value": B * reps / (e0.elapsed_time(e1) / 1000.0), "unit": "images/s",
                  "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": B * P * 8,
                  "steps": reps,
                  "h2d": "row spans of the disks of the pinned frames, read by a kernel (zm_upload_disk), "
                         "the next step's upload overlapping this step's compute"}
    for name, p in plans.items():
        if p != plan:
            zm.zm_plan_destroy(p)
    return res


def bench_pipelined(zm, torch, dev, descs, B, P, pipelines=2, batches=200):
    """The headline step on `pipelines` independent pipelines (plan, buffers
    and stream each), batches dealt round-robin: the memory-bound resampler of
    one batch overlaps the issue-bound ring FFT and projection of another.
    Whole-job frames/s; the headline stays the one-stream step."""
    pipes = []
    for _ in range(pipelines):
        plan = zm.zm_plan(N_MAX, N_RHO, N_THETA, zm.ZM_PREC_BF16X3)
        zm.zm_plan_reserve(plan, B)
        pipes.append({"plan": plan, "st": torch.cuda.Stream(dev), "out": torch.empty((B, P, 2), device=dev)})

    def step(q):
        zm.zm_moments(q["plan"], descs, q["out"], 0, q["st"])

    for k in range(4 * pipelines):
        step(pipes[k % pipelines])
    torch.cuda.synchronize(dev)
    main = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(main)
    for q in pipes:
        q["st"].wait_event(e0)
    for k in range(batches):
        step(pipes[k % pipelines])
    for q in pipes:
        ev = torch.cuda.Event()
        ev.record(q["st"])
        main.wait_event(ev)
    e1.record(main)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    for q in pipes:
        zm.zm_plan_destroy(q["plan"])
    return {"pipelines": pipelines, "batches": batches, "batch": B, "ms_per_batch": ms / batches,
            "images_per_s": B * batches / (ms / 1000.0),
            "note": "zm_moments on %d streams at once (a plan and buffers each), batches dealt round-robin"
                    % pipelines}


def bench_stability(zm, torch, dev):
    """Reconstruction error vs order up to n_max = 500 (the paper's stability
    range, Sec. 3.1): one 1024x1024 blob frame, moments with the Eq. 7 table on
    Gauss-Legendre and midpoint radial nodes, reconstruction on the polar nodes
    (Neumann), Eq. 10 / Eq. 13 errors; plan build time per order."""
    from paper_2304_14492_gb300 import synth
    size, n_rho, n_theta = 1024, 512, 1024
    img = torch.from_numpy(synth.blob_image(size, size, 16, workload=5, index=0)).to(dev)
    res = {"frame": "1024x1024 blob frame, disk d=1024 centred", "n_rho": n_rho, "n_theta": n_theta, "rows": []}
    for gname, gflag in (("gauss", zm.ZM_GRID_GAUSS), ("midpoint", zm.ZM_GRID_MIDPOINT)):
        for pname, pflag in (("fp32", zm.ZM_PREC_FP32), ("bf16x3", zm.ZM_PREC_BF16X3)):
            for n_max in (25, 50, 100, 200, 300, 400, 500):
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                plan = zm.zm_plan(n_max, n_rho, n_theta, gflag | pflag)
                torch.cuda.synchronize(dev)
                plan_ms = 1000 * (time.perf_counter() - t0)
                P = zm.zm_num_moments(n_max)
                out = torch.empty((1, P, 2), device=dev)
                fh = torch.empty((1, n_rho, n_theta), device=dev)
                err = torch.empty((1, 4), device=dev, dtype=torch.float64)
                zm.zm_moments_ex(plan, [img], out, fh)
                zm.zm_reconstruct_errors(plan, out, 1, None, fh, err, zm.ZM_NEUMANN)
                e = err.cpu().numpy()[0]
                zm.zm_plan_destroy(plan)
                res["rows"].append({"grid": gname, "precision": pname, "n_max": n_max, "eps1": float(e[0]),
                                    "eps": float(e[1]), "plan_ms": plan_ms})
    return res


def bench_colour(zm, torch, dev, plan, P, steps=20):
    """One 4K colour frame as a batch of its three bands (Sec. 2.3, Sec. 3):
    per-band min / max over the disk, moments, Cartesian reconstruction (Neumann),
    min-max normalisation to each band's stored range (Table I), Eq. 10 / Eq. 13
    per band; colour frames/s with the bands resident on the device."""
    from paper_2304_14492_gb300 import synth
    bands = [torch.from_numpy(synth.blob_image(H, W, N_BLOBS, workload=SYNTH_WORKLOAD_ID, index=1000 + c)).to(dev)
             for c in range(3)]
    descs = zm.image_array(bands)
    canv = [torch.empty((H, W), device=dev) for _ in range(3)]
    cdescs, tdescs = zm.canvas_array(canv), zm.image_array(canv)
    mm = torch.empty((3, 2), device=dev)
    out = torch.empty((3, P, 2), device=dev)
    polar = torch.empty((3, N_RHO, N_THETA), device=dev)
    err = torch.empty((3, 4), device=dev, dtype=torch.float64)
    st = torch.cuda.current_stream(dev)

    def step():
        zm.zm_disk_minmax(plan, descs, mm, st)
        zm.zm_moments(plan, descs, out, 0, st)
        zm.zm_reconstruct_cartesian(plan, out, cdescs, polar, zm.ZM_NEUMANN, st)
        zm.zm_minmax_normalize(plan, cdescs, mm, st)
        zm.zm_errors(plan, descs, tdescs, err, st)

    for _ in range(3):
        step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        step()
    e1.record(st)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    e = err.cpu().numpy()
    # algorithmic bytes per band: the disk's pixels read by the min / max pass,
    # the moments' touched sectors and spectra, the disk's pixels written by the
    # reconstruction, read and written by the normalisation, and both images'
    # disk pixels read by the error sums
    disk = int(np.count_nonzero(((2 * np.arange(W) + 1 - W)[None, :] ** 2 + (2 * np.arange(H) + 1 - H)[:, None] ** 2)
                                <= H * H)) * 4
    per_band = disk + touched_sector_bytes() + 2 * (N_MAX + 1) * N_RHO * 8 + disk + 2 * disk + 2 * disk
    gbs = 3 * per_band / (ms / 1000.0) / 1e9
    hbm = float(measured_peaks().get("hbm_gbs", 6800.0))
    return {"frame": "3 bands of 3840x2160 blob frames, n_max=100, N_rho=N_theta=1024", "ms_per_frame": ms,
            "frames_per_s": 1000.0 / ms, "eps1_per_band": [float(x) for x in e[:, 0]],
            "eps13_per_band": [float(x) for x in e[:, 1]],
            "hbm": {"algorithmic_bytes_per_frame": 3 * per_band, "achieved_gbs": gbs, "frac": gbs / hbm,
                    "note": "disk pixels: min/max read, reconstruction write, normalisation read+write, errors "
                            "read both images; plus the moments' sectors and spectra"}}


def bench_cartesian(zm, torch, dev, reps=50):
    """Cartesian summation (Eq. 3-6) with 8-point symmetry, the paper's Fig. 5
    mode: one moment of a given order of one N x N frame (disk inscribed),
    device time per moment; HBM roofline on the pixels of the disk read once."""
    from paper_2304_14492_gb300 import synth
    peaks = {}
    try:
        import json as _json
        peaks = _json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    st = torch.cuda.current_stream(dev)
    out = torch.empty((1, 1, 2), device=dev)
    work = torch.empty(zm.zm_cartesian_work_bytes(1, 1) // 8 + 1, dtype=torch.float64, device=dev)
    rows = []
    for size in (1000, 2000, 4000):
        img = torch.from_numpy(synth.blob_image(size, size, 24, workload=SYNTH_WORKLOAD_ID, index=2000 + size)).to(dev)
        descs = zm.image_array([img])
        disk_px = int(np.count_nonzero(
            ((2 * np.arange(size) + 1 - size)[None, :] ** 2 + (2 * np.arange(size) + 1 - size)[:, None] ** 2)
            <= size * size))
        for (n, m) in ((100, 36), (20, 0), (400, 2)):
            for _ in range(3):
                zm.zm_cartesian_moments(descs, [(n, m)], out, work, 0, st)
            torch.cuda.synchronize(dev)
            # `reps` calls captured in a CUDA graph: device time per call, not
            # the Python marshalling of each call
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                cs = torch.cuda.current_stream(dev)
                for _ in range(reps):
                    zm.zm_cartesian_moments(descs, [(n, m)], out, work, 0, cs)
            graph.replay()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            graph.replay()
            e1.record(st)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / reps
            del graph
            gbs = disk_px * 4 / (ms / 1000.0) / 1e9
            rows.append({"N": size, "n": n, "m": m, "ms_per_moment": ms, "moments_per_s": 1000.0 / ms,
                         "disk_bytes": disk_px * 4, "achieved_gbs": gbs, "frac_of_hbm": gbs / hbm})
        del img
    return {"mode": "one moment of one N x N blob frame per call, inscribed disk, 8-point symmetry, fp32",
            "note": "the paper's Fig. 5 reports about 20 frames/s (50 ms per moment) at 4000 x 4000 on a "
                    "Titan Xp; context only (another GPU)",
            "rows": rows}


def bench_uneven(zm, torch, dev, count=256):
    """Uneven batch (sizes 128..1024, n_max 30..80, N_rho = size/2): one graph
    launch per replay; images/s per projection precision."""
    from paper_2304_14492_gb300 import synth
    specs = synth.uneven_batch_specs(count=count, workload=3)
    pool = {}
    items = []
    for j, (size, n_max, n_rho, n_theta) in enumerate(specs):
        key = (size, j % 4)
        if key not in pool:
            pool[key] = torch.from_numpy(synth.blob_image(size, size, 8, workload=3, index=j)).to(dev)
        out = torch.empty((zm.zm_num_moments(n_max), 2), device=dev)
        items.append((pool[key], n_max, n_rho, n_theta, out))
    res = {"requests": count, "note": "4 distinct frames per size, each request its own output"}
    st = torch.cuda.current_stream(dev)
    for name, flag in (("bf16x3", zm.ZM_PREC_BF16X3), ("fp16x3", zm.ZM_PREC_FP16X3), ("fp32", zm.ZM_PREC_FP32)):
        arr = zm.requests(items)                 # marshalled once, as a caller replaying a batch would
        b = zm.zm_batch_create(arr, flag)
        try:
            for _ in range(3):
                zm.zm_batch_run(b, arr, 0, st)
            # kernels in the replayed graph: the launches of one capture (a run
            # with new output pointers captures the sequence again)
            alt = zm.requests([(im, nm, nr, nt, torch.empty_like(o)) for im, nm, nr, nt, o in items])
            l0 = zm.zm_launch_count()
            zm.zm_batch_run(b, alt, 0, st)
            kernels = zm.zm_launch_count() - l0
            zm.zm_batch_run(b, arr, 0, st)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 50
            e0.record(st)
            for _ in range(reps):
                zm.zm_batch_run(b, arr, 0, st)
            e1.record(st)
            torch.cuda.synchronize(dev)
            res[name] = {"images_per_s": count * reps / (e0.elapsed_time(e1) / 1000.0),
                         "groups": zm.zm_batch_info(b)["groups"], "kernels_per_replay": kernels,
                         "graph_launches_per_replay": 1}
        finally:
            zm.zm_batch_destroy(b)
    return res


SERVE_SIZES, SERVE_ORDERS = (256, 512, 1024, 2160), (20, 50, 100, 200)


@functools.lru_cache(maxsize=16)
def serve_image(size, k):
    """Image k of a serving size class: blob frames, 2160 = the centred
    2160x2160 crop of a 3840x2160 frame."""
    from paper_2304_14492_gb300 import synth
    if size == 2160:
        f = synth.blob_image(H, W, N_BLOBS, workload=5, index=k)
        return np.ascontiguousarray(f[:, (W - H) // 2:(W - H) // 2 + H])
    return synth.blob_image(size, size, 8, workload=5, index=k)


def serve_n_theta(n_max):
    nt = 1
    while nt < 2 * n_max + 2:
        nt *= 2
    return nt


def _oracle_request(args):
    """Worker: the FP64 oracle's moments of one served request (image rebuilt
    from its seed) and the relative max error of the served result."""
    size, k, n_max, got = args
    sys.path.insert(0, ROOT)
    import oracle
    img = serve_image(size, k).astype(np.float64)
    ref = oracle.moments.moments(img, n_max, size // 2, serve_n_theta(n_max))
    z = got[:, 0].astype(np.float64) + 1j * got[:, 1].astype(np.float64)
    return size, n_max, float(np.max(np.abs(z - ref)) / np.max(np.abs(ref)))


def bench_serving(zm, rates=(2000.0, 8000.0, 32000.0, 128000.0), max_requests=20000, seconds=10.0, seed=7,
                  per_cell=16):
    """Poisson arrivals of host images (sizes 256/512/1024/2160-crop, n_max
    20/50/100/200, N_rho = size/2, N_theta = next power of two >= 2 n_max + 2)
    into the continuous-batching server, swept from 2000 requests/s past
    saturation; latency submit -> result on the host.  At the highest rate,
    `per_cell` requests of every (size, n_max) cell are checked against the
    FP64 oracle (process pool on the host cores), and every request of that
    run is run again alone and compared with its result in the mix."""
    import multiprocessing as mp
    rng = np.random.default_rng(seed)
    pool = {sz: [serve_image(sz, k) for k in range(2 if sz == 2160 else 4)] for sz in SERVE_SIZES}
    srv = zm.zm_server_create(4 << 30, 4, 64, zm.ZM_PREC_BF16X3)
    sweep, last = [], None
    try:
        # resident plans for every grid first (plan builds are not request latency)
        warm = [(sz, nm, np.empty((zm.zm_num_moments(nm), 2), np.float32)) for sz in SERVE_SIZES
                for nm in SERVE_ORDERS]
        for sz, nm, o in warm:                 # the outputs stay referenced until drained
            zm.zm_server_submit(srv, pool[sz][0], nm, sz // 2, serve_n_theta(nm), o)
        zm.zm_server_drain(srv, 120.0)
        for rate in rates:
            n = int(min(max_requests, rate * seconds))
            arrivals = np.cumsum(rng.exponential(1.0 / rate, n))
            reqs = []
            for j in range(n):
                sz = int(rng.choice(SERVE_SIZES))
                nm = int(rng.choice(SERVE_ORDERS))
                k = j % len(pool[sz])
                reqs.append((sz, k, nm, np.empty((zm.zm_num_moments(nm), 2), np.float32)))
            zm.zm_server_reset_stats(srv)
            t0 = time.perf_counter()
            late = 0.0
            for (sz, k, nm, out), ta in zip(reqs, arrivals):
                now = time.perf_counter() - t0
                while now < ta:
                    now = time.perf_counter() - t0
                late = max(late, now - ta)
                zm.zm_server_submit(srv, pool[sz][k], nm, sz // 2, serve_n_theta(nm), out)
            zm.zm_server_drain(srv, 120.0)
            wall = time.perf_counter() - t0
            stats = zm.zm_server_stats(srv)
            done = int(stats["completed"])
            sweep.append({"arrival_rate_per_s": rate, "requests": n, "completed": done,
                          "offered_s": float(arrivals[-1]), "wall_s": wall, "images_per_s": done / wall,
                          "p50_ms": stats["p50_ms"], "p99_ms": stats["p99_ms"], "max_ms": stats["max_ms"],
                          "groups_launched": int(stats["groups_launched"]),
                          "requests_per_group": done / max(1, int(stats["groups_launched"])),
                          "peak_device_bytes": int(stats["peak_bytes"]),
                          "submit_lag_max_ms": 1000.0 * late})
            last = reqs
        # every request of the highest-rate run again, alone, against its result in the mix
        worst, rerun, t1 = 0.0, 0, time.perf_counter()
        for sz, k, nm, out in last:
            if time.perf_counter() - t1 > 60.0:
                break
            o = np.empty_like(out)
            zm.zm_server_wait(srv, zm.zm_server_submit(srv, pool[sz][k], nm, sz // 2, serve_n_theta(nm), o), 30.0)
            worst = max(worst, float(np.max(np.abs(o - out)) / max(float(np.max(np.abs(o))), 1e-30)))
            rerun += 1
        host_direct = bool(zm.zm_server_stats(srv)["host_direct"])
    finally:
        zm.zm_server_destroy(srv, 60.0)
    del warm
    # per-request error against the FP64 oracle: the first `per_cell` requests
    # of every (size, n_max) cell of the highest-rate run
    picked, seen = [], {}
    for sz, k, nm, out in last:
        if seen.get((sz, nm), 0) < per_cell:
            seen[(sz, nm)] = seen.get((sz, nm), 0) + 1
            picked.append((sz, k, nm, out))
    t2 = time.perf_counter()
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pp:
        errs = pp.map(_oracle_request, picked, chunksize=1)
    cells = {}
    for sz, nm, e in errs:
        c = cells.setdefault("%dx%d n_max=%d" % (sz, sz, nm), {"requests": 0, "max_rel_err": 0.0})
        c["requests"] += 1
        c["max_rel_err"] = max(c["max_rel_err"], e)
    return {"precision": "bf16x3", "host_direct": host_direct, "sweep": sweep,
            "alone_vs_mix": {"requests_rerun": rerun, "max_rel_diff": worst},
            "err_vs_fp64": {"cells": cells, "worst": max(c["max_rel_err"] for c in cells.values()),
                            "bar": 2e-5, "oracle_s": time.perf_counter() - t2,
                            "note": "max|Z - Z_fp64| / max|Z_fp64| per request, %d requests per (size, n_max) "
                                    "cell of the %.0f/s run" % (per_cell, rates[-1])},
            "note": "statistics reset per rate after 16 plan-warming requests; latency = submit -> moments in "
                    "host memory; submit_lag = how late the Python submitter was against the Poisson schedule"}


def profile_pass(batch=16):
    """Every kernel path of the library once, at the bench's sizes where it has
    one: plan builds, the FP32 and FP16 projection forms on 16 4K frames (the
    stage calls and the tile path), the fused resampling + ring FFT kernel and
    the two tensor-core DFT kernels on the same frames, the gather path (frames TMA cannot stage), the FP32
    reconstruction with errors, pixel reconstruction and normalisation (a
    colour frame), the upload
    of host frames, the Cartesian route at 4000 x 4000, an uneven batch and a
    few served requests.  For a launch-list capture under a profiler: prints
    one line and measures nothing."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2304_14492_gb300 import native as zm, synth
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    B = batch
    imgs = torch.from_numpy(np.stack(make_frames(B))).to(dev)
    views = [imgs[b] for b in range(B)]
    P = zm.zm_num_moments(N_MAX)
    out = torch.empty((B, P, 2), device=dev)
    fh = torch.empty((B, N_RHO, N_THETA), device=dev)
    fr = torch.empty((B, N_RHO, N_THETA), device=dev)
    err = torch.empty((B, 4), device=dev, dtype=torch.float64)
    for prec in (zm.ZM_PREC_FP32, zm.ZM_PREC_FP16X3, zm.ZM_PREC_BF16X3):
        plan = zm.zm_plan(N_MAX, N_RHO, N_THETA, prec)
        zm.zm_plan_reserve(plan, B)
        zm.zm_stage_spectra(plan, views)
        zm.zm_stage_project(plan, B, out)
        zm.zm_moments_ex(plan, views, out, fh)
        zm.zm_reconstruct_errors(plan, out, B, fr, fh, err, zm.ZM_NEUMANN)
        if prec == zm.ZM_PREC_FP32:
            # frames at a 4-byte offset: not TMA-eligible, the fused gather kernel
            shifted = [imgs[b][:, 1:] for b in range(4)]
            zm.zm_moments(plan, shifted, out[:4])
            spectra = torch.empty((N_MAX + 1, 4, 2, N_RHO), device=dev)
            zm.zm_ring_spectra(plan, views[:4], spectra, None)
            zm.zm_project(plan, spectra, 4, out[:4])
        torch.cuda.synchronize(dev)
        zm.zm_plan_destroy(plan)
    os.environ["ZM_FUSED"] = "1"                 # the fused kernel on the 4K grid as well
    for prec in (zm.ZM_PREC_FP32, zm.ZM_PREC_BF16X3):
        plan = zm.zm_plan(N_MAX, N_RHO, N_THETA, prec)
        zm.zm_moments(plan, views, out)
        torch.cuda.synchronize(dev)
        zm.zm_plan_destroy(plan)
    del os.environ["ZM_FUSED"]
    for var in ("ZM_RING_DFT", "ZM_POLAR_DFT"):   # the two tensor-core DFT kernels (opt-in) on the same frames
        os.environ[var] = "1"
        plan = zm.zm_plan(N_MAX, N_RHO, N_THETA, zm.ZM_PREC_BF16X3)
        zm.zm_moments(plan, views, out)
        torch.cuda.synchronize(dev)
        zm.zm_plan_destroy(plan)
        del os.environ[var]
    plan = zm.zm_plan(N_MAX, N_RHO, N_THETA, zm.ZM_PREC_BF16X3)
    bench_colour(zm, torch, dev, plan, P, steps=1)
    zm.zm_plan_destroy(plan)
    host = torch.empty((B, H, W), dtype=torch.float32, pin_memory=True)
    host.copy_(imgs.cpu())
    hv = [host[b] for b in range(B)]
    dbuf = torch.empty(zm.zm_upload_disk_bytes(hv) // 4 + 4, device=dev)
    zm.zm_upload_disk(hv, dbuf)
    big = torch.from_numpy(synth.blob_image(4000, 4000, 24, workload=SYNTH_WORKLOAD_ID, index=6000)).to(dev)
    cout = torch.empty((1, 1, 2), device=dev)
    work = torch.empty(zm.zm_cartesian_work_bytes(1, 1) // 8 + 1, dtype=torch.float64, device=dev)
    zm.zm_cartesian_moments([big], [(100, 36)], cout, work)
    specs = synth.uneven_batch_specs(count=64, workload=3)
    items = []
    for j, (size, n_max, n_rho, n_theta) in enumerate(specs):
        im = torch.from_numpy(synth.blob_image(size, size, 8, workload=3, index=j)).to(dev)
        items.append((im, n_max, n_rho, n_theta, torch.empty((zm.zm_num_moments(n_max), 2), device=dev)))
    b = zm.zm_batch_create(items, zm.ZM_PREC_FP16X3)
    zm.zm_batch_run(b, items)
    torch.cuda.synchronize(dev)
    zm.zm_batch_destroy(b)
    srv = zm.zm_server_create(1 << 30, 2, 8, zm.ZM_PREC_BF16X3)
    keep = []
    for j, (sz, nm) in enumerate([(256, 20), (512, 50), (1024, 100), (256, 20)]):
        im = synth.blob_image(sz, sz, 8, workload=5, index=j)
        o = np.empty((zm.zm_num_moments(nm), 2), np.float32)
        nt = 1
        while nt < 2 * nm + 2:
            nt *= 2
        keep.append((im, o))
        zm.zm_server_submit(srv, im, nm, sz // 2, nt, o)
    zm.zm_server_drain(srv)
    zm.zm_server_destroy(srv)
    torch.cuda.synchronize(dev)
    print(json.dumps({"profile_pass": "done", "launches": zm.zm_launch_count()}), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.profile_pass:
        profile_pass(args.batch)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
