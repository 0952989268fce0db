#!/usr/bin/env python
"""Benchmark: LM bundle-adjustment iterations per second on one synthetic
scene of 4,000 cameras, 1.2M points and ~8.04M observations (the ba4000
workload: views per point 2+Geom0(1/5.7), 1 px noise), FP32 per-observation
arithmetic with FP64 reductions, block-Jacobi PCG capped at 50 iterations.

A step is one LM trial: linearisation (when theta changed), block assembly,
Schur reduction, PCG on the reduced camera system, back-substitution, trial
cost and accept/reject -- all through the library's C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank solves its own
replica of the scene (no collective on the data path); value counts the
trials of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import os

for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import csv
import hashlib
import io
import json
import math
import signal
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import scenegen  # noqa: E402

METRIC = "LM iters/s and time-to-cost (1e-6 rel) vs plain GPU and oracle; HBM GB/s vs peak"
UNIT = "LM iters/s"
WORKLOAD = "ba4000"
PCG_MAXITER = 50
PCG_TOL = 1e-4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="trials of the end-to-end leg (default: --steps, the timed trials)")
    ap.add_argument("--profile-trials", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--jacobian", choices=["auto", "recompute", "store"], default="auto")
    ap.add_argument("--points", type=int, default=0,
                    help="profiling only: same recipe with fewer points")
    ap.add_argument("--workload", choices=["ba4000", "batch512", "learned", "adjoint"], default="ba4000",
                    help="batch512: 512 sliding-window problems solved by one persistent launch; "
                         "learned: time to 1e-6 relative cost with the learned block-Jacobi correction")
    ap.add_argument("--train-scenes", type=int, default=200, help="learned: training scenes")
    ap.add_argument("--batch-problems", type=int, default=512,
                    help="batch512: problems per rank (profiling only: a smaller batch of the same recipe)")
    ap.add_argument("--no-sequential", action="store_true",
                    help="batch512: skip the 512 sequential single-problem solves")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_max(value, device, world):
    """The largest value over all ranks (the slowest rank's time); the value
    itself on one rank.  No data-path collective: timing only."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def batch_seed(rank):
    """Seed of a rank's own batch of problems (weak scaling: every rank
    solves BATCH_N problems of its own, no data-path collective)."""
    return 4 + 1000 * rank


# --------------------------------------------------------------------------
# the CPU oracle on a bounded sample (cpu_baseline and --impl reference)
# --------------------------------------------------------------------------

def oracle_sample_rate(scene, n_obs_target, trials=1, warmup=0):
    """LM trials/s of the oracle on a sample of the scene, scaled to the full
    scene by its observation count (per-trial work is linear in O)."""
    import oracle as orc
    n_pts = max(50, int(round(n_obs_target * scene.P / scene.O)))
    sub = scenegen.subsample_points(scene, n_pts, seed=123)
    pix = orc.pixels_from_scene(sub)
    opts = orc.LMOptions(solver="pcg", pcg_tol=0.0, pcg_maxiter=PCG_MAXITER,
                         huber_delta=sub.huber_delta)
    if warmup:
        orc.lm(sub.cams_init, sub.points_init, sub.cam_idx, sub.pt_idx, pix, warmup, opts)
    t0 = time.perf_counter()
    _, _, tr = orc.lm(sub.cams_init, sub.points_init, sub.cam_idx, sub.pt_idx, pix, trials, opts)
    dt = time.perf_counter() - t0
    rate_sample = trials / dt
    return dict(rate_full=rate_sample * sub.O / scene.O, seconds=dt, O=sub.O, P=sub.P,
                trials=trials, pcg=[t["pcg_iters"] for t in tr])


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    scene = scenegen.config_scene(WORKLOAD)
    # per-step sample sized so (K + W) steps take about two minutes
    per_step_s = 120.0 / max(1, args.steps + args.warmup)
    n_obs = int(min(1_000_000, max(3000, per_step_s / 45e-6)))
    r = oracle_sample_rate(scene, n_obs, trials=args.steps, warmup=args.warmup)
    v = r["rate_full"]
    sample = (f"{r['P']} of {scene.P} points with their {r['O']} of {scene.O} observations, "
              f"all {scene.C} cameras; {args.steps} LM trials per run, PCG fixed at "
              f"{PCG_MAXITER} iterations; rate scaled by O_full/O_sample")
    line = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "cameras": scene.C, "points": scene.P,
                       "observations": scene.O, "pcg_maxiter": PCG_MAXITER},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.seek(0)
        text = self.f.read()
        os.unlink(self.f.name)
        return parse_clock_samples(text)


def parse_clock_samples(text):
    """Summary of nvidia-smi samples in the ClockSampler.Q column order
    (csv, no header, no units): median SM clock, the highest maximum clock,
    the throttle reasons seen Active in any sample, and the sample count;
    None without samples."""
    rows = [r for r in csv.reader(io.StringIO(text)) if len(r) >= 9]
    if not rows:
        return None
    sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def algorithmic_bytes(kind, C, P, O, npieces, tsize, mf, huber=False):
    """Compulsory HBM bytes of one launch: every array element the kernel
    must read or write, each counted once (per-observation planes, indices
    and weights; per-point / per-camera vectors once)."""
    ob = 18 * tsize if not mf else (tsize if huber else 0)   # planes or sqrt(w)
    if kind == "pass_b":   # cm_pt; point record (X, t) per point; camera table; partials
        return O * (4 + ob) + P * 8 * tsize + npieces * 9 * 8 + C * 16 * tsize
    if kind == "pass_a1":  # cm_pt (+ sqrt(w)) or planes in, one 4-vector out per obs; points once
        return O * (4 + ob + 4 * tsize) + (P * 4 * tsize if mf else 0) + C * (16 + 12) * tsize
    if kind == "pass_a2":  # order map + one 4-vector per obs; rowptr, V*^-1, t out per point
        return O * (4 + 4 * tsize) + P * (4 + 6 * tsize + 4 * tsize)
    if kind == "pass_fa":  # point index + chunk camera position (+ sqrt(w)) per obs; X in, V*^-1, t out per point
        return O * (4 + 2 + (tsize if huber else 0)) + P * (4 + 4 * tsize + 6 * tsize + 4 * tsize)
    if kind == "lin_cam":  # pixels + point index in; planes / weights out; points once; partials
        return O * (2 * tsize + 4 + ob) + P * 3 * tsize + npieces * 54 * 8
    if kind == "lin_pt":
        return O * (2 * tsize + 8 + ob) + P * (4 + 3 * tsize + 9 * 8) + C * 32 * tsize
    if kind == "schur_cam":
        return O * (4 + ob) + P * ((3 * tsize if mf else 0) + 9 * tsize) + npieces * 54 * 8
    if kind == "cost":     # pixels, point index, (model) planes; trial + current points, dp
        return O * (2 * tsize + 4 + ob) + P * 9 * tsize + npieces * 2 * 8
    if kind == "backsub":  # A1 + A2 of the back-substitution (two launches per trial)
        return (O * (4 + ob + 4 * tsize) + (P * 4 * tsize if mf else 0)
                + O * (4 + 4 * tsize) + P * (4 + 6 * tsize + 3 * tsize + 3 * 8 + 9 * tsize)) // 2
    return 0


# FP32 operations per observation of the recompute-mode passes (an FMA counts
# two): the factored Jacobian (61) plus the pass's products.
FLOPS_PER_OBS = {"pass_b": 119, "pass_a1": 113, "pass_fa": 116}


def fp32_peak_tflops(sm_mhz):
    """152 SMs x 128 FP32 lanes x 2 flops per FMA x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("ba_kernels.cuh", "ba_api.cu"):
        with open(os.path.join(ROOT, "paper_2409_12190_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, src_hash):
    """dram bytes per launch of the kernel from a committed ncu summary, only
    if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    e = d.get(kernel)
    if not e or e.get("source_hash") != src_hash:
        return None
    return e.get("dram_bytes_per_launch")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def run_ours(args):
    import torch
    import paper_2409_12190_gb300 as ba
    from paper_2409_12190_gb300 import build as bbuild

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    bbuild.build()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    if args.points:
        scene = scenegen.ring_scene(4000, args.points, seed=3, view_p=1.0 / 5.7, name="ba4000-small")
    else:
        scene = scenegen.config_scene(WORKLOAD)
    C, P, O = scene.C, scene.P, scene.O
    ci = torch.from_numpy(scene.cam_idx).to(dev)
    pi = torch.from_numpy(scene.pt_idx).to(dev)
    cams_gt = torch.tensor(scene.cams_gt, dtype=torch.float32, device=dev)
    pts_gt = torch.tensor(scene.points_gt, dtype=torch.float32, device=dev)
    pix = ba.project(cams_gt, pts_gt, ci, pi) + torch.tensor(scene.noise, dtype=torch.float32, device=dev)
    opts = ba.Options(precision="f32", pcg_maxiter=PCG_MAXITER, pcg_tol=PCG_TOL, use_graph=True,
                      jacobian=args.jacobian)
    mf = args.jacobian in ("auto", "recompute")
    prob = ba.Problem(scene.cams_init, scene.points_init, ci, pi, pix, opts, device=dev)
    torch.cuda.synchronize()

    # warm-up (captures the trial graph on first use)
    prob.solve(args.warmup)
    torch.cuda.synchronize()
    prob.stats()
    # the end-to-end leg below replays the timed trials from this state
    state0 = prob.get_state()

    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local) if rank == 0 else None
    time.sleep(0.3 if clocks else 0)
    barrier()
    torch.cuda.synchronize()
    n0 = ba.kernel_launch_count()
    e0.record(stream)
    prob.solve(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = ba.kernel_launch_count() - n0
    clk = clocks.stop() if clocks else None
    ms = e0.elapsed_time(e1)
    ms = rank_max(ms, dev, world)
    trials = prob.stats(cap=args.steps)
    value = world * args.steps / (ms / 1000.0)

    # per-kernel CUDA-event timing of the same trials (direct launches)
    per, prof_ms = prob.profile_trials(args.profile_trials)
    tsize = 4
    npieces = sum(max(1, math.ceil(n / 2048)) if n > 0 else 0 for n in np.bincount(scene.cam_idx, minlength=C))
    total = sum(v[0] for v in per.values())
    kernels = {}
    peak, peak_kind = peaks()
    sm_mhz = (clk or {}).get("sm_max_mhz") or 2070.0
    alu_peak = fp32_peak_tflops(sm_mhz)
    for name, (kms, n) in per.items():
        if n == 0:
            continue
        b = algorithmic_bytes(name, C, P, O, npieces, tsize, mf)
        avg = kms / n
        kernels[name] = {"launches": n, "avg_us": 1000.0 * avg, "share": kms / total,
                         "gbs": (b / (avg / 1000.0) / 1e9) if b else None}
        if mf and name in FLOPS_PER_OBS:
            kernels[name]["tflops"] = FLOPS_PER_OBS[name] * O / (avg / 1000.0) / 1e12
    dom = max((k for k in kernels if kernels[k]["gbs"]), key=lambda k: per[k][0])
    src_hash = kernel_source_hash()
    ach = kernels[dom]["gbs"]
    roofline = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "peak_source": peak_kind,
                "bytes_per_launch": algorithmic_bytes(dom, C, P, O, npieces, tsize, mf),
                "traffic": measured_traffic(dom, src_hash), "kernel_source": src_hash}
    if "tflops" in kernels[dom]:
        alu = {"achieved": kernels[dom]["tflops"], "peak": alu_peak, "unit": "TFLOP/s",
               "frac": kernels[dom]["tflops"] / alu_peak,
               "flops_per_launch": FLOPS_PER_OBS[dom] * O,
               "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz"}
        roofline["hbm"] = {k: roofline[k] for k in ("achieved", "peak", "unit", "frac")}
        roofline["alu"] = alu
        if alu["frac"] > roofline["frac"]:
            roofline.update({"bound": "alu", "achieved": alu["achieved"], "peak": alu["peak"],
                             "unit": alu["unit"], "frac": alu["frac"], "peak_source": alu["peak_source"]})
    # whole-iteration algorithmic bandwidth (bytes of all big passes / trial time)
    it_bytes = sum(algorithmic_bytes(k, C, P, O, npieces, tsize, mf) * per[k][1] for k in per)
    roofline["iteration_gbs"] = it_bytes / (prof_ms / 1000.0) / 1e9
    roofline["iteration_frac"] = roofline["iteration_gbs"] / peak

    # end to end through the public API: the same trials as the timed region
    # (restarted from its starting state), each step uploading parameters and
    # pixels from pinned host memory and reading parameters and cost back
    e2e_steps = args.e2e_steps if args.e2e_steps > 0 else args.steps
    prob.set_state(state0)
    hc = torch.empty((C, 9), dtype=torch.float32).pin_memory()
    hp = torch.empty((P, 3), dtype=torch.float32).pin_memory()
    hx = pix.cpu().pin_memory()
    prob.get_params_into(hc, hp)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        prob.set_params(hc, hp)
        prob.set_pixels(hx)
        prob.lm_step()
        prob.get_params_into(hc, hp)
        cost, _ = prob.scalars()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = rank_max(e2e_s, dev, world)
    e2e_trials = prob.stats(cap=e2e_steps)
    same = ([t["pcg_iters"] for t in e2e_trials] == [t["pcg_iters"] for t in trials[:e2e_steps]]
            and [t["accepted"] for t in e2e_trials] == [t["accepted"] for t in trials[:e2e_steps]])
    e2e = {"value": world * e2e_steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": (9 * C + 3 * P + 2 * O) * 4,
           "d2h_bytes_per_step": (9 * C + 3 * P) * 4 + 8, "steps": e2e_steps,
           "same_trials_as_timed": same}

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        r = oracle_sample_rate(scene, 500_000, trials=1)
        cpu = {"value": r["rate_full"], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": (f"1 LM trial on {r['P']} of {P} points with their {r['O']} of {O} "
                          f"observations, all {C} cameras, PCG fixed at {PCG_MAXITER} iterations, "
                          f"{r['seconds']:.1f} s; rate scaled by O_full/O_sample")}
    pcg = [t["pcg_iters"] for t in trials]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": scene.name, "cameras": C, "points": P, "observations": O,
                       "precision": "f32 per-observation, f64 reductions", "loss": "squared",
                       "pcg": f"block-Jacobi, maxiter {PCG_MAXITER}, tol {PCG_TOL}",
                       "pcg_iters_mean": statistics.mean(pcg) if pcg else None,
                       "pcg_iters_total": sum(pcg),
                       "accepted": sum(t["accepted"] for t in trials),
                       "l2": "inputs larger than L2 (each PCG pass streams >0.6 GB of "
                             "per-observation data; L2 129 MB)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "graph": "one CUDA graph per LM trial",
                       "jacobian": "recomputed in every pass" if mf else "stored planes"},
            "gpu_launches": launches, "clocks": clk, "roofline": roofline,
            "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e}
    print(json.dumps(line), flush=True)
    prob.close()


# --------------------------------------------------------------------------
# batch512: many small problems, one persistent launch per solve
# --------------------------------------------------------------------------

BATCH_N = 512
BATCH_ITERS = 10
# FP32 operations per observation and PCG iteration of the batched kernel's
# passes A1 and B (recompute mode, as for the single-problem kernels)
BATCH_FLOPS_PER_OBS_PCG = FLOPS_PER_OBS["pass_a1"] + FLOPS_PER_OBS["pass_b"]


def run_batch(args):
    import torch
    import paper_2409_12190_gb300 as ba
    from paper_2409_12190_gb300 import build as bbuild

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    bbuild.build()
    n_prob = args.batch_problems
    scenes = scenegen.batch_scenes(n_prob, seed=batch_seed(rank))
    O = sum(s.O for s in scenes)
    inputs = []
    for s in scenes:
        ci = torch.from_numpy(s.cam_idx).to(dev)
        pi = torch.from_numpy(s.pt_idx).to(dev)
        px = ba.project(torch.tensor(s.cams_gt, dtype=torch.float32, device=dev),
                        torch.tensor(s.points_gt, dtype=torch.float32, device=dev), ci, pi)
        px = px + torch.tensor(s.noise, dtype=torch.float32, device=dev)
        inputs.append((s.cams_init, s.points_init, ci, pi, px))
    opts = ba.Options(precision="f32", pcg_maxiter=PCG_MAXITER, pcg_tol=PCG_TOL)
    bt = ba.Batch(inputs, opts, device=dev)
    cache = os.path.join(ROOT, "paper_2409_12190_gb300", ".autotune.jsonl")
    cfg, tune_ms = bt.autotune(BATCH_ITERS, cache)
    for _ in range(args.warmup):
        bt.reset()
        bt.solve(BATCH_ITERS)
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local) if rank == 0 else None
    time.sleep(0.3 if clocks else 0)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    n0 = ba.kernel_launch_count()
    e0.record(stream)
    for _ in range(args.steps):
        bt.reset()
        bt.solve(BATCH_ITERS)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = ba.kernel_launch_count() - n0
    clk = clocks.stop() if clocks else None
    ms = e0.elapsed_time(e1)
    ms = rank_max(ms, dev, world)
    stats = bt.stats()
    pcg_total = sum(t["pcg_iters"] for st in stats for t in st)
    costs, _ = bt.scalars()
    # problem-iterations per second over all ranks
    value = world * n_prob * BATCH_ITERS * args.steps / (ms / 1000.0)

    # the solve alone (one persistent launch, no reset) for the roofline
    bt.reset()
    torch.cuda.synchronize()
    e0.record(stream)
    bt.solve(BATCH_ITERS)
    e1.record(stream)
    torch.cuda.synchronize()
    solve_ms = e0.elapsed_time(e1)
    st2 = bt.stats()
    pcg_obs = sum(t["pcg_iters"] * s.O for st, s in zip(st2, scenes) for t in st)
    flops = BATCH_FLOPS_PER_OBS_PCG * pcg_obs
    sm_mhz = (clk or {}).get("sm_max_mhz") or 2070.0
    alu_peak = fp32_peak_tflops(sm_mhz)
    ach = flops / (solve_ms / 1000.0) / 1e12
    roofline = {"bound": "alu", "kernel": "k_batch_lm", "achieved": ach, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": ach / alu_peak, "flops_per_launch": flops,
                "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz",
                "note": "PCG passes A1+B only (113+119 FP32 flops per observation and PCG iteration); "
                        "each problem's arrays stay in L2 across its trials", "traffic": None}

    # end to end: pinned host parameters in, solve, parameters out
    C, P = bt.C, bt.P
    hc = torch.from_numpy(np.concatenate([s.cams_init for s in scenes]).astype(np.float32)).pin_memory()
    hp = torch.from_numpy(np.concatenate([s.points_init for s in scenes]).astype(np.float32)).pin_memory()
    oc = torch.empty((C, 9), dtype=torch.float32).pin_memory()
    op = torch.empty((P, 3), dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    e2e_steps = args.e2e_steps if args.e2e_steps > 0 else args.steps
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        bt.reset(hc, hp)
        bt.solve(BATCH_ITERS)
        cams_d, pts_d = bt.params(split=False)
        oc.copy_(cams_d, non_blocking=True)
        op.copy_(pts_d, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": world * n_prob * BATCH_ITERS * e2e_steps / e2e_s, "unit": "problem LM iters/s",
           "h2d_bytes_per_step": (9 * C + 3 * P) * 4, "d2h_bytes_per_step": (9 * C + 3 * P) * 4,
           "steps": e2e_steps}

    if rank != 0:
        return
    seq = None
    if world == 1 and not args.no_sequential:
        # the same problems solved one after another by the single-problem path
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        tot = 0.0
        worst = 0.0
        for b, inp in enumerate(inputs):
            pr = ba.Problem(*inp, options=opts, device=dev)
            torch.cuda.synchronize()
            ev0.record(stream)
            pr.solve(BATCH_ITERS)
            ev1.record(stream)
            torch.cuda.synchronize()
            tot += ev0.elapsed_time(ev1)
            F, _ = pr.scalars()
            worst = max(worst, abs(costs[b] - F) / F)
            pr.close()
        seq = {"ms": tot, "problem_iters_per_s": n_prob * BATCH_ITERS / (tot / 1000.0),
               "speedup_of_batch": tot / solve_ms, "max_rel_final_cost_diff": worst}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle as orc
        t0 = time.perf_counter()
        n_done, obs_done = 0, 0
        for s in scenes[:3]:
            pix = orc.pixels_from_scene(s)
            orc.lm(s.cams_init, s.points_init, s.cam_idx, s.pt_idx, pix, BATCH_ITERS,
                   orc.LMOptions(solver="pcg", pcg_tol=PCG_TOL, pcg_maxiter=PCG_MAXITER))
            n_done += 1
            obs_done += s.O
        dt = time.perf_counter() - t0
        rate = n_done * BATCH_ITERS / dt * (obs_done / n_done) / (O / n_prob)
        cpu = {"value": rate, "unit": "problem LM iters/s", "cores": 1, "kind": "oracle",
               "sample": f"{n_done} of {n_prob} problems ({obs_done} observations), {BATCH_ITERS} LM trials "
                         f"each, {dt:.1f} s; rate scaled to the mean problem size"}
    line = {"metric": METRIC, "value": value, "unit": "problem LM iters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "batch512" if n_prob == BATCH_N else f"batch{n_prob}", "problems": n_prob,
                       "lm_iters_per_problem": BATCH_ITERS,
                       "cameras": bt.C, "points": bt.P, "observations": O,
                       "pcg": f"block-Jacobi, maxiter {PCG_MAXITER}, tol {PCG_TOL}",
                       "pcg_iters_mean": pcg_total / max(1, n_prob * BATCH_ITERS),
                       "step": "reset + one persistent launch solving every problem for 10 LM trials",
                       "launch": cfg, "l2": "per-problem arrays L2-resident by design; no flush"},
            "gpu_launches": launches, "clocks": clk, "roofline": roofline, "solve_ms": solve_ms,
            "sequential_single_problem": seq, "cpu_baseline": cpu, "e2e": e2e}
    print(json.dumps(line), flush=True)
    bt.close()


# --------------------------------------------------------------------------
# learned: the learned block-Jacobi correction against block-Jacobi
# --------------------------------------------------------------------------

LEARN_PCG_TOL = 1e-5
LEARN_PCG_MAXITER = 500
LEARN_TRIALS = 20


def _timed_trials(prob, trials, stream):
    """Run `trials` LM trials one by one with an event after each; returns
    (seconds after each trial, cost after each trial, PCG iterations)."""
    import torch
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(trials + 1)]
    evs[0].record(stream)
    for i in range(trials):
        prob.solve(1)
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    st = prob.stats(cap=trials, raise_nonfinite=False)
    t = [evs[0].elapsed_time(e) / 1000.0 for e in evs[1:]]
    cost = [s["cost_trial"] if s["accepted"] else s["cost"] for s in st]
    bad = sum(1 for s in st if not math.isfinite(s["cost_trial"]))
    return t, cost, [s["pcg_iters"] for s in st], bad


def time_to_cost(runs, f_ref, rel=1e-6):
    """Time to a fixed cost: runs maps a name to (cumulative seconds after
    each trial, cost after each trial, PCG iterations per trial, non-finite
    trials).  A run reaches the target at its first trial whose cost is at or
    below (1 + rel) f_ref; a run that never gets there has no time (None),
    however close it ends."""
    out = {}
    for name, (t, cost, pcg, bad) in runs.items():
        hit = next((i for i, c in enumerate(cost) if c <= (1 + rel) * f_ref), None)
        out[name] = {"time_to_cost_s": t[hit] if hit is not None else None,
                     "trials_to_cost": None if hit is None else hit + 1,
                     "pcg_iters_to_cost": None if hit is None else sum(pcg[:hit + 1]), "final_cost": cost[-1],
                     "lowest_cost": min(cost), "ms_per_pcg_iter": 1000.0 * t[-1] / max(1, sum(pcg)),
                     "pcg_iters_per_trial": pcg, "cost_per_trial": cost, "nonfinite_trials": bad}
    return out


def speedup(out, base, other):
    """Ratio of the base run's time to cost to the other's; None unless both
    reached the target."""
    a, b = out[base]["time_to_cost_s"], out[other]["time_to_cost_s"]
    return a / b if a is not None and b is not None and b > 0 else None


def run_learned(args):
    import torch
    import paper_2409_12190_gb300 as ba
    from paper_2409_12190_gb300 import build as bbuild, learned
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    bbuild.build()

    def make(scene, prec="f32", tol=1e-4, maxiter=50):
        ci = torch.from_numpy(scene.cam_idx).to(dev)
        pi = torch.from_numpy(scene.pt_idx).to(dev)
        dt = torch.float32 if prec == "f32" else torch.float64
        px = ba.project(torch.tensor(scene.cams_gt, dtype=dt, device=dev), torch.tensor(scene.points_gt, dtype=dt, device=dev),
                        ci, pi) + torch.tensor(scene.noise, dtype=dt, device=dev)
        return ba.Problem(scene.cams_init, scene.points_init, ci, pi, px,
                          ba.Options(precision=prec, pcg_maxiter=maxiter, pcg_tol=tol), device=dev)

    # training set: ring scenes of 500-2,000 cameras (seeds 1000..)
    t0 = time.perf_counter()
    rng = np.random.default_rng(1000)
    samples = []
    for i in range(args.train_scenes):
        C = int(rng.integers(500, 2001))
        sc = scenegen.ring_scene(C, 30 * C, seed=1000 + i, view_p=1.0 / 5.7, name=f"train{i}")
        with make(sc) as pr:
            samples.append(learned.collect(pr, seed=i))
    t_collect = time.perf_counter() - t0
    n_samples = sum(s[0].shape[0] for s in samples)
    t0 = time.perf_counter()
    params, hist = learned.train(samples, epochs=100, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del samples

    # evaluation on the bench scene: block-Jacobi, then the learned blocks
    scene = scenegen.config_scene(WORKLOAD)
    stream = torch.cuda.current_stream()
    runs = {}
    for name, par in (("block_jacobi", None), ("learned", params)):
        with make(scene, tol=LEARN_PCG_TOL, maxiter=LEARN_PCG_MAXITER) as pr:
            pr.set_preconditioner(par)
            pr.solve(1)  # warm-up: captures the trial graph
            pr.set_params(torch.tensor(scene.cams_init, dtype=torch.float32, device=dev),
                          torch.tensor(scene.points_init, dtype=torch.float32, device=dev))
            pr.set_lambda(1e-4)
            pr.stats()
            runs[name] = _timed_trials(pr, LEARN_TRIALS, stream)
    # the target is the plain method's own best cost: the learned run must
    # reach what block-Jacobi reaches, to 1e-6 relative
    f_ref = min(runs["block_jacobi"][1])
    out = time_to_cost(runs, f_ref)
    value = out["learned"]["time_to_cost_s"]
    line = {"metric": METRIC, "value": value, "unit": "s to 1e-6 relative cost", "n_gpus": 1,
            "steps": LEARN_TRIALS, "warmup": 1, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": scene.name, "cameras": scene.C, "points": scene.P, "observations": scene.O,
                       "pcg": f"tol {LEARN_PCG_TOL}, maxiter {LEARN_PCG_MAXITER}",
                       "f_ref": f_ref, "f_ref_rule": "block-Jacobi's lowest cost; the learned run has no time if it never reaches it",
                       "training": {"scenes": args.train_scenes, "cameras": "500-2000", "points_per_camera": 30,
                                    "samples": n_samples, "epochs": 100, "collect_s": t_collect, "train_s": t_train,
                                    "loss_first_last": [hist[0], hist[-1]]}},
            "block_jacobi": out["block_jacobi"], "learned": out["learned"],
            "speedup_time_to_cost": speedup(out, "block_jacobi", "learned")}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# adjoint: the implicit-function adjoint (ba_backward) on the ba64 scene
# --------------------------------------------------------------------------

def run_adjoint(args):
    import torch
    import paper_2409_12190_gb300 as ba
    from paper_2409_12190_gb300 import build as bbuild
    import oracle as orc
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    bbuild.build()
    scene = scenegen.config_scene("ba64")
    ci = torch.from_numpy(scene.cam_idx).to(dev)
    pi = torch.from_numpy(scene.pt_idx).to(dev)
    px = ba.project(torch.tensor(scene.cams_gt, device=dev), torch.tensor(scene.points_gt, device=dev), ci, pi) + \
        torch.tensor(scene.noise, device=dev)
    fixed = np.zeros((scene.C, 9), dtype=bool)
    fixed[0, :] = True
    fixed[1, 3] = True
    prob = ba.Problem(scene.cams_init, scene.points_init, ci, pi, px,
                      ba.Options(precision="f64", pcg_maxiter=600, pcg_tol=1e-12, lambda0=1e-6), device=dev)
    prob.set_fixed(torch.from_numpy(fixed))
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    prob.solve(30)
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1)
    cams, pts = prob.params()
    tgt = torch.tensor(scene.cams_gt[:, 3:6], device=dev)
    g = torch.zeros_like(cams)
    g[:, 3:6] = 2.0 * (cams[:, 3:6] - tgt)
    lam, maxiter, tol = 1e-8, 2000, 1e-12
    for _ in range(args.warmup):
        prob.backward(g, None, lam=lam, maxiter=maxiter, tol=tol)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        dpix, dc0, _, its, rel = prob.backward(g, None, lam=lam, maxiter=maxiter, tol=tol)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    # the oracle's adjoint at the GPU's converged parameters, timed on the host
    t0 = time.perf_counter()
    ref_pix, ref_c0, _, _ = orc.adjoint_schur(cams.cpu().numpy(), pts.cpu().numpy(), scene.cam_idx, scene.pt_idx,
                                              px.cpu().numpy(), g.cpu().numpy(), np.zeros((scene.P, 3)), fixed,
                                              0.0, lam)
    t_orc = time.perf_counter() - t0
    err = float(np.max(np.abs(dpix.cpu().numpy() - ref_pix)) / np.max(np.abs(ref_pix)))
    line = {"metric": METRIC, "value": 1000.0 / ms, "unit": "adjoint solves/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "ba64", "cameras": scene.C, "points": scene.P, "observations": scene.O,
                       "loss": "sum over cameras of |t - t_gt|^2", "gauge": "camera 0 and t_x of camera 1 frozen",
                       "forward": "30 LM trials, FP64, PCG tol 1e-12", "adjoint_pcg": f"tol {tol}, maxiter {maxiter}",
                       "step": "one ba_backward: linearisation, Schur/PCG solve of H v = dL/dtheta, dL/dpixels"},
            "forward_ms_30_trials": fwd_ms, "adjoint_pcg_iters": its, "adjoint_rel_res": rel,
            "max_rel_err_vs_oracle_dense_adjoint": err,
            "cpu_baseline": {"value": 1.0 / t_orc, "unit": "adjoint solves/s", "cores": 1, "kind": "oracle",
                             "sample": f"the whole ba64 adjoint (explicit Schur, dense Cholesky), {t_orc:.1f} s"}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch512":
        run_batch(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
