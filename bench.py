#!/usr/bin/env python3
"""FilterReg hot-path benchmark: EM iterations per second of rigid
point-to-plane registration on 320x240 synthetic depth frames (76,800 model
points, ~72,960 observation points after 5% dropout, sigma annealed
0.04 -> 0.01 over 20 EM iterations, outlier ratio 0.1).

One step = registering a batch of B frame pairs (B = --frames, default 16)
with fr_register_rigid_batch -- one launch per EM iteration for the whole
batch -- i.e. B x 20 EM iterations.  The plain path (fr_register_rigid, one
pair at a time) is timed on the same frames beside it.  The L2 cache is
flushed (256 MiB write) between steps; per-step device time is taken with
CUDA events on the library's stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: every rank registers its own frames (replicas, no
collective on the data path); the job's value is the frames of all ranks over
the slowest rank's time.  --impl reference times the CPU oracle (the paper's
method restated plainly in C, OpenMP over every host core) on the same
workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "EM iters/s at 76.8k pts; batched regs/s + p99 latency vs plain, <=0.1 deg err"
UNIT = "EM iters/s"
ITERS = 20
SIGMA0, SIGMA1, W_OUT = 0.04, 0.01, 0.1
FEAT_SIGMA_P, FEAT_SIGMA_N = 0.02, 0.25   # feature E step: position (m) and normal bandwidths
# recovery sweep: a bumpy sphere whose bumps make the rotation observable
SPHERE_RECOVERY = dict(amp=0.5, width=0.35, max_trans=0.05, exact_angle=True)
ART_ITERS, ART_SIGMA = 15, 0.01      # articulated workload: 15 EM iterations at sigma 1 cm
NG_ITERS, NG_PCG, NG_SIGMA, NG_LAMBDA = 10, 20, 0.02, 10.0  # node-graph workload
SERVE_RATE = 2000.0                   # serving stream: Poisson arrivals per second
SERVE_BUDGET = 32 << 30               # server device memory (bytes): tables and records of ~300 live requests


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames", type=int, default=16, help="frame pairs registered per step")
    ap.add_argument("--seed", type=int, default=1000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-precision", action="store_true", help="skip the 16-bit storage lines")
    ap.add_argument("--no-articulated", action="store_true", help="skip the articulated line")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving stream")
    ap.add_argument("--no-nodegraph", action="store_true", help="skip the node-graph line")
    ap.add_argument("--no-exact", action="store_true", help="skip the exact Gauss-transform line")
    ap.add_argument("--no-sigma", action="store_true", help="skip the updated-sigma line")
    ap.add_argument("--no-features", action="store_true", help="skip the feature-space E-step line")
    ap.add_argument("--no-recovery", action="store_true", help="skip the recovery-range sweeps")
    ap.add_argument("--no-tune", action="store_true", help="keep the built-in launch shapes (no autotuning)")
    ap.add_argument("--serve-requests", type=int, default=4096)
    ap.add_argument("--serve-pool", type=int, default=32, help="distinct rendered frames behind the stream")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seed(seed, rank):
    """Each rank registers its own frames (weak scaling: fixed work per GPU)."""
    return seed + 7919 * rank


def max_over_ranks(x, dist=None, device="cpu"):
    """The slowest rank's time: the job is done when the last rank is."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, slowest_s):
    """Units processed by all ranks per second of the slowest rank."""
    return units_per_rank * world / slowest_s


def workload_config(frames, pairs):
    Ns = [p.Y.shape[0] for p in pairs]
    return {
        "workload": "depth_frames_320x240_pt2pl",
        "model": "rigid FilterReg, point-to-plane, permutohedral E step (splat+slice), batched",
        "points_per_frame": 76800,
        "M": int(pairs[0].X.shape[0]),
        "N_mean": int(round(sum(Ns) / len(Ns))),
        "frames_per_step": frames,
        "em_iters": ITERS,
        "sigma": f"{SIGMA0}->{SIGMA1} geometric",
        "w": W_OUT,
        "blur": False,
        "l2": "flushed between steps (256 MiB write)",
        "global_batch": frames,
        "parallelism": "replicas",
    }


def make_pairs(seed, n):
    from paper_1811_10136_gb300 import synth
    return [synth.depth_frame_pair(seed + i) for i in range(n)]


def serving_requests(seed, n_requests, pool_size):
    """The serving stream: Poisson arrivals, sizes log-uniform in [1k, 300k]
    points (frames rendered like the 320x240 workload at 4:3, W*H ~ n/0.95,
    focal length scaled with W), sigma uniform in {0.01, 0.02, 0.04} (fixed per
    request), 20 iterations.  Rendering 4096 distinct frames would take minutes,
    so requests draw their clouds from a pool of pool_size rendered pairs whose
    sizes follow the same distribution; arrival times, sigmas and the pool
    entry are drawn per request."""
    import numpy as np
    from paper_1811_10136_gb300 import synth
    rng = np.random.default_rng(seed)
    pool = []
    for i in range(pool_size):
        n = float(np.exp(rng.uniform(np.log(1000.0), np.log(300000.0))))
        W = max(8, int(round(np.sqrt(n / 0.95 * 4.0 / 3.0))))
        H = max(6, int(round(W * 3 / 4)))
        pool.append(synth.depth_frame_pair(seed + 50_000 + i, W=W, H=H, fx=300.0 * W / 320, fy=300.0 * W / 320))
    gaps = rng.exponential(1.0 / SERVE_RATE, n_requests)
    arrivals = np.cumsum(gaps) - gaps[0]
    which = rng.integers(0, pool_size, n_requests)
    sigmas = rng.choice(np.array([0.01, 0.02, 0.04], np.float32), n_requests)
    return pool, arrivals, which, sigmas


def serving_pool(args):
    import torch
    pool, arrivals, which, sigmas = serving_requests(args.seed + 11, args.serve_requests, args.serve_pool)
    dpool = [(torch.from_numpy(p.X).cuda(), torch.from_numpy(p.Y).cuda(), torch.from_numpy(p.Yn).cuda())
             for p in pool]
    return pool, dpool, arrivals, which, sigmas


def tune_serving(ctx, pool, dpool):
    """Latency objective per size class: points per thread of a serving
    tick's blocks, timed on up to 4 pool frames of the class."""
    import numpy as np
    import paper_1811_10136_gb300 as fr
    bounds = [4096, 16384, 65536, 262144, 1 << 62]
    out = {}
    for c, hi in enumerate(bounds):
        lo = bounds[c - 1] if c else 0
        idx = [i for i, p in enumerate(pool) if lo < p.Y.shape[0] <= hi][:4]
        if not idx:
            continue
        best, b_ms, d_ms = ctx.autotune_batch([dpool[i] for i in idx], objective=fr.FR_TUNE_LATENCY, reps=3,
                                              residual=fr.FR_PT2PL, iters=ITERS, sigma_start=0.02,
                                              sigma_end=0.02, w=W_OUT)
        out[f"N<={hi}" if hi < (1 << 62) else f"N>{lo}"] = {
            "serve_points_per_thread": best["serve_points_per_thread"], "ms": round(b_ms, 4),
            "default_ms": round(d_ms, 4), "frames": len(idx)}
    return out


def run_serving(ctx, args, pool, dpool, arrivals, which, sigmas, plain=True, storage=0):
    """Open-loop stream through fr_server (continuous batching) and, on the
    same arrivals, through the plain path (fr_register_rigid, one request at
    a time, first come first served).  Latency = completion - arrival.
    storage != FR_FP32: the server keeps 16-bit lattice records, and the
    largest pose difference from a float32 server run is reported."""
    import numpy as np
    import paper_1811_10136_gb300 as fr
    n = len(arrivals)
    opts = dict(residual=fr.FR_PT2PL, iters=ITERS)

    def spin_until(t_ns):
        while time.monotonic_ns() < t_ns:
            pass

    def percentiles(lat):
        lat = np.sort(np.asarray(lat))
        return (float(np.percentile(lat, 50)), float(np.percentile(lat, 99)))

    out = {"workload": "poisson_stream_1k_300k_points", "requests": n, "arrival_rate_per_s": SERVE_RATE,
           "pool_frames": len(pool), "em_iters": ITERS, "sigma": "one of 0.01/0.02/0.04 per request, fixed",
           "sizes_mean_points": int(np.mean([pool[k].Y.shape[0] for k in which]))}
    with fr.Server(ctx, budget_bytes=SERVE_BUDGET, max_live=1024, storage=storage, **opts) as srv:
        # warm-up: one of each pool frame
        for t in [srv.submit(*dpool[i], sigma_start=0.02, w=W_OUT) for i in range(len(pool))]:
            srv.wait(t)
        st0 = srv.stats()
        t0 = time.monotonic_ns() + 2_000_000
        tickets = []
        for k in range(n):
            spin_until(t0 + int(arrivals[k] * 1e9))
            X, Y, Yn = dpool[which[k]]
            tickets.append(srv.submit(X, Y, Yn, sigma_start=float(sigmas[k]), w=W_OUT))
        res = [srv.wait(t) for t in tickets]
        st1 = srv.stats()
        lat = [(r.complete_ns - (t0 + int(a * 1e9))) * 1e-6 for r, a in zip(res, arrivals)]
        span = (max(r.complete_ns for r in res) - t0) * 1e-9
        p50, p99 = percentiles(lat)
        out["_T"] = [r.T for r in res]
        out.update({"regs_per_s": round(n / span, 1), "latency_ms_p50": round(p50, 3),
                    "latency_ms_p99": round(p99, 3),
                    "ticks": st1["ticks"] - st0["ticks"], "gpu_launches": st1["kernel_launches"] - st0["kernel_launches"],
                    "failed": sum(1 for r in res if r.status != 0)})
        # saturated throughput: every request submitted at once
        t1 = time.monotonic_ns()
        tk = [srv.submit(*dpool[which[k]], sigma_start=float(sigmas[k]), w=W_OUT) for k in range(n)]
        sat = [srv.wait(t) for t in tk]
        out["saturated_regs_per_s"] = round(n / ((max(r.complete_ns for r in sat) - t1) * 1e-9), 1)
    if not plain:
        return out
    # the plain path on the same arrivals
    plain_T = []
    lat_p = []
    t0 = time.monotonic_ns() + 2_000_000
    for k in range(n):
        a = t0 + int(arrivals[k] * 1e9)
        spin_until(a)
        X, Y, Yn = dpool[which[k]]
        T, _ = ctx.register_rigid(X, Y, Yn, sigma_start=float(sigmas[k]), sigma_end=float(sigmas[k]),
                                  w=W_OUT, **opts)
        lat_p.append((time.monotonic_ns() - a) * 1e-6)
        plain_T.append(T)
    span_p = (time.monotonic_ns() - t0) * 1e-9
    q50, q99 = percentiles(lat_p)
    # saturated plain path: every request queued, registered one at a time
    t1 = time.monotonic_ns()
    for k in range(n):
        ctx.register_rigid(*dpool[which[k]], sigma_start=float(sigmas[k]), sigma_end=float(sigmas[k]),
                           w=W_OUT, **opts)
    sat_p = n / ((time.monotonic_ns() - t1) * 1e-9)
    out["plain"] = {"regs_per_s": round(n / span_p, 1), "latency_ms_p50": round(q50, 3),
                    "latency_ms_p99": round(q99, 3), "saturated_regs_per_s": round(sat_p, 1),
                    "note": "fr_register_rigid per request, first come first served, same arrivals; "
                            "saturated: all requests queued, one at a time"}
    out["max_rot_diff_deg_vs_plain"] = round(max(synth_rot(r.T, T) for r, T in zip(res, plain_T)), 6)
    return out


def synth_rot(A, B):
    from paper_1811_10136_gb300 import synth
    return synth.rotation_angle_deg(A, B)


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.rows = []
        self.proc = None
        self.dev = device_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in self.rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s in sm if mx and s >= 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(self.rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in self.rows)}


# ---------------------------------------------------------------------------
# roofline helpers
# ---------------------------------------------------------------------------

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("kernels.cu", "lattice.cuh", "internal.h"):
        with open(os.path.join(ROOT, "paper_1811_10136_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was captured from the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic_depth320.txt")
    try:
        rows = dict(line.split(":", 1) for line in open(path) if ":" in line and not line.startswith("#"))
    except OSError:
        return None
    rows = {k.strip(): v.strip() for k, v in rows.items()}
    if rows.get("kernel_source_hash") != kernel_source_hash():
        return None
    v = rows.get(f"{kernel}_dram_bytes_per_launch")
    return float(v) if v else None


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch

    import paper_1811_10136_gb300 as fr
    from paper_1811_10136_gb300 import synth

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    pairs = make_pairs(rank_seed(args.seed, rank), args.frames)
    dev = lambda a: torch.from_numpy(a).cuda()
    dpairs = [(dev(p.X), dev(p.Y), dev(p.Yn)) for p in pairs]
    ctx = fr.Context(local, tune_table=None)   # built-in shapes; tuned in this run below
    opts = dict(residual=fr.FR_PT2PL, iters=ITERS, sigma_start=SIGMA0, sigma_end=SIGMA1, w=W_OUT)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def batched_step():
        return ctx.register_rigid_batch(dpairs, **opts)

    def plain_step():
        return [ctx.register_rigid(X, Y, Yn, **opts) for X, Y, Yn in dpairs]

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def timed_steps(fn, k_steps):
        """k_steps steps, L2 flushed before each; per-step CUDA-event times (ms)."""
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(k_steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(k_steps)]
        last = None
        for k in range(k_steps):
            flush.fill_(1.0)
            starts[k].record(stream)
            last = fn()
            ends[k].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in zip(starts, ends)], last

    def slowest(total_s):
        return max_over_ranks(total_s, dist, "cuda")

    for _ in range(args.warmup):
        flush.fill_(1.0)
        batched_step()
        plain_step()

    # ---- launch-shape autotuning of the batched path (outside the timed region)
    tuning = None
    if not args.no_tune:
        best, tuned_ms, default_ms = ctx.autotune_batch(dpairs, objective=fr.FR_TUNE_THROUGHPUT, reps=3, **opts)
    if not args.no_tune:
        tuning = {"params": best, "em_iters_per_s_tuned": round(ITERS * args.frames / (tuned_ms * 1e-3), 1),
                  "em_iters_per_s_default": round(ITERS * args.frames / (default_ms * 1e-3), 1),
                  "timing": "median of 3 whole batched calls (CUDA events) per candidate shape, L2 warm"}
    for _ in range(2):
        batched_step()

    # ---- timed region: K batched steps (the headline) ------------------------
    launches0 = ctx.kernel_launches
    barrier()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        step_ms, last = timed_steps(batched_step, args.steps)
        barrier()
        t_wall = time.perf_counter() - t_wall
    launches = ctx.kernel_launches - launches0
    total_s = slowest(sum(step_ms) / 1000.0)
    em_iters_all = ITERS * args.frames * args.steps * ws
    value = whole_job_rate(ITERS * args.frames * args.steps, ws, total_s)

    # ---- the plain path (one registration at a time, float32) on the same frames
    plain_ms, plain_last = timed_steps(plain_step, args.steps)
    plain_s = slowest(sum(plain_ms) / 1000.0)
    reg_lat_ms = []
    for X, Y, Yn in dpairs[: min(8, len(dpairs))]:
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.register_rigid(X, Y, Yn, **opts)
        b.record(stream)
        torch.cuda.synchronize()
        reg_lat_ms.append(a.elapsed_time(b))

    # accuracy of the timed results: vs the planted motion, and batched vs plain
    rot_err = max(synth.rotation_angle_deg(T, p.T_gt) for (T, _, _), p in zip(last, pairs))
    trans_err = max(float(np.linalg.norm(T[:3, 3] - p.T_gt[:3, 3])) for (T, _, _), p in zip(last, pairs))
    mix_rot = max(synth.rotation_angle_deg(T, Tp) for (T, _, _), (Tp, _) in zip(last, plain_last))
    reps = [r for _, r, _ in last]

    # ---- per-kernel durations of the batched launches (CUDA events), K steps --
    ctx.set_profiling(True)
    ctx.profile(reset=True)
    timed_steps(batched_step, args.steps)
    prof = ctx.profile(reset=True)
    ctx.set_profiling(False)
    # Algorithmic bytes per launch, each array touched once, float32 (pt2pl):
    # slice = 12 B per model point + 36 B per lattice vertex (8 B key + 28 B
    # [1, y, n]); build = 24 B per observation point + 36 B per vertex.  One
    # batched EM-iteration launch slices iteration k of every item and builds
    # k+1 (all but the last of the ITERS launches build).
    algo_iter = algo_build = 0.0
    v_means = []
    for p, r in zip(pairs, reps):
        v = r.lattice_vertices_sum / max(1, r.lattice_builds)
        v_means.append(v)
        algo_iter += 12.0 * p.X.shape[0] + 36.0 * v + (24.0 * p.Y.shape[0] + 36.0 * v) * (ITERS - 1) / ITERS
        algo_build += 24.0 * p.Y.shape[0] + 36.0 * v
    algo = {"em_iter": algo_iter, "build": algo_build}
    per_launch_ms = {k: (ms / n if n else 0.0) for k, (n, ms) in prof.items()}
    dominant = max(("em_iter", "build"), key=lambda k: prof[k][1])
    peak, peak_kind = measured_peaks()
    achieved = algo[dominant] / (per_launch_ms[dominant] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": "k_em_multi (batched EM iteration)" if dominant == "em_iter"
                else "k_em_multi (first build)", "achieved": round(achieved, 1), "peak": peak,
                "peak_source": f"{peak_kind} HBM copy GB/s", "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                "traffic": recorded_traffic(dominant),
                "algorithmic_bytes_per_launch": round(algo[dominant]),
                "launch_us": round(per_launch_ms[dominant] * 1e3, 2),
                "per_kernel_us": {k: round(v * 1e3, 2) for k, v in per_launch_ms.items() if prof[k][0]},
                "lattice_vertices_mean": round(sum(v_means) / len(v_means))}

    # ---- 16-bit lattice storage: the same batched step, bfloat16 / half records
    precision = None
    if not args.no_precision:
        precision = {}
        for name, code in (("bf16", fr.FR_BF16), ("fp16", fr.FR_FP16)):
            popts = dict(opts, storage=code)
            for _ in range(max(1, args.warmup)):
                ctx.register_rigid_batch(dpairs, **popts)
            ms, res = timed_steps(lambda: ctx.register_rigid_batch(dpairs, **popts), args.steps)
            ps = slowest(sum(ms) / 1000.0)
            precision[name] = {
                "value": round(em_iters_all / ps, 1), "unit": UNIT,
                "max_rot_diff_deg_vs_f32": round(max(synth.rotation_angle_deg(T, Tf) for (T, _, _), (Tf, _, _)
                                                     in zip(res, last)), 6),
                "max_trans_diff_vs_f32": round(max(float(np.linalg.norm(T[:3, 3] - Tf[:3, 3]))
                                                   for (T, _, _), (Tf, _, _) in zip(res, last)), 7),
                "max_rot_err_deg_vs_truth": round(max(synth.rotation_angle_deg(T, p.T_gt)
                                                      for (T, _, _), p in zip(res, pairs)), 4)}

    # ---- articulated registration (Algorithm 1): 16 links, 26 DOF, 30k points
    articulated = None
    if not args.no_articulated:
        ap = synth.articulated_pair(args.seed)
        aX, aY = dev(ap.Xref), dev(ap.Y)
        abody = torch.from_numpy(ap.body.astype(np.int32)).cuda()
        articulated = {"workload": "kintree_capsules_16_links_26dof", "M": int(ap.Xref.shape[0]),
                       "N": int(ap.Y.shape[0]), "em_iters": ART_ITERS, "sigma": ART_SIGMA}
        res32 = None
        for name, code in (("f32", fr.FR_FP32), ("bf16", fr.FR_BF16)):
            aopts = dict(iters=ART_ITERS, sigma_start=ART_SIGMA, sigma_end=ART_SIGMA, w=W_OUT, storage=code)
            run = lambda: ctx.register_articulated(aX, abody, ap.tree, aY, None, **aopts)
            for _ in range(max(1, args.warmup)):
                run()
            ms, res = timed_steps(run, args.steps)
            R, q, rep = res
            surf, surf99 = synth.posed_surface_error(ap, R, q)
            entry = {"value": round(ART_ITERS * args.steps / (sum(ms) / 1000.0), 1), "unit": UNIT,
                     "ms_per_registration": round(statistics.mean(ms), 4),
                     "max_joint_err_deg_vs_truth": round(float(np.degrees(np.abs(q - ap.q_gt).max())), 4),
                     "joint_err_deg_vs_truth": [round(float(v), 2) for v in np.degrees(np.abs(q - ap.q_gt))],
                     "posed_surface_err_mm": {"mean": round(surf * 1e3, 3), "p99": round(surf99 * 1e3, 3),
                                              "before_mean": round(synth.posed_surface_error(
                                                  ap, np.eye(4), np.zeros_like(ap.q_gt))[0] * 1e3, 3)},
                     "note": "the configuration's perturbation (joints +-20 deg) lies outside the EM's "
                             "recovery range; see recovery.articulated"}
            if res32 is None:
                res32 = q
            else:
                entry["max_joint_diff_deg_vs_f32"] = round(float(np.degrees(np.abs(q - res32).max())), 5)
            articulated[name] = entry
        # the same model and workload, 16 registrations per call
        # (fr_register_articulated_batch: concurrent streams)
        bpairs = [ap] + [synth.articulated_pair(args.seed + 1 + s, tree=ap.tree) for s in range(15)]
        bitems = [(dev(p.Xref), torch.from_numpy(p.body.astype(np.int32)).cuda(), dev(p.Y), None, None, None)
                  for p in bpairs]
        bopts = dict(iters=ART_ITERS, sigma_start=ART_SIGMA, sigma_end=ART_SIGMA, w=W_OUT)
        brun = lambda: ctx.register_articulated_batch(bitems, ap.tree, **bopts)
        for _ in range(max(1, args.warmup)):
            brun()
        ms, bres = timed_steps(brun, args.steps)
        R, q, _ = ctx.register_articulated(aX, abody, ap.tree, aY, None, **bopts)
        articulated["batched"] = {
            "registrations_per_call": len(bpairs),
            "value": round(ART_ITERS * len(bpairs) * args.steps / (sum(ms) / 1000.0), 1), "unit": UNIT,
            "ms_per_call": round(statistics.mean(ms), 4),
            "failed": sum(1 for r in bres if r[3] != 0),
            "max_joint_diff_deg_vs_single": round(float(np.degrees(np.abs(bres[0][1] - q).max())), 5),
            "note": "fr_register_articulated_batch, up to 16 registrations in flight on their own streams"}

    # ---- node-graph registration (Section 5.2): ~250k points, 1,000 nodes ---
    nodegraph = None
    if not args.no_nodegraph:
        npair = synth.nodegraph_pair(args.seed)
        ng = fr.NodeGraph(ctx, dev(npair.Xref), torch.from_numpy(npair.knn).cuda(),
                          torch.from_numpy(npair.skw).cuda(), npair.node_pos, npair.edges)
        nY, nYn = dev(npair.Y), dev(npair.Yn)
        nopts = dict(lam=NG_LAMBDA, pcg_iters=NG_PCG, residual=fr.FR_PT2PL, iters=NG_ITERS,
                     sigma_start=NG_SIGMA, sigma_end=NG_SIGMA, w=W_OUT)
        nrun = lambda: ng.register(nY, nYn, **nopts)
        # bfloat16 lattice records (float32 accumulation), the same registration
        nrun16 = lambda: ng.register(nY, nYn, storage=fr.FR_BF16, **nopts)
        for _ in range(max(1, args.warmup)):
            nrun16()
        ms16, (Tn16, _) = timed_steps(nrun16, args.steps)
        for _ in range(max(1, args.warmup)):
            nrun()
        ms, (Tn, rn) = timed_steps(nrun, args.steps)
        ctx.set_profiling(True)
        ctx.profile(reset=True)
        nrun()
        nprof = ctx.profile(reset=True)
        ctx.set_profiling(False)
        Xw = ng.warp(Tn).cpu().numpy()[:, :3]
        Xw16 = ng.warp(Tn16).cpu().numpy()[:, :3]
        en0 = float(np.abs(np.sum((npair.Xref[:, :3] - npair.X_true) * npair.Xn_true, 1)).mean())
        en = float(np.abs(np.sum((Xw - npair.X_true) * npair.Xn_true, 1)).mean())
        en16 = float(np.abs(np.sum((Xw16 - npair.X_true) * npair.Xn_true, 1)).mean())
        per = lambda k: round(nprof[k][1] / max(1, nprof[k][0]), 4)
        nodegraph = {"workload": "height_field_640x480_nodegraph", "M": int(npair.Xref.shape[0]),
                     "N": int(npair.Y.shape[0]), "K": int(npair.node_pos.shape[0]),
                     "E": int(npair.edges.shape[0]), "em_iters": NG_ITERS, "pcg_iters": NG_PCG,
                     "sigma": NG_SIGMA, "lambda": NG_LAMBDA,
                     "value": round(NG_ITERS * args.steps / (sum(ms) / 1000.0), 1), "unit": UNIT,
                     "ms_per_registration": round(statistics.mean(ms), 4),
                     "e_step_assembly_ms_per_iter": per("ng_assemble"),
                     "pcg_update_ms_per_iter": per("ng_solve"), "build_ms": per("build"),
                     "normal_err_mm": {"before": round(en0 * 1e3, 4), "after": round(en * 1e3, 4)},
                     "bf16": {"value": round(NG_ITERS * args.steps / (sum(ms16) / 1000.0), 1), "unit": UNIT,
                              "ms_per_registration": round(statistics.mean(ms16), 4),
                              "normal_err_mm_after": round(en16 * 1e3, 4),
                              "rms_warp_diff_vs_f32_mm": round(float(np.sqrt(((Xw16 - Xw) ** 2).sum(1).mean())) * 1e3, 5)}}
        ng.close()

    # ---- the exact Gauss transform on the GPU (O(N M)) beside the lattice -----
    exact = None
    if not args.no_exact:
        X0, Y0, Yn0 = dpairs[0]
        p0 = pairs[0]
        sig = float(SIGMA1)

        def ev_time(fn, reps=5):
            fn()
            ts = []
            for _ in range(reps):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            return statistics.median(ts)

        ex_ms = ev_time(lambda: ctx.gauss_transform(X0, Y0, Yn0, sigma=sig, T=p0.T_gt))
        la_ms = ev_time(lambda: ctx.estep(X0, Y0, Yn0, sigma=sig, T=p0.T_gt))
        ex = ctx.gauss_transform(X0, Y0, Yn0, sigma=sig, T=p0.T_gt).double().cpu().numpy()
        la = ctx.estep(X0, Y0, Yn0, sigma=sig, T=p0.T_gt).double().cpu().numpy()
        live = (ex[:, 0] > 1e-3 * ex[:, 0].max()) & (la[:, 0] > 0)
        terr = np.linalg.norm(la[live, 1:4] / la[live, :1] - ex[live, 1:4] / ex[live, :1], axis=1) / sig
        npairs = float(p0.X.shape[0]) * float(p0.Y.shape[0])
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        peak = sms * 128 * 2.07e9 / 15.0   # FP32 lanes x max SM clock / FP32 operations per pair
        achieved = npairs / (ex_ms * 1e-3)
        exact = {"workload": f"one 320x240 pair, {p0.X.shape[0]} x {p0.Y.shape[0]} points, pt2pl, sigma {SIGMA1}",
                 "ms_per_estep": round(ex_ms, 4), "pairs_per_s": round(achieved, 1),
                 "lattice_estep_ms": round(la_ms, 4),
                 "lattice_target_err_over_sigma": {"median": round(float(np.median(terr)), 5),
                                                   "p99": round(float(np.percentile(terr, 99)), 5),
                                                   "points": int(live.sum())},
                 "roofline": {"bound": "alu", "achieved": round(achieved, 1), "peak": round(peak, 1),
                              "unit": "pairs/s", "frac": round(achieved / peak, 4),
                              "peak_source": f"{sms} SMs x 128 FP32 lanes x 2.07 GHz / 15 FP32 operations "
                                             "per pair (3 differences, squared distance 3, exponent scale 1, "
                                             "sums 7, exp2 argument 1)"}}

    # ---- feature-space E step: 6-d [position, normal] features ---------------
    features = None
    if not args.no_features:
        fp = synth.feature_frame_pair(args.seed)
        sf = np.array([FEAT_SIGMA_P] * 3 + [FEAT_SIGMA_N] * 3, np.float32)
        FX, FY, FYp, FYn = dev(fp.FX), dev(fp.FY), dev(fp.Y), dev(fp.Yn)

        def ev_ms(fn, reps=7):
            fn()
            ts = []
            for _ in range(reps):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            return statistics.median(ts)

        la_out, nv = ctx.estep_features(FX, FY, sf, FYp, FYn)
        l0 = ctx.kernel_launches
        la_out, nv = ctx.estep_features(FX, FY, sf, FYp, FYn)
        per_call = ctx.kernel_launches - l0
        la_ms = ev_ms(lambda: ctx.estep_features(FX, FY, sf, FYp, FYn))
        # per-kernel device times: event pairs around each launch
        ctx.profile(reset=True)
        ctx.set_profiling(True)
        for _ in range(20):
            ctx.estep_features(FX, FY, sf, FYp, FYn)
        ctx.set_profiling(False)
        kp = ctx.profile(reset=True)
        k_us = {name: round(1000.0 * kp[name][1] / max(1, kp[name][0]), 3) for name in ("build", "slice", "clear")}
        ex_ms = ev_ms(lambda: ctx.estep_features(FX, FY, sf, FYp, FYn, exact=True), reps=3)
        la = la_out.double().cpu().numpy()
        ex = ctx.estep_features(FX, FY, sf, FYp, FYn, exact=True)[0].double().cpu().numpy()
        live = (ex[:, 0] > 1e-3 * ex[:, 0].max()) & (la[:, 0] > 0)
        terr = np.linalg.norm(la[live, 1:4] / la[live, :1] - ex[live, 1:4] / ex[live, :1], axis=1) / FEAT_SIGMA_P
        M, N = fp.FX.shape[0], fp.FY.shape[0]
        # algorithmic bytes of the build (the dominant kernel): observation
        # features, points and normals read once, every vertex record (64 B)
        # written once
        alg = N * (24 + 16 + 16) + nv * 64
        hbm, hbm_src = measured_peaks()
        ach = alg / (k_us["build"] * 1e-6) / 1e9
        features = {"workload": f"one 320x240 pair, 6-d [position, normal] features, {M} x {N} points, "
                                f"pt2pl values, sigma_f ({FEAT_SIGMA_P} m x 3, {FEAT_SIGMA_N} x 3)",
                    "lattice_ms_per_estep": round(la_ms, 4), "estep_per_s": round(1000.0 / la_ms, 1),
                    "kernel_us": k_us, "kernels_us_sum": round(sum(k_us.values()), 3),
                    "lattice_vertices": nv, "launches_per_estep": per_call,
                    "exact_ms_per_estep": round(ex_ms, 4),
                    "lattice_over_exact_speedup": round(ex_ms / la_ms, 1),
                    "lattice_target_err_over_sigma_p": {"median": round(float(np.median(terr)), 5),
                                                        "p99": round(float(np.percentile(terr, 99)), 5),
                                                        "points": int(live.sum())},
                    "roofline": {"kernel": "k_feat_build", "bound": "hbm", "achieved": round(ach, 1),
                                 "peak": hbm, "unit": "GB/s", "frac": round(ach / hbm, 4),
                                 "peak_source": hbm_src, "algorithmic_bytes": int(alg),
                                 "timing": "CUDA events around each build launch (20 calls); "
                                           "lattice_ms_per_estep brackets the whole call (3 kernels, a "
                                           "memset, the counter read-back and the synchronisation)"}}

    # ---- recovery range: perturbations the EM brings back (GPU) --------------
    recovery = None
    if not args.no_recovery:
        f32 = lambda x: float(np.float32(x))
        sph = {"workload": "bumpy sphere 2000 x 2200 points (10% outliers), pronounced bumps (amplitude 0.5, "
                           "width 0.35), rotation exactly the stated angle, translation up to 5 cm, "
                           "point-to-point, sigma 0.2 -> 0.02 over 60 iterations, w 0.1, seeds 0-7",
               "success": "rotation error < 2 deg"}
        for ang in (10, 20, 30, 45):
            sp = [synth.sphere_bumps_pair(s, max_angle_deg=ang, **SPHERE_RECOVERY) for s in range(8)]
            res = ctx.register_rigid_batch([(dev(q.X), dev(q.Y), None) for q in sp],
                                           sigmas=[(f32(0.2), f32(0.02))] * len(sp), residual=fr.FR_PT2PT,
                                           iters=60, w=f32(W_OUT))
            errs = [synth.rotation_angle_deg(T, q.T_gt) for (T, _, _), q in zip(res, sp)]
            sph[f"{ang}_deg"] = {"success_rate": sum(e < 2.0 for e in errs) / len(errs),
                                 "median_rot_err_deg": round(float(np.median(errs)), 3)}
        # the configuration's own sphere (default bumps, sigma 0.02): rotation
        # is nearly unobservable there, whatever the start
        sp = [synth.sphere_bumps_pair(s, max_angle_deg=5.0, max_trans=0.05, exact_angle=True) for s in range(8)]
        res = ctx.register_rigid_batch([(dev(q.X), dev(q.Y), None) for q in sp],
                                       sigmas=[(f32(0.02), f32(0.02))] * len(sp), residual=fr.FR_PT2PT,
                                       iters=60, w=f32(W_OUT))
        errs = [synth.rotation_angle_deg(T, q.T_gt) for (T, _, _), q in zip(res, sp)]
        sph["default_bumps_5_deg_sigma_0.02"] = {"success_rate": sum(e < 2.0 for e in errs) / len(errs),
                                                 "median_rot_err_deg": round(float(np.median(errs)), 3)}
        art = {"workload": "kintree 16 links / 26 DOF, 30,000 points (10% outliers, 2 mm noise), "
                           "sigma 0.01 -> 0.005 over 30 iterations, w 0.1, seeds 1000-1002",
               "metric": "mean distance (mm) between the model posed at the estimate and at the truth; "
                         "recovered: below the 2 mm noise"}
        for mj, rd in ((2, 1), (5, 2), (10, 5), (20, 5)):
            errs, before = [], []
            for s in range(3):
                apr = synth.articulated_pair(1000 + s, max_joint_deg=mj, root_deg=rd)
                R, q, _ = ctx.register_articulated(dev(apr.Xref), torch.from_numpy(apr.body.astype(np.int32)).cuda(),
                                                   apr.tree, dev(apr.Y), None, iters=30, sigma_start=f32(0.01),
                                                   sigma_end=f32(0.005), w=f32(W_OUT))
                errs.append(synth.posed_surface_error(apr, R, q)[0] * 1e3)
                before.append(synth.posed_surface_error(apr, np.eye(4), np.zeros_like(apr.q_gt))[0] * 1e3)
            art[f"joints_{mj}_deg_root_{rd}_deg"] = {"before_mm": [round(v, 2) for v in before],
                                                     "after_mm": [round(v, 2) for v in errs],
                                                     "recovered": sum(v < 2.0 for v in errs)}
        recovery = {"sphere": sph, "articulated": art}

    # ---- sigma as a decision variable vs a fixed sigma (bumpy sphere) --------
    sigma_upd = None
    if not args.no_sigma:
        f32 = lambda x: float(np.float32(x))
        rows = {"fixed_0.05": dict(sigma_start=f32(0.05), sigma_end=f32(0.05)),
                "updated_from_0.1_floor_0.005": dict(sigma_start=f32(0.1), sigma_end=f32(0.005), update_sigma=1)}
        sigma_upd = {"workload": "bumpy sphere 2000 x 2200 points (10% outliers), pronounced bumps (amplitude 0.5, "
                                 "width 0.35), rotation 5 deg, translation up to 3 cm, point-to-point, w 0.1, "
                                 "stop at |dzeta| < 1e-5, at most 100 iterations, seeds 0-4"}
        for name, kw in rows.items():
            its, errs, ms, sig_last = [], [], [], []
            for seed in range(5):
                sp = synth.sphere_bumps_pair(seed, max_angle_deg=5.0, amp=0.5, width=0.35, max_trans=0.03,
                                             exact_angle=True)
                Xs, Ys = dev(sp.X), dev(sp.Y)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                Ts, rs = ctx.register_rigid(Xs, Ys, None, residual=fr.FR_PT2PT, iters=100, w=f32(0.1),
                                            stop_twist=1e-5, **kw)
                b.record(stream)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
                its.append(rs.iters_run)
                sig_last.append(rs.last_sigma)
                errs.append(synth.rotation_angle_deg(Ts, sp.T_gt))
            sigma_upd[name] = {"em_iters_to_stop_mean": round(statistics.mean(its), 1), "iters": its,
                               "ms_per_registration_mean": round(statistics.mean(ms), 4),
                               "rot_err_deg_vs_truth_mean": round(statistics.mean(errs), 4),
                               "last_sigma": [round(float(r), 4) for r in sig_last]}

    # ---- serving: Poisson stream through fr_server vs the plain path ---------
    serving = None
    if not args.no_serving:
        sp = serving_pool(args)
        serving = run_serving(ctx, args, *sp)          # default launch shapes
        serving.pop("_T")
        serving["tuning"] = tune_serving(ctx, sp[0], sp[1])
        tuned = run_serving(ctx, args, *sp, plain=False)
        serving["tuned"] = {k: tuned[k] for k in ("regs_per_s", "latency_ms_p50", "latency_ms_p99",
                                                   "saturated_regs_per_s", "failed")}
        # the batched, served, mixed-precision form: bfloat16 lattice records
        mixed = run_serving(ctx, args, *sp, plain=False, storage=fr.FR_BF16)
        serving["tuned_bf16"] = {k: mixed[k] for k in ("regs_per_s", "latency_ms_p50", "latency_ms_p99",
                                                        "saturated_regs_per_s", "failed")}
        serving["tuned_bf16"]["max_rot_diff_deg_vs_f32_server"] = round(
            max(synth_rot(a, b) for a, b in zip(mixed["_T"], tuned["_T"])), 6)

    # ---- end to end through the C ABI with host buffers ----------------------
    e2e = None
    if not args.no_e2e:
        hpairs = [(torch.from_numpy(p.X).pin_memory(), torch.from_numpy(p.Y).pin_memory(),
                   torch.from_numpy(p.Yn).pin_memory()) for p in pairs]
        hp = [(a.numpy(), b.numpy(), c.numpy()) for a, b, c in hpairs]
        ctx.register_rigid_batch(hp, host=True, **opts)
        b0 = ctx.transfer_bytes()
        barrier()
        t0 = time.perf_counter()
        for k in range(args.steps):
            ctx.register_rigid_batch(hp, host=True, **opts)
        barrier()
        te = slowest(time.perf_counter() - t0)
        b1 = ctx.transfer_bytes()
        e2e = {"value": round(em_iters_all / te, 1), "unit": UNIT,
               "h2d_bytes_per_step": (b1[0] - b0[0]) // args.steps,
               "d2h_bytes_per_step": (b1[1] - b0[1]) // args.steps,
               "timing": "host wall clock around fr_register_rigid_batch_host calls (pinned inputs)"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(pairs[0], args.seed)
    lat = sorted(reg_lat_ms)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(statistics.mean(step_ms), 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded ray-cast depth frames)",
            "config": workload_config(args.frames, pairs),
            "registrations_per_s": round(args.frames * args.steps * ws / total_s, 1),
            "plain": {"em_iters_per_s": round(em_iters_all / plain_s, 1),
                      "registrations_per_s": round(args.frames * args.steps * ws / plain_s, 1),
                      "ms_per_step": round(statistics.mean(plain_ms), 4),
                      "latency_ms_p50": round(lat[len(lat) // 2], 4),
                      "note": "fr_register_rigid one frame pair at a time, same frames, same flush"},
            "batched_over_plain": round(plain_s / total_s, 3),
            "accuracy": {"max_rot_err_deg_vs_truth": round(rot_err, 4),
                         "max_trans_err_vs_truth": round(trans_err, 6),
                         "max_rot_diff_deg_batched_vs_plain": round(mix_rot, 6)},
            "roofline": roofline,
            "tuning": tuning,
            "precision": precision,
            "articulated": articulated,
            "serving": serving,
            "nodegraph": nodegraph,
            "exact": exact,
            "sigma_update": sigma_upd,
            "features": features,
            "recovery": recovery,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "wall_s_timed_region": round(t_wall, 3),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def _timed_registrations(pair, budget_s, max_n=20, **kw):
    """Full registrations of one pair until about budget_s; (EM iters/s, n, seconds)."""
    import oracle
    n, t0 = 0, time.perf_counter()
    while True:
        oracle.register_rigid(pair.X, pair.Y, pair.Yn, **kw)
        n += 1
        el = time.perf_counter() - t0
        if el > budget_s or n >= max_n:
            return n * kw["iters"] / el, n, el


def cpu_baseline(pair, seed):
    """The oracle as it stands on this machine's host cores: the lattice
    back-end on the benchmark workload single-threaded and OpenMP-parallel
    over every core (same sources, bit-identical results), and the exact
    O(N M) back-end at the bumpy-sphere size and on a 10k-point subsample of
    the depth frames (one E step, scaled by N M to the full frame)."""
    import numpy as np
    import oracle
    from paper_1811_10136_gb300 import synth
    oracle.build()
    oracle.build(openmp=True)
    cores = os.cpu_count() or 1
    lat = dict(sigma=SIGMA0, sigma_end=SIGMA1, w=W_OUT, iters=ITERS, residual=oracle.PT2PL, backend=oracle.LATTICE)
    out = {"kind": "oracle", "unit": UNIT, "host_cores": cores}
    try:
        oracle.set_parallel(False)
        v1, n1, e1 = _timed_registrations(pair, 6.0, **lat)
        oracle.set_parallel(True, cores)
        threads = oracle.num_threads()
        vp, n_p, ep = _timed_registrations(pair, 4.0, **lat)
        out.update({"value": round(vp, 2), "cores": threads,
                    "sample": f"{n_p} full {ITERS}-iteration registrations of one 320x240 frame pair "
                              f"({ep:.1f} s, lattice back-end, {threads} OpenMP threads)",
                    "single_thread": {"value": round(v1, 2), "cores": 1,
                                      "sample": f"{n1} registrations ({e1:.1f} s)"}})
        # exact back-end, bumpy-sphere workload (2,000 x 2,200 points, 30 iterations, point-to-point)
        sph = synth.sphere_bumps_pair(seed)
        ex = dict(sigma=0.02, w=W_OUT, iters=30, residual=oracle.PT2PT, backend=oracle.EXACT)
        exact = {"workload": f"bumpy sphere {sph.X.shape[0]} x {sph.Y.shape[0]} points, 30 iterations"}
        for name, par in (("single_thread", False), ("all_cores", True)):
            oracle.set_parallel(par, cores if par else None)
            t0 = time.perf_counter()
            oracle.register_rigid(sph.X, sph.Y, None, **ex)
            el = time.perf_counter() - t0
            exact[name] = {"em_iters_per_s": round(30 / el, 2), "cores": oracle.num_threads()}
        # one exact E step on a 10k subsample of both depth frames, scaled by N M
        rng = np.random.default_rng(seed)
        xi = rng.choice(pair.X.shape[0], 10_000, replace=False)
        yi = rng.choice(pair.Y.shape[0], 10_000, replace=False)
        full = pair.X.shape[0] * pair.Y.shape[0] / 1e8
        sub = {"sample": "one exact E step (pt2pl sums) of 10,000 model x 10,000 observation points, "
                         f"scaled by N M to {pair.X.shape[0]} x {pair.Y.shape[0]}"}
        for name, par in (("single_thread", False), ("all_cores", True)):
            oracle.set_parallel(par, cores if par else None)
            t0 = time.perf_counter()
            oracle.estep(pair.X[xi], pair.Y[yi], pair.Yn[yi], SIGMA1, backend=oracle.EXACT)
            el = time.perf_counter() - t0
            sub[name] = {"s_per_estep_10k": round(el, 3), "s_per_estep_full_extrapolated": round(el * full, 2),
                         "cores": oracle.num_threads()}
        exact["depth_frame_estep"] = sub
        out["exact"] = exact
        # one feature-space lattice E step (6-d [position, normal]) on the full frame
        oracle.set_parallel(False)
        fp = synth.feature_frame_pair(seed)
        sf = np.array([FEAT_SIGMA_P] * 3 + [FEAT_SIGMA_N] * 3, np.float32)
        t0 = time.perf_counter()
        oracle.estep_features(fp.FX, fp.FY, sf, fp.Y, fp.Yn, backend=oracle.LATTICE)
        el = time.perf_counter() - t0
        out["features"] = {"sample": f"one 6-d lattice E step, {fp.FX.shape[0]} x {fp.FY.shape[0]} points",
                           "s_per_estep": round(el, 3), "cores": 1}
    finally:
        oracle.set_parallel(False)
    return out


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------

def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build(openmp=True)
    cores = os.cpu_count() or 1
    oracle.set_parallel(True, cores)
    threads = oracle.num_threads()
    pair = make_pairs(args.seed, 1)[0]
    # One step = one registration (20 EM iterations) on every host core;
    # shortened when K is large so that the whole run stays within a few
    # minutes.
    est = 0.25
    iters = ITERS if (args.steps + args.warmup) * est <= 150 else max(2, int(ITERS * 150 / ((args.steps + args.warmup) * est)))

    def step():
        oracle.register_rigid(pair.X, pair.Y, pair.Yn, sigma=SIGMA0, sigma_end=SIGMA1 if iters == ITERS else
                              SIGMA0 * (SIGMA1 / SIGMA0) ** ((iters - 1) / (ITERS - 1)), w=W_OUT, iters=iters,
                              residual=oracle.PT2PL, backend=oracle.LATTICE)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    value = iters * args.steps / el
    cfg = workload_config(1, [pair])
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded ray-cast depth frames)", "config": cfg,
        "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{args.steps} steps x {iters} EM iterations of one 320x240 pair, "
                                   f"OpenMP build over {threads} threads"},
        "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
