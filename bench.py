#!/usr/bin/env python
"""Benchmark of the BSGD hot path on one GB300 (or N replicas).

Workload (the 3D cone-beam configuration): 256^3 voxels of 1 mm, 360 views over
360 deg, 256 x 256 detector of 1.6 mm pixels, source-origin 500 mm,
source-detector 1000 mm; seeded 10-ellipsoid phantom (attenuation 0.01/mm x
density), Poisson data with I0 = 1e4; BSGD with 8 angular row blocks x 8 z-slab
column blocks, alpha = gamma = 1/8, pair sampling weighted by the residual mass
on each pair's detector band, step rho / max_J ||A^J||^2 (rho = 0.25, FP64 power
iteration). One step = one epoch = 64 block iterations (device sampling, FP with
the fused residual update, BP of the residual change, block update).

Metric: voxel-ray updates per second (FP + BP), one update being a (ray, voxel)
pair of positive length, counted exactly per pair by the library's count pass.

  python bench.py [--gpus N --steps K --warmup W]          # CUDA library
  python bench.py --impl reference [--steps K --warmup W]  # FP64 CPU oracle
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

GEOM = dict(kind="cone3d", nx=256, ny=256, nz=256, dx=1.0, dy=1.0, dz=1.0, n_views=360,
            nu=256, nv=256, du=1.6, dv=1.6, dso=500.0, dsd=1000.0)
M, N = 8, 8
ITERS_PER_EPOCH = 64
KAPPA = 0.01          # attenuation per mm of unit density
I0 = 1e4
RHO = 0.25
WORKLOAD = ("cone3d 256^3 (1 mm), 360 views / 360 deg, 256x256 det (1.6 mm), DSO 500 / DSD 1000, "
            "10 ellipsoids, Poisson I0=1e4; BSGD 8x8 blocks, alpha=gamma=1/8, residual-weighted "
            "pairs; step = 1 epoch = 64 block iterations")
METRIC = "GVox-ray updates/s (FP+BP)"
UNIT = "GVox-ray/s"
# FP32-pipe instructions every Siddon update needs at the least: two minima for
# the next crossing, the segment difference, the accumulate / weight product and
# the recomputed crossing.
ALU_OPS_PER_UPDATE = 5
# DRAM bytes (read + write) per launch of the fused kernel, mean over the 64
# launches of one epoch of this workload, from one ncu capture of the current
# kernel (its DRAM-traffic capture is summarised under profiles/); null for the
# split kernels, which were not captured.
TRAFFIC_PER_LAUNCH = {"fpbp": 46_481_784}
# What does bind the fused kernel, from the same kernel's ncu --set full capture
# (the full capture summarised under profiles/, the heavier of two pairs):
# L2 and L1/TEX throughput in % of their peaks, issue-active cycles in %, and
# L1 -> L2 sector operations per voxel-ray update (FP + BP) and per BP update
# (the reductions).
ON_CHIP_NCU = {"fpbp": {"l2_pct": 64.6, "l1tex_pct": 68.3, "issue_active_pct": 46.8,
                        "l2_sectors_per_update": 0.30, "red_sectors_per_bp_update": 0.51,
                        "thread_instructions_per_update": 23.7}}


# Serving workload: Poisson arrivals (20 / s), request sizes n^3 with (256 / n) mm
# voxels, views over 360 deg, n x n detector of 1.6 * 256 / n mm, FP32 or BF16
# storage, 8 x 8 blocks, uniform pairs, epochs per request. The default run
# serves a bounded stream (16 requests, n <= 256, 2 epochs); --serving full is
# the whole stream (200 requests, n up to 384, 10 epochs, 160 GB budget).
SERVE_FULL = dict(n_req=200, sizes=(64, 128, 256, 384), views=(90, 180, 360, 720), epochs=10)
SERVE_SMALL = dict(n_req=16, sizes=(64, 128, 256), views=(90, 180, 360), epochs=2)


# Paper-scale 3D workload (Sec. 5, Table 1): source 1536 mm from the rotation
# centre, detector 1000 mm behind it (DSD 2536), a 400 mm square detector, a
# 256 mm cube, 360 views at 1 deg; M = 5 view groups (a seeded random partition
# into equal groups, as in Sec. 5), N = 8 column blocks, alpha = 1/5,
# gamma = 2/8 (two column blocks per iteration). Noise-free projections, as in
# the paper's FP / BP timing runs.
PAPER_CASES = {"case1": (256, 400), "case2": (512, 1000), "case3": (1024, 2000)}
# Sec. 6's BSGD-IM set-up: a 256^3 grid of 1 mm voxels, 360 views, a 512^2
# detector of 1 mm pixels, source 1000 mm and detector 536 mm from the centre;
# M = 5, N = 8, alpha = 0.2, gamma = 0.5 (four column blocks per iteration),
# one of four detector quadrants per view and pair drawn by Algorithm 2. The
# paper's projections carry white noise (28.1 dB); the timing does not depend
# on the data, so they are noise-free here.
IM_GEOM = dict(kind="cone3d", nx=256, ny=256, nz=256, dx=1.0, dy=1.0, dz=1.0, n_views=360,
               nu=512, nv=512, du=1.0, dv=1.0, dso=1000.0, dsd=1536.0)


def paper_geom(n, nd):
    h, p = 256.0 / n, 400.0 / nd
    return dict(kind="cone3d", nx=n, ny=n, nz=n, dx=h, dy=h, dz=h, n_views=360, nu=nd, nv=nd,
                du=p, dv=p, dso=1536.0, dsd=2536.0)


def paper_partition(seed=5):
    import numpy as np
    vb = np.repeat(np.arange(5, dtype=np.int32), 72)
    np.random.default_rng(seed).shuffle(vb)
    return vb


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving", default="small", choices=["off", "small", "full"])
    ap.add_argument("--split", action="store_true",
                    help="run FP and BP as two kernels (to time them apart)")
    ap.add_argument("--paper-scale", default="case1,case2,case3,im",
                    help="paper-scale cases to time (comma list of case1, case2, case3, im; 'off')")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the BF16-storage, TV-prox and autograd legs")
    ap.add_argument("--legs", default="all",
                    help="extra legs to run (comma list of " + ",".join(LEGS) + "; 'all')")
    return ap.parse_args()


LEGS = ("update", "power", "geometry", "bf16", "automu", "tv", "autograd", "precision", "full_solve",
        "shard")


def bench_config(world):
    """The workload both arms run (the same dict on both, so that their lines
    compare)."""
    return {"workload": WORKLOAD, "global_batch": world, "seq_len": None,
            "parallelism": "replicas" if world > 1 else "single"}


def leg_wanted(args, name):
    return args.legs == "all" or name in args.legs.split(",")


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def reduce_over_ranks(torch, dist, seconds, units, device):
    """Whole-job figures of N replicas: the slowest rank's time and the units
    all ranks processed (one rank: the values themselves)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds), float(units)
    t = torch.tensor([float(seconds)], device=device, dtype=torch.float64)
    u = torch.tensor([float(units)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.lines = index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
            # the timed region opens once the sampler is running (its first
            # line), so every sample of the region is taken under load
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.lines.clear()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, flag in zip(names, parts[4:8]):
                if flag.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# inputs

def make_inputs(B, gg, torch, dev, seed_offset=0):
    """Phantom -> line integrals with the library's own FP -> Poisson data."""
    import numpy as np
    from paper_1903_11874_gb300 import synth
    vol = synth.ellipsoid_phantom(256, 256, 256, 10, seed=0 + seed_offset) * KAPPA
    xt = torch.from_numpy(vol.reshape(-1)).to(dev)
    p = torch.zeros(gg.n_rows, device=dev)
    B.bsgd_forward_project(gg, xt, p)
    y = synth.poisson_log_data(p.cpu().numpy(), I0, seed=2 + seed_offset)
    return np.ascontiguousarray(y), xt


def algorithmic_bytes(gg, n_pairs_avg_rays, storage_bytes=4):
    """Compulsory DRAM bytes of one pair in the FP, BP and fused FP+BP kernels,
    per the kernels' data flow: FP reads x_J and, per traced ray, y, r and the
    z^j of the blocks whose band holds the ray (compact band storage; on
    average `nb` of them, from the geometry's band areas), and writes z^J and
    r; BP reads r and r~^J, writes r~^J and read-modify-writes g_J; the fused
    kernel does both without re-reading r."""
    vox_j = gg.n_cols // N
    rays = n_pairs_avg_rays
    nb = max(1.0, gg.compact_rows / gg.n_rows)
    fp = vox_j * storage_bytes + rays * storage_bytes * (1 + nb + 1 + 2)
    bp = rays * storage_bytes * 3 + vox_j * 8
    fpbp = vox_j * (storage_bytes + 8) + rays * storage_bytes * (nb + 6)
    return {"fp": fp, "bp": bp, "fpbp": fpbp}


def run_cuda(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1903_11874_gb300 import binding as B

    rank, local, world = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = "cuda:%d" % local
    B.load()
    gg = B.Geometry(M=M, N=N, **GEOM)
    y_np, _ = make_inputs(B, gg, torch, dev, seed_offset=rank)
    y = torch.from_numpy(y_np).to(dev)
    prm = B.SolveParams(alpha=1 / M, gamma=1 / N, step_rule=B.STEP_STRIP, rho=RHO,
                        power_iters=30, pair_sampling=B.PAIRS_RESIDUAL, seed=1 + rank)
    st = B.State(gg, prm, y)
    st.set_split(args.split)
    mu = st.query()["mu"]
    x = torch.zeros(gg.n_cols, device=dev)
    for _ in range(args.warmup):
        st.block_step(x, ITERS_PER_EPOCH)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    q0 = st.query()
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    # timed region 1, the headline: K epochs as a user runs them (no per-stage
    # events between the launches)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        st.block_step(x, ITERS_PER_EPOCH)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    q1 = st.query()
    updates = q1["updates"] - q0["updates"]
    # timed region 2: K more epochs with a CUDA event pair around every launch
    # on the launching stream (per-kernel durations for the roofline and the
    # stage times; the events add ~2 % to an epoch)
    st.profile(True)
    ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    for _ in range(args.steps):
        st.block_step(x, ITERS_PER_EPOCH)
    ev3.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms_profiled = ev2.elapsed_time(ev3)
    prof = st.read_profile()
    q2 = st.query()
    updates_prof = q2["updates"] - q1["updates"]
    ms, updates_all = reduce_over_ranks(torch, dist, ms, updates, dev)
    value = updates_all / (ms * 1e-3) / 1e9

    # ---- roofline of the dominant kernel (FP or BP), timed live above
    peaks = measured_peaks()
    iters = args.steps * ITERS_PER_EPOCH
    dom = max(("fp", "bp", "fpbp"), key=lambda k: prof[k]["ms"])
    # the fused kernel does every update of an iteration; FP and BP half each
    upd_per_launch = updates_prof / iters / (1.0 if dom == "fpbp" else 2.0)
    launch_ms = prof[dom]["ms"] / max(prof[dom]["launches"], 1)
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = 152 * 128 * sm_max * 1e6 / 1e12         # FP32-pipe instr/s, in T/s
    achieved = ALU_OPS_PER_UPDATE * upd_per_launch / (launch_ms * 1e-3) / 1e12
    avg_rays = np.mean([gg.pair_rays(i, j) for i in range(M) for j in range(N)])
    # one launch covers the iteration's pairs: (alpha M) x (gamma N) = 1 x 1
    dom_bytes = algorithmic_bytes(gg, avg_rays)[dom]
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_ach = dom_bytes / (launch_ms * 1e-3) / 1e9
    roofline = {
        "bound": "alu", "kernel": "%s_solve_kernel" % dom,
        "achieved": round(achieved, 3), "peak": round(alu_peak, 2),
        "unit": "T FP32-pipe instr/s (%d per update)" % ALU_OPS_PER_UPDATE,
        "frac": round(achieved / alu_peak, 4), "traffic": TRAFFIC_PER_LAUNCH.get(dom),
        "peak_source": "152 SMs x 128 FP32 lanes x %.0f MHz (max SM clock)" % sm_max,
        "launch_ms": round(launch_ms, 4), "updates_per_launch": int(upd_per_launch),
        "hbm_algorithmic_gbs": round(hbm_ach, 1), "hbm_peak_gbs": hbm_peak,
        "hbm_frac": round(hbm_ach / hbm_peak, 4),
        "on_chip_ncu": ON_CHIP_NCU.get(dom),
    }
    stages = {k: {"launches": v["launches"], "ms": round(v["ms"], 3)} for k, v in prof.items()
              if v["launches"]}
    launches = sum(v["launches"] for v in prof.values())

    # ---- end to end through the public one-call API with host buffers
    e2e = None
    if not args.no_e2e:
        yh = torch.from_numpy(y_np).pin_memory()
        xh = torch.zeros(gg.n_cols, dtype=torch.float32).pin_memory()
        pe = B.SolveParams(alpha=1 / M, gamma=1 / N, epochs=1, step_rule=B.STEP_FIXED, mu=mu,
                           pair_sampling=B.PAIRS_RESIDUAL, seed=1 + rank, zero_start=True)
        B.bsgd_solve(gg, pe, yh, xh)       # warm-up
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        upd_e2e = 0
        for _ in range(args.steps):
            rep = B.bsgd_solve(gg, pe, yh, xh)
            upd_e2e += rep["updates"]
        t_e2e = time.perf_counter() - t0
        t_e2e, upd_e2e = reduce_over_ranks(torch, dist, t_e2e, upd_e2e, dev)
        e2e = {"value": round(upd_e2e / t_e2e / 1e9, 3), "unit": UNIT,
               "h2d_bytes_per_step": int(gg.n_rows * 4), "d2h_bytes_per_step": int(gg.n_cols * 4),
               "api": "bsgd_solve (1 epoch per call from x0 = 0 (zero_start), pinned host y and x, fixed mu)"}

    full_solve = None
    if not args.no_e2e and rank == 0 and world == 1 and leg_wanted(args, "full_solve"):
        full_solve = full_solve_leg(B, torch, y_np)

    extra = None
    if not args.no_extra and rank == 0 and world == 1:
        extra = extra_legs(B, torch, dev, gg, y, mu, prof, iters, updates, peaks,
                           lambda name: leg_wanted(args, name))

    if extra is not None and leg_wanted(args, "precision"):
        extra["P_precision_config"] = precision_leg(B, torch, dev)

    paper = None
    if args.paper_scale != "off" and rank == 0 and world == 1:
        paper = paper_scale_leg(B, torch, dev, [c for c in args.paper_scale.split(",") if c])

    serving = None
    if args.serving != "off":
        serving = serving_leg(B, torch, dev, SERVE_FULL if args.serving == "full" else SERVE_SMALL,
                              seed=3 + rank)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(y_np, mu, n_iters=2)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded ellipsoid phantom, Poisson noise)",
            "config": bench_config(world),
            "method": {"l2": "inputs larger than L2 (state ~0.8 GB resident; one iteration "
                             "touches ~100 MB across launches of different slabs)",
                       "timing": "value over K epochs without per-stage events; roofline and "
                                 "stages_ms from K more epochs with a CUDA event pair around "
                                 "every launch (ms_per_step_profiled)"},
            "run": {"mu": mu, "residual_norm_end": q1["residual_norm"],
                    "compact_rows_frac": round(gg.compact_rows / (N * gg.n_rows), 4),
                    "state_gb": round(B.bsgd_request_bytes(GEOM, M, N, prm) / 1e9, 3)},
            "gpu_launches": int(launches), "stages_ms": stages,
            "ms_per_step_profiled": round(ms_profiled / args.steps, 3),
            "kernels": "split FP / BP" if args.split else "fused FP+residual+BP",
            "roofline": roofline, "clocks": clk, "e2e": e2e, "e2e_full_solve": full_solve,
            "cpu_baseline": cpu,
            "serving": serving, "paper_scale": paper, "rows": extra,
        }
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def full_solve_leg(B, torch, y_np, n_solves=5, epochs=20):
    """The whole configuration-2 reconstruction as one user call: bsgd_solve
    with the STRIP step rule (its FP64 power iteration inside the call), 20
    epochs of residual-weighted pairs, pinned host y and x. `cold`: the first
    call on a new geometry (geometry tables, update-count pass and power
    iteration included); then n_solves calls on that geometry (the step's
    Lipschitz estimate and the update counts are kept with it), p50 / p99 of
    their latency, and the same request served by a bsgd_server one at a time."""
    import numpy as np
    yh = torch.from_numpy(y_np).pin_memory()
    xh = torch.zeros(int(np.prod([GEOM["nx"], GEOM["ny"], GEOM["nz"]])), dtype=torch.float32).pin_memory()
    prm = B.SolveParams(alpha=1 / M, gamma=1 / N, epochs=epochs, step_rule=B.STEP_STRIP, rho=RHO,
                        power_iters=30, pair_sampling=B.PAIRS_RESIDUAL, seed=1, zero_start=True)
    t0 = time.perf_counter()
    gg = B.Geometry(M=M, N=N, **GEOM)
    rep = B.bsgd_solve(gg, prm, yh, xh)
    cold = time.perf_counter() - t0
    lat, upd = [], 0
    for _ in range(n_solves):
        t0 = time.perf_counter()
        rep = B.bsgd_solve(gg, prm, yh, xh)
        lat.append(time.perf_counter() - t0)
        upd += rep["updates"]
    srv = B.Server(budget_bytes=16 << 30, max_slots=4)
    slat = []
    try:
        yn = np.ascontiguousarray(y_np)
        srv.wait(srv.submit(GEOM, M, N, prm, yn), timeout_ms=600000)     # warm-up
        for _ in range(n_solves):
            t0 = time.perf_counter()
            srv.wait(srv.submit(GEOM, M, N, prm, yn), timeout_ms=600000)
            slat.append(time.perf_counter() - t0)
    finally:
        srv.close()
    q = lambda v, f: sorted(v)[min(len(v) - 1, int(math.floor(f * (len(v) - 1) + 0.5)))]
    return {"epochs": epochs, "step_rule": "STRIP (rho %.2f, 30 power iterations)" % RHO,
            "cold_first_call_ms": round(cold * 1e3, 1),
            "p50_ms": round(q(lat, 0.5) * 1e3, 1), "p99_ms": round(q(lat, 0.99) * 1e3, 1),
            "value": round(upd / sum(lat) / 1e9, 3), "unit": UNIT,
            "served_alone_p50_ms": round(q(slat, 0.5) * 1e3, 1),
            "served_alone_p99_ms": round(q(slat, 0.99) * 1e3, 1),
            "calls": n_solves, "residual_norm_end": rep["residual_norm"], "mu": rep["mu"]}


# ---------------------------------------------------------------------------
# Serving: served mixed stream vs the plain single-request FP32 path

def serve_geometry(n, views):
    h = 256.0 / n
    return dict(kind="cone3d", nx=n, ny=n, nz=n, dx=h, dy=h, dz=h, n_views=views, nu=n, nv=n,
                du=1.6 * h, dv=1.6 * h, dso=500.0, dsd=1000.0)


# Autograd workload: a batch of 16 volumes of 128^3 (1 mm), 180 views over
# 360 deg, 192^2 detector of 1.6 mm, DSO 500 / DSD 1000.
AUTOGRAD_GEOM = dict(kind="cone3d", nx=128, ny=128, nz=128, dx=1.0, dy=1.0, dz=1.0, n_views=180,
                     nu=192, nv=192, du=1.6, dv=1.6, dso=500.0, dsd=1000.0)
AUTOGRAD_BATCH = 16


def epoch_rate(B, torch, dev, gg, y, prm, warm=2, epochs=3, profile=False):
    """(GVox-ray/s, profile or None, ms per epoch) of whole epochs of a fresh
    state, timed without per-stage events; with profile, the same number of
    further epochs with an event pair around every launch give the stage
    times."""
    st = B.State(gg, prm, y)
    x = torch.zeros(gg.n_cols, device=dev,
                    dtype={B.F32: torch.float32, B.BF16: torch.bfloat16, B.F16: torch.float16}[prm.storage])
    for _ in range(warm):
        st.block_step(x, ITERS_PER_EPOCH)
    torch.cuda.synchronize()
    q0 = st.query()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(epochs):
        st.block_step(x, ITERS_PER_EPOCH)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    upd = st.query()["updates"] - q0["updates"]
    prof = None
    if profile:
        st.profile(True)
        for _ in range(epochs):
            st.block_step(x, ITERS_PER_EPOCH)
        prof = st.read_profile()
    st.close()
    return upd / (ms * 1e-3) / 1e9, prof, ms / epochs


def extra_legs(B, torch, dev, gg, y, mu, prof, iters, updates, peaks, want=lambda name: True):
    """Measurements of the other rows of the hot path: the block update and the
    TV prox against the HBM roofline, BF16 storage, the autograd projector
    (`want(name)` selects the legs)."""
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    out = {}
    if want("update"):
        out.update(update_leg(B, torch, dev, gg, y, mu, prof, hbm))
    if want("power"):
        out.update(power_leg(B, torch, gg))
    if want("geometry"):
        t0 = time.perf_counter()
        g2 = B.Geometry(M=M, N=N, **GEOM)
        out["a1_geometry_ms"] = round((time.perf_counter() - t0) * 1e3, 2)
        g2.close()
    if want("bf16"):
        prm16 = B.SolveParams(alpha=1 / M, gamma=1 / N, step_rule=B.STEP_FIXED, mu=mu,
                              pair_sampling=B.PAIRS_RESIDUAL, storage=B.BF16, seed=1)
        v16, _, ms16 = epoch_rate(B, torch, dev, gg, y, prm16)
        out["P_bf16_storage"] = {"value": round(v16, 3), "unit": UNIT, "ms_per_epoch": round(ms16, 3)}
    if want("automu"):
        out.update(automu_leg(B, torch, dev, gg, y, mu))
    if want("tv"):
        out.update(tv_leg(B, torch, dev, gg, y, mu, hbm))
    if want("autograd"):
        out.update(autograd_leg(B, torch, dev))
    if want("shard"):
        out["NEXT4_shard_one_process"] = shard_leg(B, torch, dev)
    return out


def shard_leg(B, torch, dev, warm=2, iters=20):
    """The owner-computes path (bsgd_shard_begin / _end) run by one process
    owning every column block, against the same iterations through
    bsgd_block_step, on Sec. 5's case-1 set-up (two column blocks per
    iteration: the setting the paper shards over two GPUs). With one process
    the exchange is the identity; on N GPUs it is one all-reduce of the buffer
    per iteration. Per-iteration times, CUDA events."""
    from paper_1903_11874_gb300 import shard, synth
    n, nd = PAPER_CASES["case1"]
    gg = B.Geometry(M=5, N=8, view_block=paper_partition(), **paper_geom(n, nd))
    vol = torch.from_numpy(synth.ellipsoid_phantom(n, n, n, 10, seed=0).reshape(-1) * KAPPA).to(dev)
    y = torch.zeros(gg.n_rows, device=dev)
    B.bsgd_forward_project(gg, vol, y)
    del vol
    prm = B.SolveParams(alpha=1 / 5, gamma=2 / 8, step_rule=B.STEP_FIXED, mu=1e-6,
                        pair_sampling=B.PAIRS_UNIFORM, seed=1)
    out = {"set_up": "Table 1 case 1: 256^3, 360 views, 400^2 detector, M=5, N=8, "
                     "alpha=1/5, gamma=2/8 (two column blocks per iteration)"}
    for name in ("block_step", "sharded"):
        st = B.State(gg, prm, y)
        x = torch.zeros(gg.n_cols, device=dev)
        if name == "sharded":
            solver = shard.ShardedSolver(st, list(range(gg.N)), lambda b: b,
                                         torch.empty(0, device=dev))
            step = solver.block_step
            out["exchange_floats"] = int(solver.buf.numel())
        else:
            step = st.block_step
        step(x, warm)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step(x, iters)
        e1.record()
        torch.cuda.synchronize()
        out[name + "_ms_per_iteration"] = round(e0.elapsed_time(e1) / iters, 3)
        st.close()
    return out


def update_leg(B, torch, dev, gg, y, mu, prof, hbm):
    out = {}
    # a7 and a2/a3 on their own: one iteration per call, so every call runs a
    # standalone draw and a plain block update (in longer calls the update
    # launch also carries the next draw)
    prm1 = B.SolveParams(alpha=1 / M, gamma=1 / N, step_rule=B.STEP_FIXED, mu=mu,
                         pair_sampling=B.PAIRS_RESIDUAL, seed=1)
    st1 = B.State(gg, prm1, y)
    x1 = torch.zeros(gg.n_cols, device=dev)
    for _ in range(8):
        st1.block_step(x1, 1)
    torch.cuda.synchronize()
    st1.profile(True)
    for _ in range(64):
        st1.block_step(x1, 1)
    p1 = st1.read_profile()
    st1.close()
    # a7: block update, 20 B per voxel of the slab (read x, g, gT; write x, xT)
    vox_j = gg.n_cols // N
    ms_u = p1["update"]["ms"] / max(p1["update"]["launches"], 1)
    gbs = 20.0 * vox_j / (ms_u * 1e-3) / 1e9
    out["a7_update"] = {"ms_per_launch": round(ms_u, 4), "bytes_per_launch": 20 * vox_j,
                        "achieved_gbs": round(gbs, 1), "peak_gbs": hbm, "frac": round(gbs / hbm, 4),
                        "bound": "hbm"}
    ms_s = p1["sample"]["ms"] / max(p1["sample"]["launches"], 1)
    ms_us = prof["update"]["ms"] / max(prof["update"]["launches"], 1)
    out["a2_a3_sample"] = {"ms_per_launch": round(ms_s, 4),
                           "bound": "latency (one CTA standalone; inside the update launch the "
                                    "pair weights are split over 8 CTAs)",
                           "update_with_next_draw_ms": round(ms_us, 4)}
    return out


def power_leg(B, torch, gg):
    # a8: the step size's FP64 power iteration, 30 steps (FP + BP) of one strip
    out = {}
    j = 0
    per_fp = B.bsgd_count_updates(gg, col_blocks=[j])
    B.bsgd_power_iteration(gg, j, 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B.bsgd_power_iteration(gg, j, 30)
    dt = time.perf_counter() - t0
    out["a8_power_iteration"] = {"ms": round(dt * 1e3, 2), "iterations": 30,
                                 "value": round(2 * 30 * per_fp / dt / 1e9, 3), "unit": UNIT,
                                 "note": "one column strip, all views; FP64 vector state"}
    return out


def automu_leg(B, torch, dev, gg, y, mu):
    out = {}
    # NEXT-1: Algorithm 3 on (a test at the end of every epoch: FP64 EUD
    # accumulation in the update, a reduction and the decision on the device)
    # against the same epochs with a fixed step
    prm32 = B.SolveParams(alpha=1 / M, gamma=1 / N, step_rule=B.STEP_FIXED, mu=mu,
                          pair_sampling=B.PAIRS_RESIDUAL, seed=1)
    v32, _, ms32 = epoch_rate(B, torch, dev, gg, y, prm32)
    prmam = B.SolveParams(alpha=1 / M, gamma=1 / N, step_rule=B.STEP_FIXED, mu=mu,
                          pair_sampling=B.PAIRS_RESIDUAL, auto_mu=True, auto_window=1, seed=1)
    vam, _, msam = epoch_rate(B, torch, dev, gg, y, prmam)
    out["NEXT1_auto_mu"] = {"value": round(vam, 3), "unit": UNIT, "ms_per_epoch": round(msam, 3),
                            "fixed_step_value": round(v32, 3),
                            "overhead_pct": round(100.0 * (v32 / vam - 1.0), 2), "window_epochs": 1}
    return out


def tv_leg(B, torch, dev, gg, y, mu, hbm):
    out = {}
    # a9: TV prox (FGP, 20 iterations) once per epoch; algorithmic bytes: 52 B
    # per voxel and FGP iteration (one pass: b, r_xyz, p_xyz read; p_xyz,
    # r_xyz written; u is formed on chip) + 80 B per voxel for the set-up and
    # the final primal (the float4 layout of the dual fields moves 68 B)
    prmtv = B.SolveParams(alpha=1 / M, gamma=1 / N, step_rule=B.STEP_FIXED, mu=mu,
                          pair_sampling=B.PAIRS_RESIDUAL, tv_lambda=1e-3, tv_iters=20, seed=1)
    _, ptv, _ = epoch_rate(B, torch, dev, gg, y, prmtv, warm=1, epochs=2, profile=True)
    ms_tv = ptv["tv"]["ms"] / max(1, ptv["tv"]["launches"] // 43)
    btv = gg.n_cols * (52 * 20 + 80)
    out["a9_tv_prox"] = {"ms_per_prox": round(ms_tv, 3), "bytes_per_prox": btv,
                         "achieved_gbs": round(btv / (ms_tv * 1e-3) / 1e9, 1), "peak_gbs": hbm,
                         "frac": round(btv / (ms_tv * 1e-3) / 1e9 / hbm, 4), "bound": "hbm",
                         "fgp_iterations": 20}
    return out


def autograd_leg(B, torch, dev):
    out = {}
    # D: Projector forward + backward on a batch
    from paper_1903_11874_gb300.autograd import Projector
    ga = B.Geometry(M=1, N=1, **AUTOGRAD_GEOM)
    per_vol = B.bsgd_count_updates(ga)
    xb = torch.rand((AUTOGRAD_BATCH,) + tuple(ga.vol_shape), device=dev, requires_grad=True)
    for _ in range(2):
        Projector.apply(xb, ga).sum().backward()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record()
    for _ in range(reps):
        Projector.apply(xb, ga).sum().backward()
    e1.record()
    torch.cuda.synchronize()
    ms_ag = e0.elapsed_time(e1) / reps
    out["D_autograd"] = {"batch": AUTOGRAD_BATCH, "volume": "128^3", "views": 180, "detector": "192^2",
                         "ms_per_forward_backward": round(ms_ag, 3),
                         "value": round(2 * per_vol * AUTOGRAD_BATCH / (ms_ag * 1e-3) / 1e9, 3),
                         "unit": UNIT}
    ga.close()
    return out


# Precision configuration: 512^3 (0.5 mm), 720 views over 360 deg, 512^2
# detector of 0.8 mm, DSO 500 / DSD 1000, M = N = 16 (alpha = gamma = 1/16, an
# epoch of 256 iterations), TV lambda = 1e-3 with 20 FGP iterations once per
# epoch, noise-free projections; BF16 storage of y, x, z^j, r, r~^j with FP32
# arithmetic, against the same run with FP32 storage.
PRECISION_GEOM = dict(kind="cone3d", nx=512, ny=512, nz=512, dx=0.5, dy=0.5, dz=0.5, n_views=720,
                      nu=512, nv=512, du=0.8, dv=0.8, dso=500.0, dsd=1000.0)


def precision_leg(B, torch, dev, epochs=2):
    from paper_1903_11874_gb300 import synth
    gg = B.Geometry(M=16, N=16, **PRECISION_GEOM)
    vol = torch.from_numpy(synth.ellipsoid_phantom(256, 256, 256, 10, seed=0) * KAPPA).to(dev)
    vol = vol.repeat_interleave(2, 0).repeat_interleave(2, 1).repeat_interleave(2, 2)
    y = torch.zeros(gg.n_rows, device=dev)
    B.bsgd_forward_project(gg, vol.reshape(-1).contiguous(), y)
    lam = None
    out = {"volume": "512^3 (0.5 mm)", "views": 720, "detector": "512^2 (0.8 mm)",
           "blocks": "M=N=16, alpha=gamma=1/16", "tv": "lambda 1e-3, 20 FGP iterations per epoch"}
    xs = {}
    for name, storage, tdt in (("fp32", B.F32, torch.float32), ("bf16", B.BF16, torch.bfloat16)):
        prm = B.SolveParams(alpha=1 / 16, gamma=1 / 16, step_rule=B.STEP_STRIP if lam is None else B.STEP_FIXED,
                            rho=RHO, power_iters=5, mu=lam or 0.0, pair_sampling=B.PAIRS_UNIFORM,
                            tv_lambda=1e-3, tv_iters=20, storage=storage, seed=1)
        st = B.State(gg, prm, y)
        lam = st.query()["mu"]            # the same step for both runs
        x = torch.zeros(gg.n_cols, device=dev, dtype=tdt)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(epochs):
            st.block_step(x, 256)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / epochs
        q = st.query()
        xs[name] = x.float().clone()
        # one more epoch with per-stage events for the TV prox's share
        st.profile(True)
        st.block_step(x, 256)
        prof = st.read_profile()
        out[name] = {"ms_per_epoch": round(ms, 2), "value": round(q["updates"] / epochs / (ms * 1e-3) / 1e9, 3),
                     "unit": UNIT, "tv_ms_per_epoch": round(prof["tv"]["ms"], 2),
                     "residual_norm": q["residual_norm"]}
        st.close()
    d = float(torch.linalg.vector_norm(xs["bf16"] - xs["fp32"]) / torch.linalg.vector_norm(xs["fp32"]))
    out["bf16_vs_fp32_rel_l2"] = round(d, 6)
    out["mu"] = lam
    out["vs_oracle_reduced"] = precision_vs_oracle(B, torch, dev)
    return out


def precision_vs_oracle(B, torch, dev):
    """The same BSGD-TV set-up at 1/8 resolution (synth.PRECISION_REDUCED: 64^3,
    90 views, 64^2 detector, 16 x 16 blocks, 10 epochs) against the FP64
    oracle's stored trajectory (tests/golden/precision_reduced.json, written by
    tests/golden/make_precision_reduced.py; same draws and step): relative L2
    error after every epoch over the stored sample voxels, for FP32 storage,
    BF16 with the compensated image and BF16 with the plain image."""
    import numpy as np
    from paper_1903_11874_gb300 import synth
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden",
                        "precision_reduced.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        gold = json.load(f)
    w = synth.PRECISION_REDUCED
    gg = B.Geometry(M=w["M"], N=w["N"], **w["geometry"])
    vol = torch.from_numpy(synth.precision_reduced_phantom().reshape(-1)).to(dev)
    y = torch.zeros(gg.n_rows, device=dev)
    B.bsgd_forward_project(gg, vol, y)
    idx = torch.tensor(gold["sample_indices"], device=dev)
    ref = [torch.tensor(v, device=dev, dtype=torch.float64) for v in gold["x_samples"]]
    out = {"workload": "64^3 (4 mm), 90 views, 64^2 detector (6.4 mm), M=N=16, BSGD-TV lambda 1e-3, "
                       "10 epochs, noise-free; y by this library's FP (the oracle's own y differs by "
                       "FP32 rounding)",
           "samples": len(gold["sample_indices"]), "mu": gold["mu"]}
    for name, storage, tdt, plain in (("fp32", B.F32, torch.float32, False),
                                      ("bf16", B.BF16, torch.bfloat16, False),
                                      ("bf16_plain", B.BF16, torch.bfloat16, True)):
        prm = B.SolveParams(alpha=1 / w["M"], gamma=1 / w["N"], step_rule=B.STEP_FIXED,
                            mu=gold["mu"], seed=w["seed"], tv_lambda=w["tv_lambda"],
                            tv_iters=w["tv_iters"], storage=storage, image_plain=plain)
        st = B.State(gg, prm, y)
        x = torch.zeros(gg.n_cols, device=dev, dtype=tdt)
        errs = []
        for e in range(w["epochs"]):
            st.block_step(x, w["M"] * w["N"])
            got = x.double()[idx]
            errs.append(float(torch.linalg.vector_norm(got - ref[e]) / torch.linalg.vector_norm(ref[e])))
        st.close()
        out[name + "_rel_l2_per_epoch"] = [float("%.3e" % v) for v in errs]
    out["image_bytes_per_voxel"] = {"fp32": 4, "bf16": 4, "bf16_plain": 2}
    return out


def paper_scale_leg(B, torch, dev, cases, warm=2, iters=10):
    """FP and BP time per BSGD iteration on the paper's Table 1 cases (the
    analogue of Sec. 5's per-iteration FP / BP timing), one GPU."""
    import numpy as np
    from paper_1903_11874_gb300 import synth
    out = {}
    for name in cases:
        im = name == "im"
        n, nd = (256, 512) if im else PAPER_CASES[name]
        geo = dict(IM_GEOM) if im else paper_geom(n, nd)
        gg = B.Geometry(M=5, N=8, view_block=paper_partition(), **geo)
        base = synth.ellipsoid_phantom(256, 256, 256, 10, seed=0) * KAPPA
        vol = torch.from_numpy(base).to(dev)
        if n != 256:   # the same phantom at the finer grid (nearest neighbour)
            f = n // 256
            vol = vol.repeat_interleave(f, 0).repeat_interleave(f, 1).repeat_interleave(f, 2)
        y = torch.zeros(gg.n_rows, device=dev)
        B.bsgd_forward_project(gg, vol.reshape(-1).contiguous(), y)
        del vol
        if im:
            prm = B.SolveParams(alpha=0.2, gamma=0.5, step_rule=B.STEP_STRIP, rho=RHO,
                                power_iters=5, pair_sampling=B.PAIRS_UNIFORM,
                                cells=B.CELLS_GEOMETRIC, n_cells=4, seed=1)
        elif n <= 512:
            prm = B.SolveParams(alpha=1 / 5, gamma=2 / 8, step_rule=B.STEP_STRIP, rho=RHO,
                                power_iters=5, pair_sampling=B.PAIRS_UNIFORM, seed=1)
        else:   # a power iteration at 1024^3 takes minutes; the timing does not depend on mu
            prm = B.SolveParams(alpha=1 / 5, gamma=2 / 8, step_rule=B.STEP_FIXED, mu=1e-6,
                                pair_sampling=B.PAIRS_UNIFORM, seed=1)
        t0 = time.perf_counter()
        st = B.State(gg, prm, y)
        t_setup = time.perf_counter() - t0
        x = torch.zeros(gg.n_cols, device=dev)
        st.block_step(x, warm)
        torch.cuda.synchronize()
        q0 = st.query()
        st.profile(True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        st.block_step(x, iters)
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / iters
        prof = st.read_profile()
        q1 = st.query()
        upd = (q1["updates"] - q0["updates"]) / iters
        # the same iterations with FP, residual and BP as separate passes: the
        # per-iteration FP and BP times of Sec. 5's comparison
        st.set_split(True)
        st.profile(False)
        st.block_step(x, 1)
        torch.cuda.synchronize()
        st.profile(True)
        ev0.record()
        st.block_step(x, iters)
        ev1.record()
        torch.cuda.synchronize()
        ms_split = ev0.elapsed_time(ev1) / iters
        prs = st.read_profile()
        out[name] = {
            "volume": "%d^3 (%.2f mm)" % (n, 256.0 / n),
            "detector": "%d^2 (%.2f mm)" % (nd, geo["du"]),
            "rows": gg.n_rows, "cols": gg.n_cols,
            "blocks": "M=5 (random partition), N=8 z-slabs, " + (
                "alpha=0.2, gamma=0.5, geometric detector quadrants (Algorithm 2)" if im
                else "alpha=1/5, gamma=2/8"),
            "ms_per_iteration": round(ms, 3),
            "fused_ms_per_iteration": round(prof["fpbp"]["ms"] / iters, 3),
            "split_ms_per_iteration": round(ms_split, 3),
            "fp_ms_per_iteration": round(prs["fp"]["ms"] / iters, 3),
            "residual_ms_per_iteration": round(prs["residual"]["ms"] / iters, 3),
            "bp_ms_per_iteration": round(prs["bp"]["ms"] / iters, 3),
            "updates_per_iteration": int(upd),
            "value": round(upd / (ms * 1e-3) / 1e9, 3), "unit": UNIT,
            "state_setup_s": round(t_setup, 2), "step": "strip, 5 power iterations" if n <= 512
            else "fixed", "compact_rows_frac": round(gg.compact_rows / (8 * gg.n_rows), 4),
        }
        st.close()
        del y, x
        torch.cuda.empty_cache()
    return out


def serving_leg(B, torch, dev, cfg, seed=3, rate=20.0, budget=160 << 30):
    import numpy as np
    from paper_1903_11874_gb300 import synth
    rng = np.random.default_rng(seed)
    n_req = cfg["n_req"]
    reqs = [(int(rng.choice(cfg["sizes"])), int(rng.choice(cfg["views"])),
             B.F32 if rng.random() < 0.5 else B.BF16) for _ in range(n_req)]
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    data = {}
    phantoms = {}
    for n, v, _ in reqs:
        if (n, v) in data:
            continue
        if n not in phantoms:
            phantoms[n] = torch.from_numpy(
                (synth.ellipsoid_phantom(n, n, n, 10, seed=0) * KAPPA).reshape(-1)).to(dev)
        gg = B.Geometry(M=M, N=N, **serve_geometry(n, v))
        p = torch.zeros(gg.n_rows, device=dev)
        B.bsgd_forward_project(gg, phantoms[n], p)
        data[(n, v)] = p.cpu().numpy().astype(np.float32)
        del gg

    def params(storage, k):
        return B.SolveParams(alpha=1 / M, gamma=1 / N, epochs=cfg["epochs"], rho=RHO,
                             power_iters=8, pair_sampling=B.PAIRS_UNIFORM, storage=storage,
                             seed=100 + k)

    # served: submit at the arrival times, continuous batching on the GPU
    def served_stream(priority):
        srv = B.Server(budget_bytes=budget, max_slots=16, device=torch.cuda.current_device(),
                       priority=priority)
        t0 = time.perf_counter()
        ids = []
        for k, (n, v, st) in enumerate(reqs):
            delay = t0 + arrivals[k] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            ids.append(srv.submit(serve_geometry(n, v), M, N, params(st, k), data[(n, v)]))
        for i in ids:
            srv.wait(i, timeout_ms=3600 * 1000)
        makespan = time.perf_counter() - t0
        stats = srv.stats()
        srv.close()
        return {"p50_ms": round(stats["p50_ms"], 1), "p99_ms": round(stats["p99_ms"], 1),
                "mean_ms": round(stats["mean_ms"], 1),
                "value": round(stats["updates"] / makespan / 1e9, 2), "unit": UNIT,
                "peak_resident": stats["peak_resident"], "peak_gb": round(stats["peak_bytes"] / 1e9, 1),
                "rounds": stats["rounds"]}

    served = served_stream(B.SERVE_SHARED)
    # age priority: the oldest resident request advances every round, the
    # others every second round
    served_age = served_stream(B.SERVE_AGE)
    # the largest request rate the server sustains on this mix: every request
    # submitted at once (a queue that never runs dry), requests / makespan
    srv = B.Server(budget_bytes=budget, max_slots=16, device=torch.cuda.current_device())
    t0 = time.perf_counter()
    ids = [srv.submit(serve_geometry(n, v), M, N, params(st, k), data[(n, v)])
           for k, (n, v, st) in enumerate(reqs)]
    for i in ids:
        srv.wait(i, timeout_ms=3600 * 1000)
    sat = time.perf_counter() - t0
    srv.close()
    served["max_sustainable_req_per_s"] = round(n_req / sat, 2)
    # plain single-request FP32 path, first come first served, same arrivals
    finish, lat, upd, busy = 0.0, [], 0, 0.0
    for k, (n, v, _) in enumerate(reqs):
        gg = B.Geometry(M=M, N=N, **serve_geometry(n, v))
        x = np.zeros(gg.n_cols, dtype=np.float32)
        ts = time.perf_counter()
        rep = B.bsgd_solve(gg, params(B.F32, k), data[(n, v)], x)
        dur = time.perf_counter() - ts
        upd += rep["updates"]
        busy += dur
        finish = max(finish, arrivals[k]) + dur
        lat.append(1e3 * (finish - arrivals[k]))
        del gg
    lat.sort()
    pct = lambda q: lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]
    plain = {"p50_ms": round(pct(0.5), 1), "p99_ms": round(pct(0.99), 1),
             "value": round(upd / max(finish, 1e-9) / 1e9, 2), "unit": UNIT,
             "max_sustainable_req_per_s": round(n_req / max(busy, 1e-9), 2)}
    return {"workload": "Poisson %g req/s, %d requests, n^3 in %s, views in %s, FP32/BF16 mixed, "
                        "8x8 blocks, %d epochs" % (rate, n_req, list(cfg["sizes"]),
                                                    list(cfg["views"]), cfg["epochs"]),
            "offered_req_per_s": rate,
            "served": served, "served_age_priority": served_age, "plain_fp32": plain}


# ---------------------------------------------------------------------------
# CPU side: the FP64 oracle as it stands, on a bounded sample of the workload

def oracle_sample(y_np, mu, n_iters):
    """n_iters BSGD iterations of the oracle (snapshot form, residual-weighted
    pairs) on the same workload; returns (updates, seconds, threads)."""
    import numpy as np
    from oracle import bsgd as OB
    from oracle import projector as OP
    og = OP.Geometry(**GEOM)
    prm = OB.Params(M, N, 1 / M, 1 / N, mu, seed=1, pair_sampling="residual")
    st = OB.BSGDState(og, np.asarray(y_np, dtype=np.float64), prm)
    t0 = time.perf_counter()
    for _ in range(n_iters):
        st.step()
    dt = time.perf_counter() - t0
    upd = 0
    for sel in st.history:
        for (i, j) in sel.pairs:
            rows = OP.rows_of_views(og, OP.row_block_views(og, M, i))
            upd += 2 * OP.count_rows(og, rows, OP.column_block(og, N, j))
    return upd, dt, OP.num_threads()


# One epoch (16 block iterations) of the 64^2 parallel-beam set-up (90 views,
# 96 bins, 4 x 4 blocks) by the FP64 oracle, run in a child process so that its
# OpenMP thread count can be set; prints {"updates", "seconds", "threads"}.
_CONFIG1_EPOCH = r"""
import json, sys, time
sys.path.insert(0, %r)
import numpy as np
from oracle import bsgd as OB
from oracle import projector as OP
from paper_1903_11874_gb300 import synth
og = OP.Geometry("par2d", 64, 64, 1, 1.0, 1.0, 1.0, 90, 96, 1, 1.0, 1.0)
y = OP.fp(og, synth.ellipse_phantom(64, 64, 6, 0).reshape(-1)).reshape(-1)
prm = OB.Params(4, 4, 0.25, 0.25, 1e-3, seed=1)
st = OB.BSGDState(og, y, prm)
st.step()
t0 = time.perf_counter()
for _ in range(16):
    st.step()
dt = time.perf_counter() - t0
upd = 0
for sel in st.history[1:]:
    for (i, j) in sel.pairs:
        upd += 2 * OP.count_rows(og, OP.rows_of_views(og, OP.row_block_views(og, 4, i)),
                                 OP.column_block(og, 4, j))
print(json.dumps({"updates": upd, "seconds": dt, "threads": OP.num_threads()}))
"""


def oracle_config1_epoch(threads):
    env = dict(os.environ)
    if threads:
        env["OMP_NUM_THREADS"] = str(threads)
    r = subprocess.run([sys.executable, "-c", _CONFIG1_EPOCH % os.path.dirname(os.path.abspath(__file__))],
                       capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        return None
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": round(d["updates"] / d["seconds"] / 1e9, 5), "unit": UNIT,
            "cores": d["threads"], "epoch_s": round(d["seconds"], 4)}


def cpu_baseline(y_np, mu, n_iters):
    upd, dt, threads = oracle_sample(y_np, mu, n_iters)
    return {"value": round(upd / dt / 1e9, 5), "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d BSGD iterations (one (row block, z-slab) pair each) of the workload, "
                      "FP64 oracle, %.1f s" % (n_iters, dt),
            # an epoch is 64 such iterations; the oracle's time per iteration does
            # not depend on the iteration (each walks one pair's rays), so one
            # epoch is extrapolated from the sample
            "epoch_s_extrapolated": round(dt / n_iters * ITERS_PER_EPOCH, 1),
            "config1_epoch": {"all_cores": oracle_config1_epoch(None),
                              "single_thread": oracle_config1_epoch(1)}}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    import numpy as np
    from paper_1903_11874_gb300 import synth
    from oracle import projector as OP
    og = OP.Geometry(**GEOM)
    vol = synth.ellipsoid_phantom(256, 256, 256, 10, seed=0).astype(np.float64) * KAPPA
    p = OP.fp(og, vol.reshape(-1)).reshape(-1)
    y = synth.poisson_log_data(p, I0, seed=2)
    from oracle import bsgd as OB
    mu = RHO / 1.0e5          # a fixed step of the right scale; the timing does not depend on it
    prm = OB.Params(M, N, 1 / M, 1 / N, mu, seed=1, pair_sampling="residual")
    st = OB.BSGDState(og, y.astype(np.float64), prm)
    for _ in range(args.warmup):
        st.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st.step()
    dt = time.perf_counter() - t0
    upd = 0
    for sel in st.history[args.warmup:]:
        for (i, j) in sel.pairs:
            rows = OP.rows_of_views(og, OP.row_block_views(og, M, i))
            upd += 2 * OP.count_rows(og, rows, OP.column_block(og, N, j))
    value = upd / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3 / args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded ellipsoid phantom, Poisson noise)",
        "config": bench_config(world),
        "method": {"step": "1 oracle BSGD block iteration per step (a bounded sample of the "
                           "workload's epoch of 64 iterations)"},
        "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": OP.num_threads(),
                         "kind": "oracle",
                         "sample": "%d oracle BSGD iterations after %d warm-up" % (args.steps, args.warmup)},
        "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_cuda(args)


if __name__ == "__main__":
    main()
