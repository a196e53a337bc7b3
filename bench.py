#!/usr/bin/env python
"""Benchmark: observations/s per ADMM iteration of distributed bundle adjustment.

Workload (default): the 4M-observation scene -- 1,000 nadir cameras on a
serpentine 25x40 flight grid at 150 m over 500,000 ground points, power-law
track lengths on [2,50] with mean 8, sigma 0.5 px pixel noise, 5% outliers,
Huber 2 px, FP32 local solves with FP64 consensus and duals.  One step is one
full consensus-ADMM iteration (Eqs. 9-13: every local solve, both consensus
means, the dual ascent) over all observations; inputs are resident in HBM
(~1 GB per iteration, larger than the 129 MB L2, so no flush is needed).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  --impl reference times the FP64 CPU oracle on the
host cores on a bounded sample of the same workload.  For N > 1 (torchrun)
every rank solves its own copy of the scene (independent replicas, no
collective on the data path: weak scaling).
"""
from __future__ import annotations

import argparse
import csv
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

METRIC = "observations/s per ADMM iteration"
UNIT = "obs/s"


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["f32", "f64"], default="f32")
    ap.add_argument("--workload", type=int, choices=[2, 3], default=2,
                    help="2: the 4M-observation scene; 3: a batch of 256 uneven scenes")
    ap.add_argument("--n-pts", type=int, default=500000, help="points of the scene (default: full size)")
    ap.add_argument("--inner-steps", type=int, default=5, help="damped Gauss-Newton steps per local solve")
    ap.add_argument("--tile-obs", type=int, default=0,
                    help="observations per tile (64, 128, 256; 0: the library's choice, -1: autotune)")
    ap.add_argument("--warm-start", action="store_true",
                    help="time the iteration with the learned warm start (shipped weights) in front of the local solves")
    ap.add_argument("--local-solver", choices=["gn", "lbfgs"], default="gn",
                    help="local solver of Eq. (9): damped Gauss-Newton or L-BFGS (Sec. 3.1)")
    ap.add_argument("--block-points", type=int, default=0,
                    help="> 0: time the block subproblems of Eq. (14) with this many points per block")
    ap.add_argument("--block-cams", type=int, default=1, help="cameras per block (with --block-points)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ttt", action="store_true", help="skip the time-to-0.5-px measurement")
    ap.add_argument("--no-workload3", action="store_true", help="skip the batch-of-256-scenes sub-record")
    ap.add_argument("--no-blocks", action="store_true",
                    help="skip the sub-record of the block subproblems (32 points x 2 cameras)")
    ap.add_argument("--blocks-steps", type=int, default=20)
    ap.add_argument("--workload3-steps", type=int, default=100)
    ap.add_argument("--ttt-max-iters", type=int, default=400)
    ap.add_argument("--cpu-iters", type=int, default=2)
    ap.add_argument("--profile-iters", type=int, default=200)
    ap.add_argument("--reference-seconds", type=float, default=90.0,
                    help="wall-clock budget of the whole --impl reference run")
    return ap.parse_args(argv)


def make_scene(args):
    from paper_1708_07954_gb300 import scenes as S

    if args.workload == 3:
        return S.scene3()
    return S.scene2(n_pts=args.n_pts)


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(
        os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(ms, world, device):
    """The slowest rank's time: a MAX all-reduce over the initialised process group."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, n_obs, steps, ms):
    """Whole-job observations per second: every replica solves n_obs observations per step."""
    return world * n_obs * steps / (ms * 1e-3)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait(timeout=10)
        rows = []
        with open(self.path) as fh:
            for r in csv.reader(fh):
                if len(r) >= 9:
                    rows.append([x.strip() for x in r])
        os.unlink(self.path)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(rows), "reasons": reasons}


# ------------------------------------------------------------------ traffic model
def algorithmic_bytes(scene, layout, fp32):
    """Bytes the tile_iterate kernel must move per launch (steady state, each datum once)."""
    esz = 4 if fp32 else 8
    l, n, m = scene.n_obs, scene.n_pts, scene.n_cams
    per_obs = 4 + 4 + 2 * esz + 1 + 2 * 9 * esz + 2 * 9 * 8  # idx, z, camera rank, copies r/w, duals r/w
    per_point = 16 + 24 + 24 + 4 * 3 * esz                     # run table, X read/write, mirror+change r/w
    per_cam_run = 12 + 48                                       # run table, partial sums write
    per_cam = 2 * 6 * esz                                       # camera mirror + change read
    per_tile = 12
    total = (per_obs * l + per_point * n + per_cam_run * layout["camera_runs"] + per_cam * m +
             per_tile * layout["tiles"] + 24 * layout["point_slots"])
    return total, per_obs


# FP32 operations of the method per observation and ADMM iteration, counted from the
# tile kernel's arithmetic (add/sub/mul 1, fma 2, rcp/sqrt/sin/cos 1), every Gauss-Newton
# step counted as a full step with its trial objective (the kernel skips only the trial
# objective of a last step that every lane of a warp accepts by the noise rule, whose value
# is never read: the count is at most 58 / 2684 = 2.2 % above the executed flops):
#   start: copy + pose + objective 111, first damping 50, deferred dual re-base 9, run sums 9;
#   per step: linearisation and Jacobian 64, gradient 64, damping reciprocals 6,
#   capacitance terms 126, 2x2 solve 17, step + model decrease 96, noise bound 7,
#   trial point 18, trial pose 44, trial objective 58, damping update 1  -> 501.
FLOPS_START, FLOPS_PER_STEP = 179, 501
# The same count for the L-BFGS local solve (memory 4, one line-search trial per iteration):
#   start: copy + pose + objective 111, scaling 9, gradient 125, re-base 9, run sums 9;
#   per iteration: two-loop recursion 2 x 83 (on average two stored pairs over five
#   iterations), H0 scaling 37, direction and slope 27, trial point 36, trial pose 44,
#   trial objective 58, gradient at the new point 125, pair update 37      -> 530.
FLOPS_START_LBFGS, FLOPS_PER_STEP_LBFGS = 263, 530

# 152 SMs x 128 FP32 lanes x 2 flops per FMA x 2.07 GHz (maximum SM clock)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


MLP_FLOPS_PER_OBS = 2 * (32 * 64 + 64 * 64 + 64 * 64 + 64 * 16)


def mlp_bytes_per_obs(fp32):
    """Warm-start pass per observation: its offset and dual (9 each), pixel, point and
    camera index read; candidate start (9) written."""
    t = 4 if fp32 else 8
    return 9 * t + 9 * 8 + 2 * t + 4 + 4 + 9 * t


def flops_per_obs(inner_steps, lbfgs=False):
    if lbfgs:
        return FLOPS_START_LBFGS + FLOPS_PER_STEP_LBFGS * inner_steps
    return FLOPS_START + FLOPS_PER_STEP * inner_steps


def algorithmic_flops(n_obs, inner_steps, lbfgs=False):
    return n_obs * flops_per_obs(inner_steps, lbfgs)


def block_bytes(layout, n_obs, fp32):
    """Algorithmic bytes of one block_solve launch: per observation its pixel pair and local
    camera; per point copy its point id, observation offset, offset (read and write) and dual;
    the point's consensus; per camera copy the same with 6 values; a 24-byte block record."""
    t = 4 if fp32 else 8
    per_pc = 4 + 4 + 2 * 3 * t + 3 * 8 + 3 * 8
    per_cc = 4 + 2 * 6 * t + 6 * 8 + 6 * 8
    return n_obs * (2 * t + 1) + layout["n_point_copies"] * per_pc + layout["n_camera_copies"] * per_cc + \
        layout["n_blocks"] * 24


# the sources tile_iterate_kernel is built from; their joint sha256 keys the ncu counters
KERNEL_SOURCES = ("dba_kernels.cu", "dba_device.cuh", "dba_internal.h")


def ncu_traffic(n_obs):
    """DRAM bytes per tile_iterate launch from the committed ncu summary, scaled to n_obs,
    or None when the kernel source changed since the counters were taken."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", "tile_iterate_workload2.json")) as fh:
            prof = json.load(fh)
        sha = hashlib.sha256()
        for name in KERNEL_SOURCES:
            with open(os.path.join(ROOT, "paper_1708_07954_gb300", "csrc", name), "rb") as fh:
                sha.update(fh.read())
        sha = sha.hexdigest()
    except (OSError, ValueError):
        return None
    if prof.get("kernel_source_sha256") != sha:
        return None
    return prof["dram_bytes_per_obs"] * n_obs


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle as O
    from paper_1708_07954_gb300 import scenes as S

    t_gen = time.perf_counter()
    sc = make_scene(args)
    cfg = O.config_for(sc)
    # bounded sample: a sub-problem of whole point tracks sized so that warmup + steps
    # iterations fit the time budget (calibrated on a small probe)
    budget = max(5.0, args.reference_seconds - (time.perf_counter() - t_gen) - 5.0)
    steps = args.steps + args.warmup

    def sub(n_keep):
        keep = sc.pt_idx < n_keep
        s2 = S.Scene(n_cams=sc.n_cams, n_pts=n_keep, pt_idx=sc.pt_idx[keep], cam_idx=sc.cam_idx[keep],
                     z=sc.z[keep], z_true=sc.z_true[keep], outlier=sc.outlier[keep], cams_gt=sc.cams_gt,
                     pts_gt=sc.pts_gt[:n_keep], cams0=sc.cams0, pts0=sc.pts0[:n_keep], name="sample")
        return s2

    # the probe is large enough (~160k observations) for the OpenMP oracle to reach its
    # full-scene rate, so that the whole scene is taken whenever it fits the budget
    n_probe = min(sc.n_pts, 20000)
    probe = sub(n_probe)
    st = O.State(probe)
    t0 = time.perf_counter()
    st.iterate(cfg, 1)
    rate = probe.n_obs / max(time.perf_counter() - t0, 1e-6)
    n_keep = int(min(sc.n_pts, max(50, n_probe * (rate * budget / steps) / max(probe.n_obs, 1))))
    sample = sub(n_keep)
    st = O.State(sample)
    for _ in range(args.warmup):
        st.iterate(cfg, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st.iterate(cfg, 1)
    dt = time.perf_counter() - t0
    value = sample.n_obs * args.steps / dt
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": sc.name, "n_obs": sc.n_obs, "n_cams": sc.n_cams, "n_pts": sc.n_pts,
                   "loss": "huber", "precision": "f64 (CPU oracle)", "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": (f"the whole workload ({sample.n_obs} observations), one ADMM iteration per step"
                                    if n_keep == sc.n_pts else
                                    f"{sample.n_obs} observations ({n_keep} whole tracks, all {sc.n_cams} cameras) "
                                    f"of the workload, one ADMM iteration per step")},
        "whole_workload": n_keep == sc.n_pts,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1708_07954_gb300 import build, dba
    from paper_1708_07954_gb300 import scenes as S

    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    build.build()
    dba.load()
    fp32 = args.precision == "f32"
    prec = dba.DBA_PREC_F32_LOCAL if fp32 else dba.DBA_PREC_F64
    sc = make_scene(args)
    stream = torch.cuda.Stream()  # a real stream: the library launches on it, events are recorded on it
    lbfgs = args.local_solver == "lbfgs"
    lsolver = dba.DBA_SOLVER_LBFGS if lbfgs else dba.DBA_SOLVER_GN
    solver = dba.Solver(sc, precision=prec, inner_steps=args.inner_steps, stream=stream.cuda_stream,
                        local_solver=lsolver, tile_obs=args.tile_obs)
    if args.warm_start:
        from paper_1708_07954_gb300 import warmstart

        solver.set_warm_start(warmstart.load())
    layout = solver.layout()
    solver.iterate(args.warmup, stats=False)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    clocks = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
    clocks.start()
    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solver.iterate(args.steps, stats=False)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    value = job_throughput(world, sc.n_obs, args.steps, ms)
    # the same steps again as five separately timed runs: their per-step times and median
    runs = []
    for _ in range(5):
        r0 = torch.cuda.Event(enable_timing=True)
        r1 = torch.cuda.Event(enable_timing=True)
        n_run = max(1, args.steps // 5)
        r0.record(stream)
        solver.iterate(n_run, stats=False)
        r1.record(stream)
        torch.cuda.synchronize()
        runs.append(max_over_ranks(r0.elapsed_time(r1), world, "cuda") / n_run)
    final = solver.evaluate()
    # K5 (the metrics of Sec. 4 at consensus: reprojection RMSE, objective, residuals) is not
    # part of the timed steps, which run K1-K4; one metrics pass is timed here on its own
    k5 = []
    for _ in range(5):
        m0 = torch.cuda.Event(enable_timing=True)
        m1 = torch.cuda.Event(enable_timing=True)
        m0.record(stream)
        solver.evaluate()
        m1.record(stream)
        torch.cuda.synchronize()
        k5.append(m0.elapsed_time(m1))
    k5_ms = float(np.median(k5))

    # per-kernel device time (CUDA events around each launch on the same stream)
    prof = solver.profile(min(args.profile_iters, max(args.steps, 1)))
    tile_ms = prof["tile_iterate"]
    bytes_launch, per_obs = algorithmic_bytes(sc, layout, fp32)
    peaks, src = measured_peaks()
    flops = algorithmic_flops(sc.n_obs, args.inner_steps, lbfgs)
    achieved_tf = flops / (tile_ms * 1e-3) / 1e12
    achieved_gbs = bytes_launch / (tile_ms * 1e-3) / 1e9
    roofline = {"bound": "alu", "achieved": achieved_tf, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved_tf / FP32_PEAK_TFLOPS, "traffic": None if lbfgs else ncu_traffic(sc.n_obs),
                "kernel": "tile_iterate", "kernel_ms": tile_ms, "kernel_share": tile_ms / sum(prof.values()),
                "algorithmic_flops_per_launch": flops,
                "algorithmic_flops_per_obs": flops_per_obs(args.inner_steps, lbfgs),
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz (unit counts and maximum clock)",
                "hbm": {"achieved": achieved_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": achieved_gbs / peaks["hbm_gbs"], "algorithmic_bytes_per_launch": bytes_launch,
                        "algorithmic_bytes_per_obs": per_obs,
                        "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else "fallback"},
                "kernels_ms": prof}
    if args.warm_start:
        # the network pass: 11,264 multiply-adds per observation on the tensor cores; state in, start out
        mlp_ms = prof["mlp_warm_start"]
        mlp_tf = sc.n_obs * MLP_FLOPS_PER_OBS / (mlp_ms * 1e-3) / 1e12
        mlp_gbs = sc.n_obs * mlp_bytes_per_obs(fp32) / (mlp_ms * 1e-3) / 1e9
        roofline["warm_start"] = {
            "kernel": "mlp_warm_start", "kernel_ms": mlp_ms, "tensor_tflops": mlp_tf,
            "tensor_frac": mlp_tf / peaks["bf16_tflops"], "tensor_peak": peaks["bf16_tflops"],
            "hbm_gbs": mlp_gbs, "hbm_frac": mlp_gbs / peaks["hbm_gbs"],
            "algorithmic_flops_per_obs": MLP_FLOPS_PER_OBS, "algorithmic_bytes_per_obs": mlp_bytes_per_obs(fp32)}
    solver.close()

    e2e = None
    if not args.no_e2e:
        # end to end through the C ABI with host buffers: upload + layout, all iterations, read back
        iters = sc.iters if args.workload == 2 else 50
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with dba.Solver(sc, precision=prec, inner_steps=args.inner_steps, stream=stream.cuda_stream,
                        ground_truth=False, local_solver=lsolver) as s2:
            s2.iterate(iters, stats=False)
            s2.params()
        dt = time.perf_counter() - t0
        h2d = sc.n_obs * (4 + 4 + 16) + sc.n_cams * 48 + sc.n_pts * 24
        d2h = sc.n_cams * 48 + sc.n_pts * 24
        e2e = {"value": sc.n_obs * iters / dt, "unit": UNIT, "h2d_bytes_per_step": h2d / iters,
               "d2h_bytes_per_step": d2h / iters, "iters_per_solve": iters, "seconds_per_solve": dt,
               "what": "dba_create + dba_set_observations (host arrays, layout, upload) + dba_iterate("
                       f"{iters}) + dba_get_params, wall clock"}

    w3 = None
    if args.workload == 2 and not args.no_workload3 and world == 1:
        # the batch of 256 uneven scenes (workload 3): one persistent tile launch per iteration
        # over all scenes, tile size picked by the library's autotuner
        sc3 = S.scene3()
        with dba.Solver(sc3, precision=prec, inner_steps=args.inner_steps, stream=stream.cuda_stream,
                        tile_obs=-1, ground_truth=False, local_solver=lsolver) as s3:
            lay3 = s3.layout()
            s3.iterate(args.warmup, stats=False)
            torch.cuda.synchronize()
            b0 = torch.cuda.Event(enable_timing=True)
            b1 = torch.cuda.Event(enable_timing=True)
            b0.record(stream)
            s3.iterate(args.workload3_steps, stats=False)
            b1.record(stream)
            torch.cuda.synchronize()
            ms3 = b0.elapsed_time(b1)
            prof3 = s3.profile(min(50, args.workload3_steps))
        w3 = {"workload": "batch256-uneven", "n_scenes": len(sc3.scene_off) - 1, "n_obs": sc3.n_obs,
              "n_cams": sc3.n_cams, "n_pts": sc3.n_pts, "steps": args.workload3_steps,
              "value": sc3.n_obs * args.workload3_steps / (ms3 * 1e-3), "unit": UNIT,
              "ms_per_step": ms3 / args.workload3_steps, "tile_obs": lay3["tile_obs"],
              "finalize_threads": lay3.get("finalize_threads"), "kernels_ms": prof3,
              "tile_iterate_frac_of_fp32_peak": sc3.n_obs * flops_per_obs(args.inner_steps, lbfgs) /
              (prof3["tile_iterate"] * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
              "what": "all scenes in one tile_iterate launch + one finalize per ADMM iteration (CUDA graph), "
                      "tile size and finalize block size by the autotuner (tile_obs = -1)"}

    blocks = None
    if args.workload == 2 and fp32 and not args.no_blocks and world == 1 and not args.warm_start:
        blocks = block_subrecord(args, sc, stream)

    ttt = None
    if not args.no_ttt and args.workload == 2:
        # time to rmse_gt <= 0.5 px (noise-free projections, observations of outlier-free tracks),
        # device time of iterations + per-iteration metrics, each precision from the initial state
        ttt = {"target_px": 0.5, "rmse": "vs noise-free projections over observations of outlier-free tracks",
               "max_iters": args.ttt_max_iters}
        for name, pr in (("fp32_plain", dba.DBA_PREC_F32_LOCAL), ("fp64_plain", dba.DBA_PREC_F64)):
            with dba.Solver(sc, precision=pr, inner_steps=args.inner_steps, stream=stream.cuda_stream,
                            local_solver=lsolver) as s3:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                m = s3.iterate_until(args.ttt_max_iters, 0.5)
                wall = time.perf_counter() - t0
            ttt[name] = {"seconds": m["seconds"], "wall_seconds": wall, "iters": m["iters_done"],
                         "rmse_gt": m["rmse_gt"], "reached": m["rmse_gt"] <= 0.5}
        # learned warm start (one Gauss-Newton step per local solve) beside the same
        # solver without it; the network's weights ship with the package
        from paper_1708_07954_gb300 import warmstart

        ttt["fp32_learned"] = None
        if os.path.exists(warmstart.WEIGHTS):
            mlp = warmstart.load()
            for name, warm in (("fp32_plain_1step", False), ("fp32_learned", True)):
                with dba.Solver(sc, precision=dba.DBA_PREC_F32_LOCAL, inner_steps=1,
                                stream=stream.cuda_stream) as s3:
                    if warm:
                        s3.set_warm_start(mlp)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    m = s3.iterate_until(args.ttt_max_iters, 0.5)
                    wall = time.perf_counter() - t0
                ttt[name] = {"seconds": m["seconds"], "wall_seconds": wall, "iters": m["iters_done"],
                             "rmse_gt": m["rmse_gt"], "reached": m["rmse_gt"] <= 0.5, "inner_steps": 1}
            ttt["fp32_learned"]["network"] = "32-64-64-64-16 GELU MLP, BF16 tcgen05 inference, FP32 accumulation"
            mlp.close()
        for a, b in (("fp32_plain", "fp64_plain"), ("fp32_learned", "fp64_plain"), ("fp32_learned", "fp32_plain"),
                     ("fp32_learned", "fp32_plain_1step")):
            if ttt.get(a) and ttt.get(b) and ttt[a]["reached"] and ttt[b]["reached"]:
                ttt[f"speedup_{a}_vs_{b}"] = ttt[b]["seconds"] / ttt[a]["seconds"]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O

        cfg = O.config_for(sc, local_solver=O.SOLVER_LBFGS if lbfgs else O.SOLVER_GN)
        st = O.State(sc)
        t0 = time.perf_counter()
        st.iterate(cfg, args.cpu_iters)
        dt = time.perf_counter() - t0
        cpu = {"value": sc.n_obs * args.cpu_iters / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{args.cpu_iters} ADMM iterations of the full {sc.n_obs}-observation scene (FP64, "
                         f"OpenMP over local solves and dual updates)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "admm_iterations_per_s": 1e3 * args.steps / ms,
            "ms_per_step_runs": runs, "ms_per_step_median_of_runs": float(np.median(runs)),
            "vs_baseline": None, "dtype": "f32+f64" if fp32 else "f64", "data": "synthetic",
            "config": {"workload": sc.name, "n_obs": sc.n_obs, "n_cams": sc.n_cams, "n_pts": sc.n_pts,
                       "n_scenes": 1 if sc.scene_off is None else len(sc.scene_off) - 1,
                       "loss": "huber", "inner_steps": args.inner_steps, "local_solver": args.local_solver,
                       "warm_start": bool(args.warm_start),
                       "precision": "f32 local solves, f64 consensus/duals" if fp32 else "f64",
                       "l2": "inputs larger than L2 (~1 GB per iteration), no flush",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "time_to_target": ttt,
            "metrics_pass": {"ms": k5_ms, "in_timed_steps": False,
                             "value_with_metrics_every_step": sc.n_obs / ((ms / args.steps + k5_ms) * 1e-3),
                             "what": "K5: consensus camera poses, per-observation reprojection and residual "
                                     "sums, final reduction (one dba_evaluate, CUDA events)"},
            "workload3": w3,
            "blocks": blocks,
            "clocks": clk, "gpu_launches": (3 if args.warm_start else 2) * args.steps,
            "final": {k: final[k] for k in ("rmse_obs", "rmse_gt", "objective", "iters_done")},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ------------------------------------------------------------------ block subproblems
def block_subrecord(args, sc, stream, pi=32, kappa=2):
    """The same scene solved with block subproblems of Eq. (14), pi points x kappa cameras
    per update (Sec. 4 finds about 32 points per update fastest): ms per iteration by CUDA
    events, the block solve's share and roofline, and the time to 0.5 px."""
    import torch

    from paper_1708_07954_gb300 import dba

    with dba.BlockSolver(sc, pi, kappa, precision=dba.DBA_PREC_F32_LOCAL, inner_steps=args.inner_steps,
                         stream=stream.cuda_stream) as s:
        layout = s.layout()
        launches = s.launches_per_iteration()
        s.iterate(args.warmup, stats=False)
        torch.cuda.synchronize()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        s.iterate(args.blocks_steps, stats=False)
        b1.record(stream)
        torch.cuda.synchronize()
        ms = b0.elapsed_time(b1) / args.blocks_steps
        prof = s.profile(args.blocks_steps)
        flops = s.algorithmic_flops()
    achieved_tf = flops / (prof["block_solve"] * 1e-3) / 1e12
    rec = {"block_points": pi, "block_cams": kappa, **layout, "steps": args.blocks_steps, "ms_per_step": ms,
           "value": sc.n_obs / (ms * 1e-3), "unit": UNIT, "kernels_ms": prof,
           "block_solve_roofline": {"bound": "alu", "achieved": achieved_tf, "peak": FP32_PEAK_TFLOPS,
                                    "unit": "TFLOP/s", "frac": achieved_tf / FP32_PEAK_TFLOPS,
                                    "algorithmic_flops_per_launch": flops},
           "gpu_launches_per_step": launches, "time_to_target": None,
           "what": "block solves + point and camera consensus per ADMM iteration, FP32 block solves, "
                   "FP64 consensus and duals"}
    if not args.no_ttt:
        with dba.BlockSolver(sc, pi, kappa, precision=dba.DBA_PREC_F32_LOCAL, inner_steps=args.inner_steps,
                             stream=stream.cuda_stream) as s:
            m = s.iterate_until(args.ttt_max_iters, 0.5)
        rec["time_to_target"] = {"target_px": 0.5, "seconds": m["seconds"], "iters": m["iters_done"],
                                 "rmse_gt": m["rmse_gt"], "reached": m["rmse_gt"] <= 0.5}
    return rec


def run_blocks(args, rank, world, local_rank):
    """The same line for the block subproblems of Eq. (14): block_points x block_cams per
    update, one iteration = block solves, consensus over copies, dual ascent."""
    import torch

    from paper_1708_07954_gb300 import build, dba

    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    build.build()
    dba.load()
    fp32 = args.precision == "f32"
    prec = dba.DBA_PREC_F32_LOCAL if fp32 else dba.DBA_PREC_F64
    P, K = args.block_points, args.block_cams
    sc = make_scene(args)
    stream = torch.cuda.Stream()
    solver = dba.BlockSolver(sc, P, K, precision=prec, inner_steps=args.inner_steps, stream=stream.cuda_stream)
    layout = solver.layout()
    classes = solver.size_classes()
    launches = solver.launches_per_iteration()
    solver.iterate(args.warmup, stats=False)
    clocks = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
    clocks.start()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solver.iterate(args.steps, stats=False)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    value = job_throughput(world, sc.n_obs, args.steps, ms)
    final = solver.iterate(0)
    prof = solver.profile(min(args.profile_iters, max(args.steps, 1)))
    flops = solver.algorithmic_flops()
    solve_ms = prof["block_solve"]
    peaks, src = measured_peaks()
    achieved_tf = flops / (solve_ms * 1e-3) / 1e12
    bytes_launch = block_bytes(layout, sc.n_obs, fp32)
    achieved_gbs = bytes_launch / (solve_ms * 1e-3) / 1e9
    roofline = {"bound": "alu", "achieved": achieved_tf, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved_tf / FP32_PEAK_TFLOPS, "traffic": None, "kernel": "block_solve",
                "kernel_ms": solve_ms, "kernel_share": solve_ms / sum(prof.values()),
                "algorithmic_flops_per_launch": flops, "algorithmic_flops_per_obs": flops / sc.n_obs,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz (unit counts and maximum clock)",
                "hbm": {"achieved": achieved_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": achieved_gbs / peaks["hbm_gbs"], "algorithmic_bytes_per_launch": bytes_launch,
                        "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else "fallback"},
                "kernels_ms": prof}
    solver.close()
    e2e = None
    if not args.no_e2e:
        iters = sc.iters
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with dba.BlockSolver(sc, P, K, precision=prec, inner_steps=args.inner_steps, stream=stream.cuda_stream,
                             ground_truth=False) as s2:
            s2.iterate(iters, stats=False)
            s2.params()
        dt = time.perf_counter() - t0
        h2d = sc.n_obs * (4 + 4 + 16) + sc.n_cams * 48 + sc.n_pts * 24
        d2h = sc.n_cams * 48 + sc.n_pts * 24
        e2e = {"value": sc.n_obs * iters / dt, "unit": UNIT, "h2d_bytes_per_step": h2d / iters,
               "d2h_bytes_per_step": d2h / iters, "iters_per_solve": iters, "seconds_per_solve": dt,
               "what": f"dba_block_create + dba_block_set_observations + dba_block_iterate({iters}) + "
                       "dba_block_get_params, wall clock"}
    ttt = None
    if not args.no_ttt:
        with dba.BlockSolver(sc, P, K, precision=prec, inner_steps=args.inner_steps, stream=stream.cuda_stream) as s3:
            m = s3.iterate_until(args.ttt_max_iters, 0.5)
        ttt = {"target_px": 0.5, "seconds": m["seconds"], "iters": m["iters_done"], "rmse_gt": m["rmse_gt"],
               "reached": m["rmse_gt"] <= 0.5}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        from paper_1708_07954_gb300 import scenes as S

        # the oracle's block iteration on whole tracks of the first points, all cameras
        n_keep = min(sc.n_pts, 20000)
        keep = sc.pt_idx < n_keep
        sample = S.Scene(n_cams=sc.n_cams, n_pts=n_keep, pt_idx=sc.pt_idx[keep], cam_idx=sc.cam_idx[keep],
                         z=sc.z[keep], z_true=sc.z_true[keep], outlier=sc.outlier[keep], cams_gt=sc.cams_gt,
                         pts_gt=sc.pts_gt[:n_keep], cams0=sc.cams0, pts0=sc.pts0[:n_keep], name="sample")
        cfg = O.config_for(sc)
        cfg.inner_steps = args.inner_steps
        st = O.BlockState(sample, P, K)
        t0 = time.perf_counter()
        st.iterate(cfg, args.cpu_iters)
        dt = time.perf_counter() - t0
        cpu = {"value": sample.n_obs * args.cpu_iters / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{args.cpu_iters} block ADMM iterations of {sample.n_obs} observations ({n_keep} whole "
                         f"tracks, all cameras) of the workload (FP64, OpenMP over blocks)"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "admm_iterations_per_s": 1e3 * args.steps / ms,
            "vs_baseline": None, "dtype": "f32+f64" if fp32 else "f64", "data": "synthetic",
            "config": {"workload": sc.name, "n_obs": sc.n_obs, "n_cams": sc.n_cams, "n_pts": sc.n_pts,
                       "path": "blocks", "block_points": P, "block_cams": K, **layout,
                       "blocks_per_size_class": classes,
                       "loss": "huber", "inner_steps": args.inner_steps,
                       "precision": "f32 block solves, f64 consensus/duals" if fp32 else "f64",
                       "l2": "inputs larger than L2, no flush",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "time_to_target": ttt,
            "clocks": clk, "gpu_launches": launches * args.steps,
            "final": {k: final[k] for k in ("rmse_obs", "rmse_gt", "objective", "iters_done")},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.block_points > 0:
        return run_blocks(args, rank, world, local_rank)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
