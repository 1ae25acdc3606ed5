"""Benchmark of the articulated radiance-field render path on B300.

Workload (one step = one animated frame, the whole forward hot path):
  540 x 540 render of the 24-joint SMPL-like subject (synthetic, seed 0), poses
  drawn from a 32-pose seeded sequence; per step the bone chain and blended
  skinning grid are rebuilt (ia_set_pose), the 64^3 occupancy grid is refreshed
  for the pose (ia_update_occupancy) and the frame is rendered (ia_render) with
  plain fp32 24-start Broyden correspondence search, 16 x 2 hash grid (T = 2^19),
  64-wide MLP, <= 128 slots per ray, early termination at T < 1e-4.

`value` is frames/s over all ranks (replicas: every rank renders its own frames,
no collective on the data path).  L2 is flushed (256 MiB write) before every
timed step.  `--impl reference` times the fp64 CPU oracle on bounded samples of
the same workload.
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

import synthetic as S  # noqa: E402

METRIC = "posed samples/s, 540² frames/s, fwd+bwd step ms: FP16+proposal vs plain FP32"
WORKLOAD = ("540x540 render, 24-joint SMPL-like synthetic subject, 32-pose sequence, per-pose 64^3 "
            "occupancy refresh, plain fp32 24-start Broyden, hash 16x2 T=2^19, MLP 64x2, <=128 slots, "
            "early stop T<1e-4")
EARLY_T = 1e-4
N_POSES = 32

# FLOPs of one algorithmic step of the path (multiply-add = 2), counted from the
# operations the method performs, not from the instructions the kernel issues.
FLOP_START = 306       # x0 = N_k^-1 x', LBS value (8-corner trilinear blend of 3x4), residual, 3x3 inverse
FLOP_ITER = 320        # Broyden step: H r, LBS value, residual difference, rank-one update of H
FLOP_ROOT = 620 + 960 + 12800 + 40  # Newton polish with the analytic Jacobian, hash encoding, MLP, activations
FLOP_SAMPLE = 20       # alpha, transmittance, colour accumulation


def fp32_peak_tflops(sm_mhz: float) -> float:
    return 148 * 128 * 2 * sm_mhz * 1e6 / 1e12


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait(timeout=10)
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s in sm if s > 0.5 * (max(mx) if mx else 1)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ our arm

def setup_ours(torch, ia, rank):
    sc = S.make_scene("full", 0)
    table, mlp = S.make_field(sc, 0)
    cfg = ia.make_config(n_levels=sc.n_levels, log2_table=sc.log2_table, level_res=sc.level_res,
                         max_samples=sc.max_samples, broyden_max_iter=sc.broyden_max_iter,
                         broyden_tol=sc.broyden_tol, occ_res=sc.occ_res, occ_tau=sc.occ_tau,
                         occ_dilate=sc.occ_dilate, early_stop_T=EARLY_T)
    ctx = ia.ia_create(cfg)
    ia.ia_set_skeleton(ctx, sc.parents, sc.rest_joints, sc.skin_grid, sc.canon_min, sc.canon_max,
                       sc.norm_min, sc.norm_max)
    ia.ia_set_params(ctx, torch.from_numpy(table).cuda(), torch.from_numpy(S.pack_mlp(mlp)).cuda())
    poses = [S.make_pose(sc, (rank * N_POSES + i) % 1024) for i in range(N_POSES)]
    cam = S.make_camera(sc)
    icam = ia.make_camera(cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["width"], cam["height"], cam["c2w"])
    return sc, table, mlp, ctx, poses, cam, icam


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2212_10550_b300 as ia

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    sc, table, mlp, ctx, poses, cam, icam = setup_ours(torch, ia, rank)
    W, H = cam["width"], cam["height"]
    rgb = torch.zeros(W * H, 3, device=dev)
    alpha = torch.zeros(W * H, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(i):
        th, tr = poses[i % N_POSES]
        ia.ia_set_pose(ctx, th[None], tr[None], stream=stream)
        ia.ia_update_occupancy(ctx, 0, ia.IA_OCC_POSE, stream=stream)
        ia.ia_render(ctx, 0, icam, rgb, alpha, stream=stream)

    # per-step work counters (one untimed pass over the whole sequence)
    tot = {}
    occ_tot = {}
    for i in range(N_POSES):
        th, tr = poses[i]
        ia.ia_set_pose(ctx, th[None], tr[None])
        o = ia.ia_update_occupancy(ctx, 0, ia.IA_OCC_POSE, stats=True)
        r = ia.ia_render(ctx, 0, icam, rgb, alpha, stats=True)
        for k, v in r.items():
            tot[k] = tot.get(k, 0) + v
        for k, v in o.items():
            occ_tot[k] = occ_tot.get(k, 0) + v
    per_frame = {k: v / N_POSES for k, v in tot.items()}
    occ_per_frame = {k: v / N_POSES for k, v in occ_tot.items()}

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()  # L2 flush outside the timed events
        a, b, c = ev[i]
        th, tr = poses[i % N_POSES]
        a.record(stream)
        ia.ia_set_pose(ctx, th[None], tr[None], stream=stream)
        ia.ia_update_occupancy(ctx, 0, ia.IA_OCC_POSE, stream=stream)
        b.record(stream)
        ia.ia_render(ctx, 0, icam, rgb, alpha, stream=stream)
        c.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(c) for a, b, c in ev]
    render_ms = [b.elapsed_time(c) for a, b, c in ev]
    local_total_s = sum(step_ms) / 1e3

    # ---- end to end through the C ABI with host buffers (pinned), copies inside
    h_rgb = torch.empty(W * H, 3, dtype=torch.float32, pin_memory=True).numpy()
    h_a = torch.empty(W * H, dtype=torch.float32, pin_memory=True).numpy()
    e2e_s = []
    for i in range(max(3, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        th, tr = poses[i % N_POSES]
        t = time.perf_counter()
        ia.ia_set_pose(ctx, th[None], tr[None], stream=stream)
        ia.ia_update_occupancy(ctx, 0, ia.IA_OCC_POSE, stream=stream)
        ia.ia_render(ctx, 0, icam, h_rgb, h_a, stream=stream)  # copies back and synchronises
        e2e_s.append(time.perf_counter() - t)

    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([local_total_s], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_s = float(tt.item())
    else:
        total_s = local_total_s
    ia.ia_destroy(ctx)
    if rank != 0:
        return None
    frames = args.steps * world
    ms_per_step = 1e3 * total_s / args.steps
    fps = frames / total_s
    peaks, peak_kind = load_peaks()
    sm_mhz = peaks.get("sm_max_mhz", 2032.0)
    peak = fp32_peak_tflops(sm_mhz)
    flop_render = (FLOP_START * per_frame["starts"] + FLOP_ITER * per_frame["broyden_iters"] +
                   FLOP_ROOT * per_frame["roots"] + FLOP_SAMPLE * per_frame["occupied_samples"])
    r_ms = statistics.mean(render_ms)
    achieved = flop_render / (r_ms * 1e-3) / 1e12
    line = {
        "metric": METRIC,
        "value": round(fps, 3),
        "unit": "frames/s (540x540, pose + occupancy refresh + render)",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "flushed (256 MiB write) before every timed step",
                   "parallelism": f"replicas x{world}", "precision": "fp32", "starts": "all 24 bones"},
        "samples_per_s": round(per_frame["occupied_samples"] * fps, 1),
        "render_only_fps": round(1e3 / r_ms, 3),
        "per_frame": {k: round(v, 1) for k, v in per_frame.items()},
        "occupancy_per_frame": {k: round(v, 1) for k, v in occ_per_frame.items()},
        "step_ms": {"mean": round(statistics.mean(step_ms), 4), "min": round(min(step_ms), 4),
                    "max": round(max(step_ms), 4)},
        "render_ms": {"mean": round(r_ms, 4), "min": round(min(render_ms), 4)},
        "wall_s": round(wall, 3),
        "roofline": {"kernel": "render_kernel", "bound": "alu", "achieved": round(achieved, 3),
                     "peak": round(peak, 2), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                     "traffic": None,
                     "peak_source": f"fp32 FMA: 148 SM x 128 lanes x 2 x {sm_mhz:.0f} MHz ({peak_kind} max clock)",
                     "flop_per_frame": round(flop_render)},
        "e2e": {"value": round(1.0 / statistics.mean(e2e_s), 3), "unit": "frames/s",
                "h2d_bytes_per_step": int(sc.n_bones * 3 * 8 + 3 * 8),
                "d2h_bytes_per_step": int(W * H * 4 * 4)},
        "gpu_launches": 5 * args.steps,
        "clocks": clk,
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(sc, table, mlp, poses[0], cam)
    return line


# ------------------------------------------------------------------ oracle

def cpu_baseline(sc, table, mlp, pose, cam):
    """Oracle, as it stands, on the host cores: full occupancy grid plus a quarter
    of the image rows (4-row stripes), scaled to one frame."""
    import oracle as O
    nthreads = os.cpu_count() or 1
    om = O.OracleModel(sc, table, mlp, early_T=EARLY_T)
    p = om.pose(*pose)
    t = time.perf_counter()
    _, bits = om.occupancy(p, nthreads)
    t_occ = time.perf_counter() - t
    W, H = cam["width"], cam["height"]
    rows = [r for r in range(H) if (r // 4) % 4 == 0]
    pix = np.concatenate([np.arange(r * W, (r + 1) * W) for r in rows]).astype(np.int32)
    t = time.perf_counter()
    om.render_pixels(p, cam, bits, pix, nthreads)
    t_ren = time.perf_counter() - t
    frame_s = t_occ + t_ren * H / len(rows)
    return {"value": round(1.0 / frame_s, 5), "unit": "frames/s", "cores": nthreads, "kind": "oracle",
            "sample": f"pose 0: full 64^3 occupancy ({t_occ:.1f} s) + {len(rows)} of {H} image rows "
                      f"({t_ren:.1f} s) scaled to {H} rows; fp64 C, OpenMP over cells and rays"}


def run_reference(args, rank, world):
    """The fp64 oracle on bounded samples of the workload: step i evaluates
    part i of 64 of one frame (a z-slab of the occupancy grid and every 64th
    2-row stripe of the image) and scales each part's time by 64."""
    if rank != 0:
        return None
    import oracle as O
    sc = S.make_scene("full", 0)
    table, mlp = S.make_field(sc, 0)
    cam = S.make_camera(sc)
    nthreads = os.cpu_count() or 1
    om = O.OracleModel(sc, table, mlp, early_T=EARLY_T)
    p = om.pose(*S.make_pose(sc, 0))
    _, bits = om.occupancy(p, nthreads)  # the render samples need the whole grid; built once, untimed
    R, W, H = sc.occ_res, cam["width"], cam["height"]
    n_parts = 64

    def one(i):
        part = (i * 17) % n_parts
        z0, z1 = part * R // n_parts, (part + 1) * R // n_parts
        cells = np.arange(z0 * R * R, max(z1, z0 + 1) * R * R)
        t = time.perf_counter()
        om.occupancy_cells(p, cells, nthreads)
        t_occ = time.perf_counter() - t
        rows = [r for r in range(H) if (r // 2) % n_parts == part]
        pix = np.concatenate([np.arange(r * W, (r + 1) * W) for r in rows]).astype(np.int32)
        t = time.perf_counter()
        om.render_pixels(p, cam, bits, pix, nthreads)
        t_ren = time.perf_counter() - t
        return t_occ * (R ** 3) / len(cells) + t_ren * H / len(rows)

    for i in range(args.warmup):
        one(i)
    est = []
    t0 = time.perf_counter()
    for i in range(args.steps):
        est.append(one(args.warmup + i))
    wall = time.perf_counter() - t0
    fps = 1.0 / statistics.mean(est)
    return {"impl": "reference", "metric": METRIC, "value": round(fps, 5), "unit": "frames/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * statistics.mean(est), 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "parallelism": f"{nthreads} host threads"},
            "wall_s": round(wall, 2),
            "cpu_baseline": {"value": round(fps, 5), "unit": "frames/s", "cores": nthreads, "kind": "oracle",
                             "sample": f"pose 0; per step 1/{n_parts} of the occupancy grid (a z-slab) and of "
                                       "the image rows (2-row stripes), each part's time scaled by 64 to a frame"},
            "e2e": {"value": round(fps, 5), "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        line = run_ours(args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
