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
timed step.  The line also carries the metric's other parts (fp16 + proposal
frames/s and samples/s, fwd+bwd train-step times), per-kernel rooflines (work
per launch from the library's counters over per-launch device times from its
launch tracing), the correspondence residual of both searches, the training
quality run and the empty-space-skipping ablation.  `--impl reference` times
the fp64 CPU oracle on bounded samples of the same workload.
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
FLOP_MLP_BWD = 12800 + 25600        # recomputed MLP forward + its backward, per sample
# Algorithmic bytes, from the data each step must touch (not from what a kernel
# happens to load):
GATHER_LBS = 8 * 48          # one LBS evaluation: 8 corners of the blended grid, 3 x float4 each
GATHER_HASH = 16 * 8 * 8     # one field evaluation: 16 levels x 8 corners x 2 fp32 features
GATHER_HASH_H = 16 * 8 * 4   # the same from the fp16 shadow table
GATHER_PROP = 8 * 8 * 8      # one proposal evaluation: 8 levels x 8 corners x 2 fp32 features
WGRAD_ROW_BYTES = 384 * 2    # the weight-gradient GEMM streams one 384-row fp16 column per sample


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

def job_seconds(local_s, world, device):
    """The job's time under torchrun: the slowest rank's (all-reduce MAX over
    the process group); with one process, the local time."""
    if world <= 1:
        return local_s
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_s], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, local_s, world, device):
    """Whole-job throughput of independent replicas: every rank's units over
    the slowest rank's time; returns (rate, job seconds)."""
    total_s = job_seconds(local_s, world, device)
    return units_per_rank * world / total_s, total_s


def make_ctx(torch, ia, sc, table, mlp, precision, early_T):
    cfg = ia.make_config(n_levels=sc.n_levels, log2_table=sc.log2_table, level_res=sc.level_res,
                         max_samples=sc.max_samples, broyden_max_iter=sc.broyden_max_iter,
                         broyden_tol=sc.broyden_tol, occ_res=sc.occ_res, occ_tau=sc.occ_tau,
                         occ_dilate=sc.occ_dilate, early_stop_T=early_T, precision=precision)
    ctx = ia.ia_create(cfg)
    ia.ia_set_skeleton(ctx, sc.parents, sc.rest_joints, sc.skin_grid, sc.canon_min, sc.canon_max,
                       sc.norm_min, sc.norm_max)
    ia.ia_set_params(ctx, torch.from_numpy(table).cuda(), torch.from_numpy(S.pack_mlp(mlp)).cuda())
    return ctx


def occupied_points(bits, sc, n, rng):
    """Uniform points inside the occupied cells of a packed grid (training-pair sampling)."""
    R = sc.occ_res
    occ = np.unpackbits(np.asarray(bits).view(np.uint8), bitorder="little")[:R ** 3].astype(bool)
    c = rng.choice(np.nonzero(occ)[0], n)
    ijk = np.stack([c % R, (c // R) % R, c // (R * R)], -1)
    cs = (sc.norm_max.astype(np.float64) - sc.norm_min) / R
    return (sc.norm_min + (ijk + rng.uniform(size=(n, 3))) * cs).astype(np.float32)


def train_proposal(torch, ia, ctx, sc, n_poses=256, per_pose=8192, steps=1000, batch=8192, lr=2e-3):
    """Proposal pairs from the plain search over n_poses seed-drawn poses (not the
    benchmark sequence), then training with the library's kernels."""
    pc = S.proposal_config()
    ia.ia_proposal_init(ctx, ia.make_proposal_config(pc["n_levels"], pc["log2_table"], pc["level_res"],
                                                     pc["top_k"], pc["offset_weight"]))
    pt, pm = S.proposal_init(sc, pc, 0)
    ia.ia_proposal_set_params(ctx, torch.from_numpy(pt).cuda(), torch.from_numpy(S.pack_proposal(pm)).cuda())
    poses = [S.make_pose(sc, 5000 + i) for i in range(n_poses)]
    ia.ia_set_pose(ctx, np.stack([p[0] for p in poses]), np.stack([p[1] for p in poses]))
    rng = np.random.default_rng(77)
    R = sc.occ_res
    bits = torch.zeros((R ** 3 + 31) // 32, dtype=torch.int32, device="cuda")
    X, P, L, T = [], [], [], []
    for i in range(n_poses):
        ia.ia_update_occupancy(ctx, i, ia.IA_OCC_POSE, None, bits)
        x = torch.from_numpy(occupied_points(bits.cpu().numpy().view(np.uint32), sc, per_pose, rng)).cuda()
        lab = torch.zeros(per_pose, dtype=torch.int32, device="cuda")
        off = torch.zeros(per_pose, 3, device="cuda")
        ia.ia_proposal_pairs(ctx, i, x, lab, off)
        X.append(x); P.append(torch.full((per_pose,), i, dtype=torch.int32, device="cuda"))
        L.append(lab); T.append(off)
    X, P, L, T = (torch.cat(a) for a in (X, P, L, T))
    keep = torch.nonzero(L >= 0).squeeze(1)
    perm = keep[torch.from_numpy(rng.permutation(len(keep))).cuda()]
    X, P, L, T = (a[perm].contiguous() for a in (X, P, L, T))
    losses = torch.zeros(steps, device="cuda")
    t = time.perf_counter()
    ia.ia_proposal_train(ctx, X, P, L, T, steps, batch, lr, losses)
    torch.cuda.synchronize()
    ls = losses.cpu().numpy()
    return {"pairs": int(len(perm)), "poses": n_poses, "steps": steps, "batch": batch,
            "train_s": round(time.perf_counter() - t, 3), "loss_first": round(float(ls[0]), 4),
            "loss_last": round(float(ls[-50:].mean()), 4)}


def time_frames(torch, ia, ctx, poses, icam, rgb, alpha, flush, steps, warmup, stream):
    """Per step: pose + occupancy refresh + render; CUDA events on the stream,
    L2 flushed before each step outside the events."""
    def step(i):
        th, tr = poses[i % len(poses)]
        ia.ia_set_pose(ctx, th[None], tr[None], stream=stream)
        ia.ia_update_occupancy(ctx, 0, ia.IA_OCC_POSE, stream=stream)
        ia.ia_render(ctx, 0, icam, rgb, alpha, stream=stream)

    for i in range(warmup):
        step(i)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for i in range(steps):
        flush.zero_()
        a, b, c = ev[i]
        th, tr = poses[i % len(poses)]
        a.record(stream)
        ia.ia_set_pose(ctx, th[None], tr[None], stream=stream)
        ia.ia_update_occupancy(ctx, 0, ia.IA_OCC_POSE, stream=stream)
        b.record(stream)
        ia.ia_render(ctx, 0, icam, rgb, alpha, stream=stream)
        c.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(c) for a, b, c in ev], [b.elapsed_time(c) for a, b, c in ev]


def time_occupancy(torch, ia, ctx, poses, flush, steps, stream, cull):
    """ia_update_occupancy alone (with culling on or off): mean ms per pose, CUDA
    events on the stream, L2 flushed before each call outside the events."""
    ia.ia_set_occupancy_culling(ctx, cull)
    ms = []
    for i in range(3 + steps):
        th, tr = poses[i % len(poses)]
        ia.ia_set_pose(ctx, th[None], tr[None], stream=stream)
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ia.ia_update_occupancy(ctx, 0, ia.IA_OCC_POSE, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        if i >= 3:
            ms.append(a.elapsed_time(b))
    ia.ia_set_occupancy_culling(ctx, True)
    return statistics.mean(ms)


def frame_stats(ia, ctx, poses, icam, rgb, alpha):
    tot, occ = {}, {}
    for th, tr in poses:
        ia.ia_set_pose(ctx, th[None], tr[None])
        o = ia.ia_update_occupancy(ctx, 0, ia.IA_OCC_POSE, stats=True)
        r = ia.ia_render(ctx, 0, icam, rgb, alpha, stats=True)
        for k, v in r.items():
            tot[k] = tot.get(k, 0) + v
        for k, v in o.items():
            occ[k] = occ.get(k, 0) + v
    n = len(poses)
    return {k: v / n for k, v in tot.items()}, {k: v / n for k, v in occ.items()}


def time_train_step(torch, ia, sc, table, mlp, flush, steps, warmup, stream, n_rays=8192, n_poses=16,
                    precision=0, prop=None):
    """fwd+bwd training step: n_rays random rays over 16 poses, L2 loss, occupancy =
    union of the 16 per-pose grids, no early termination; optimiser excluded.
    prop: (table, packed MLP) device tensors of a trained proposal (fp16 / bf16
    only): the correspondence search starts from its top-2 bones."""
    ctx = make_ctx(__import__("torch"), ia, sc, table, mlp, precision, 0.0)
    poses = [S.make_pose(sc, 200 + i) for i in range(n_poses)]
    ia.ia_set_pose(ctx, np.stack([p[0] for p in poses]), np.stack([p[1] for p in poses]))
    for i in range(n_poses):
        ia.ia_update_occupancy(ctx, i, ia.IA_OCC_UNION)
    if prop is not None:
        pc = S.proposal_config()
        ia.ia_proposal_init(ctx, ia.make_proposal_config(pc["n_levels"], pc["log2_table"], pc["level_res"],
                                                         pc["top_k"], pc["offset_weight"]))
        ia.ia_proposal_set_params(ctx, prop[0], prop[1])
        ia.ia_set_search(ctx, ia.IA_SEARCH_PROPOSAL)
    rb = S.make_ray_batch(sc, n_rays, n_poses, seed=3)
    dev = {k: torch.from_numpy(np.ascontiguousarray(rb[k])).cuda() for k in ("origin", "direction", "pose", "target")}
    nt, nm = ia.ia_param_sizes(ctx)
    g = dict(table=torch.zeros(nt, device="cuda"), mlp=torch.zeros(nm, device="cuda"),
             skin=torch.zeros(sc.skin_res ** 3 * sc.n_bones, device="cuda"),
             bones=torch.zeros(n_poses * sc.n_bones * 12, device="cuda"))
    loss = torch.zeros(1, device="cuda")

    def step():
        loss.zero_()
        ia.ia_train_step(ctx, dev["origin"], dev["direction"], dev["pose"], dev["target"], loss, g,
                         occ_grid=ia.IA_OCC_UNION, stream=stream)

    for _ in range(warmup):
        step()
    ms = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    scale, skipped = ia.ia_loss_scale(ctx)
    st = ia.ia_train_stats(ctx)
    ia.ia_destroy(ctx)
    occ = max(st["occupied_samples"], 1)
    return {"ms": round(statistics.mean(ms), 4), "min_ms": round(min(ms), 4), "rays": n_rays, "poses": n_poses,
            "samples": st["occupied_samples"], "mean_starts_per_sample": round(st["starts"] / occ, 3),
            "mean_broyden_iters_per_sample": round(st["broyden_iters"] / occ, 3),
            "fallback_rate": round(st["fallbacks"] / max(st["proposed"], 1), 4),
            "point_culled_rate": round(st.get("point_culled", 0) / max(st["proposed"], 1), 4),
            "loss_scale": scale, "last_step_skipped": skipped}


def train_quality(torch, ia, sc, table, mlp, prop=None, iters=2000, batch=8192, n_frames=16, eval_every=250,
                  lr=1e-2, start=("scratch",), skip=True, stop_db=None):
    """Time to quality of the whole training loop (Sec. 3.3-3.4) on a synthetic
    video: 16 frames of 540x540 rendered by the library from the fixture field
    (targets: colour and alpha mask), a learner that starts from an untrained
    field (or a seeded perturbation of the fixture), and per iteration: 8192 random pixels of random
    frames, the fp16 step with the loss set (Huber colour, alpha L1, hard
    surface) and the density regulariser on 8192 random points, an Adam step;
    every 16 iterations a training-mode occupancy update from a random frame.
    PSNR of a held-out frame is taken every eval_every iterations (outside the
    timed total).  skip=False is the Table 3 ablation: no occupancy grid (every
    cell occupied, root culling off, so every sample of every ray is searched
    and evaluated, in training and in the evaluation renders), and therefore no
    occupancy-based regulariser and no grid updates.  stop_db: end the run at
    the first evaluation at or above this PSNR."""
    dev = "cuda"
    poses = [S.make_pose(sc, 300 + i) for i in range(n_frames + 1)]  # the last one is held out
    th = np.stack([p[0] for p in poses])
    tr = np.stack([p[1] for p in poses])
    cam = S.make_camera(sc)
    icam = ia.make_camera(cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["width"], cam["height"], cam["c2w"])
    HW = cam["width"] * cam["height"]
    gt = make_ctx(torch, ia, sc, table, mlp, 0, EARLY_T)
    ia.ia_set_pose(gt, th, tr)
    T_rgb = torch.zeros(n_frames + 1, HW, 3, device=dev)
    T_a = torch.zeros(n_frames + 1, HW, device=dev)
    for i in range(n_frames + 1):
        ia.ia_update_occupancy(gt, i)
        ia.ia_render(gt, i, icam, T_rgb[i], T_a[i])
    ia.ia_destroy(gt)
    o_np, d_np = S.pixel_rays(sc)
    O = torch.from_numpy(o_np).to(dev)
    D = torch.from_numpy(d_np).to(dev)
    t0, m0 = S.init_field(sc, 0) if start[0] == "scratch" else S.perturb_field(table, mlp, 0, start[1], start[2])
    ctx = make_ctx(torch, ia, sc, t0, m0, 1, EARLY_T)
    ia.ia_set_pose(ctx, th, tr)
    if prop is not None:
        pc = S.proposal_config()
        ia.ia_proposal_init(ctx, ia.make_proposal_config(pc["n_levels"], pc["log2_table"], pc["level_res"],
                                                         pc["top_k"], pc["offset_weight"]))
        ia.ia_proposal_set_params(ctx, prop[0], prop[1])
        ia.ia_set_search(ctx, ia.IA_SEARCH_PROPOSAL)
    ia.ia_set_loss(ctx, ia.IA_LOSS_HUBER, 0.1, 1.0, 1.0, 0.1)
    R = sc.occ_res
    gen = torch.Generator(device=dev)
    gen.manual_seed(123)
    frame_rng = np.random.default_rng(124)
    full = all_occupied(R)
    if skip:
        for i in range(n_frames):  # the sequence grid from every frame once
            ia.ia_update_occupancy_ema(ctx, i, None, 1.0 if i else 0.0)
        grid = ia.IA_OCC_UNION
    else:
        ia.ia_set_occupancy_culling(ctx, False)
        ia.ia_set_occupancy(ctx, full)
        grid = ia.IA_OCC_POSE
    reg_w = 0.1 if skip else 0.0
    nt, nm = ia.ia_param_sizes(ctx)
    ns, nbn = ia.ia_grad_sizes(ctx)
    g = dict(table=torch.zeros(nt, device=dev), mlp=torch.zeros(nm, device=dev), skin=torch.zeros(ns, device=dev),
             bones=torch.zeros(nbn, device=dev))
    loss = torch.zeros(1, device=dev)
    eval_rgb = torch.zeros(HW, 3, device=dev)
    eval_a = torch.zeros(HW, device=dev)
    nmin = torch.from_numpy(sc.norm_min.astype(np.float32)).to(dev)
    ext = torch.from_numpy((sc.norm_max - sc.norm_min).astype(np.float32)).to(dev)

    def psnr():
        if skip:
            ia.ia_update_occupancy(ctx, n_frames)
        else:
            ia.ia_set_occupancy(ctx, full)
        ia.ia_render(ctx, n_frames, icam, eval_rgb, eval_a)
        mse = torch.mean((eval_rgb - T_rgb[n_frames]) ** 2).item()
        return float(10 * np.log10(1.0 / max(mse, 1e-12)))

    curve = [(0, 0.0, round(psnr(), 3))]
    # one untimed step first: the workspaces are allocated on the first call
    f = torch.randint(0, n_frames, (batch,), device=dev, dtype=torch.int32)
    px = torch.randint(0, HW, (batch,), device=dev)
    ia.ia_train_step(ctx, O[px].contiguous(), D[px].contiguous(), f, T_rgb[f.long(), px].contiguous(), loss, g,
                     occ_grid=grid, alpha_target=T_a[f.long(), px].contiguous(),
                     reg_x=(nmin + ext * torch.rand(batch, 3, device=dev)).contiguous(), reg_pose=f, reg_weight=reg_w)
    torch.cuda.synchronize()
    timed = 0.0
    skips = 0
    losses = []
    for it in range(1, iters + 1):
        torch.cuda.synchronize()
        t = time.perf_counter()
        f = torch.randint(0, n_frames, (batch,), device=dev, generator=gen, dtype=torch.int32)
        px = torch.randint(0, HW, (batch,), device=dev, generator=gen)
        rx = nmin + ext * torch.rand(batch, 3, device=dev, generator=gen)
        rp = torch.randint(0, n_frames, (batch,), device=dev, generator=gen, dtype=torch.int32)
        loss.zero_()
        ia.ia_train_step(ctx, O[px].contiguous(), D[px].contiguous(), f, T_rgb[f.long(), px].contiguous(), loss, g,
                         occ_grid=grid, alpha_target=T_a[f.long(), px].contiguous(), reg_x=rx.contiguous(),
                         reg_pose=rp, reg_weight=reg_w)
        ia.ia_adam_step(ctx, g["table"], g["mlp"], lr, 0.9, 0.99, 1e-15)
        if skip and it % 16 == 0:
            jit = torch.rand(R ** 3, 3, device=dev, generator=gen)
            ia.ia_update_occupancy_ema(ctx, int(frame_rng.integers(0, n_frames)), jit, 0.95)
        torch.cuda.synchronize()
        timed += time.perf_counter() - t
        if it % 50 == 0:
            losses.append(round(loss.item(), 5))
            scale, skipped = ia.ia_loss_scale(ctx)
            skips += int(skipped)
        if it % eval_every == 0 or it == iters:
            curve.append((it, round(timed, 3), round(psnr(), 3)))
            if stop_db is not None and curve[-1][2] >= stop_db:
                break
    ia.ia_destroy(ctx)
    reach = {}
    for db in (30, 40, 50):
        hit = [c for c in curve if c[2] >= db]
        reach[f"{db}dB"] = {"iteration": hit[0][0], "seconds": hit[0][1]} if hit else None
    done = curve[-1][0]
    return {"iterations": done, "batch_rays": batch, "frames": n_frames, "seconds": round(timed, 3),
            "skipping": skip, "time_to_psnr": reach,
            "iters_per_s": round(done / timed, 1), "psnr_curve": curve, "loss_every_50": losses[:8] + losses[-4:],
            "psnr_start": curve[0][2], "psnr_end": curve[-1][2], "start": list(start),
            "skipped_steps_seen": skips,
            "what": "fp16 step (+proposal) with Huber/alpha/hard losses and the density regulariser, Adam, "
                    "training-mode occupancy every 16 iterations; PSNR on a held-out frame"}


def all_occupied(R):
    """Packed occupancy bits with every cell occupied."""
    full = np.full((R ** 3 + 31) // 32, 0xFFFFFFFF, dtype=np.uint32)
    if R ** 3 % 32:
        full[-1] = (1 << (R ** 3 % 32)) - 1
    return full


def skip_ablation(torch, ia, sc, table, mlp, icam, rgb, alpha, stream, poses, frames=10):
    """Empty-space skipping on and off (the Table 3 analogue): plain fp32 render
    of a frame with the pose's occupancy grid (and root culling) against an
    all-occupied grid with root culling off, and a fp32 training step (8192 rays,
    16 poses) on the union grid (and root culling) against an all-occupied grid
    with root culling off: 'off' searches every sample."""
    ctx = make_ctx(torch, ia, sc, table, mlp, 0, EARLY_T)
    full = all_occupied(sc.occ_res)
    out = {"frames": frames}
    for name, skip in (("skip", True), ("no_skip", False)):
        ia.ia_set_occupancy_culling(ctx, skip)
        ms = []
        for th, tr in poses[:frames]:
            ia.ia_set_pose(ctx, th[None], tr[None])
            if skip:
                ia.ia_update_occupancy(ctx, 0)
            else:
                ia.ia_set_occupancy(ctx, full)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ia.ia_render(ctx, 0, icam, rgb, alpha, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        out[f"render_ms_{name}"] = round(statistics.mean(ms), 3)
    ia.ia_destroy(ctx)
    # training step: union grid vs all occupied (IA_OCC_POSE carrying the full grid)
    ctx = make_ctx(torch, ia, sc, table, mlp, 0, 0.0)
    tposes = [S.make_pose(sc, 200 + i) for i in range(16)]
    ia.ia_set_pose(ctx, np.stack([p[0] for p in tposes]), np.stack([p[1] for p in tposes]))
    for i in range(16):
        ia.ia_update_occupancy(ctx, i, ia.IA_OCC_UNION)
    ia.ia_set_occupancy(ctx, full)
    rb = S.make_ray_batch(sc, 8192, 16, seed=3)
    dev = {k: torch.from_numpy(np.ascontiguousarray(rb[k])).cuda() for k in ("origin", "direction", "pose", "target")}
    nt, nm = ia.ia_param_sizes(ctx)
    ns, nbn = ia.ia_grad_sizes(ctx)
    g = dict(table=torch.zeros(nt, device="cuda"), mlp=torch.zeros(nm, device="cuda"),
             skin=torch.zeros(ns, device="cuda"), bones=torch.zeros(nbn, device="cuda"))
    loss = torch.zeros(1, device="cuda")
    for name, grid in (("skip", ia.IA_OCC_UNION), ("no_skip", ia.IA_OCC_POSE)):
        ia.ia_set_occupancy_culling(ctx, grid == ia.IA_OCC_UNION)
        ms = []
        for it in range(11):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ia.ia_train_step(ctx, dev["origin"], dev["direction"], dev["pose"], dev["target"], loss, g, occ_grid=grid,
                             stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            if it:
                ms.append(a.elapsed_time(b))
        out[f"train_step_ms_{name}"] = round(statistics.mean(ms), 3)
    ia.ia_destroy(ctx)
    out["render_speedup"] = round(out["render_ms_no_skip"] / out["render_ms_skip"], 2)
    out["train_speedup"] = round(out["train_step_ms_no_skip"] / out["train_step_ms_skip"], 2)
    return out


def table_entries(level_res, log2_table):
    """Entries of a hash table (the documented storage: dense levels (res + 1)^3,
    hashed levels 2^log2_table)."""
    T = 1 << log2_table
    return sum(min((int(r) + 1) ** 3, T) for r in level_res)


def gather_peaks(torch, ia, stream, num_sms, hash_entries=None, prop_entries=None, skin_floats=None):
    """Random-record rates of the library's probes, useful GB/s, best of 5 launches:
    48-byte gathers (ia_gather_probe) from a 64 KiB table (l1, L1 resident) and
    from a table the size of one blended grid, 64^3 vertices (l2, 12.6 MB, L2
    resident); with the sizes given, 4- and 8-byte gathers from tables of the
    field's hash-table entries (hash4: the fp16 shadow, hash8: fp32) and of the
    proposal's (prop8), 8-byte vector atomics on the field's table (atomic8: the
    hash-gradient scatter) and 16-byte ones on a skinning-grid-sized table
    (atomic16: the implicit gradient's scatter)."""
    out = {}
    sink = torch.zeros(1, device="cuda")
    blocks = num_sms * 8

    def best_of(run, nbytes):
        run(8)  # warm-up
        best = 0.0
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            run(640)
            b.record(stream)
            torch.cuda.synchronize()
            best = max(best, blocks * 256 * 640 * nbytes / (a.elapsed_time(b) * 1e-3) / 1e9)
        return round(best, 1)

    gathers = [("l1", 65536 // 48, 48), ("l2", 64 ** 3, 48)]
    if hash_entries:
        gathers += [("hash4", hash_entries, 4), ("hash8", hash_entries, 8)]
    if prop_entries:
        gathers += [("prop8", prop_entries, 8)]
    for name, n_rec, rb in gathers:
        table = torch.rand(n_rec * rb // 4, device="cuda")
        out[name] = best_of(lambda it: ia.ia_gather_probe(table, n_rec, it, blocks, sink, stream=stream,
                                                          record_bytes=rb), rb)
        del table
    atomics = []
    if hash_entries:
        atomics.append(("atomic8", hash_entries, 8))
    if skin_floats:
        atomics.append(("atomic16", skin_floats // 4, 16))
    for name, n_rec, rb in atomics:
        table = torch.zeros(n_rec * rb // 4, device="cuda")
        out[name] = best_of(lambda it: ia.ia_atomic_probe(table, n_rec, it, blocks, stream=stream,
                                                          record_bytes=rb), rb)
        del table
    return out


# ------------------------------------------------------------------ per-kernel measurement

def profile_frames(ia, ctx, poses, icam, rgb, alpha, frames):
    """Per-kernel device times (library launch tracing: CUDA events around each
    launch on its stream) over `frames` animated frames (pose + occupancy
    refresh + render): {kernel: (launches per frame, ms per launch)}."""
    import torch
    torch.cuda.synchronize()
    ia.ia_profile_begin()
    for i in range(frames):
        th, tr = poses[i % len(poses)]
        ia.ia_set_pose(ctx, th[None], tr[None])
        ia.ia_update_occupancy(ctx, 0, ia.IA_OCC_POSE)
        ia.ia_render(ctx, 0, icam, rgb, alpha)
    prof = ia.ia_profile_end()
    return {k: (n / frames, tot / n) for k, (n, tot, _) in prof.items()}


def profile_train(torch, ia, sc, table, mlp, steps, n_rays, precision, prop=None):
    """Per-kernel device times of the training step (as time_train_step sets it
    up) and its counters: ({kernel: (launches per step, ms per launch)}, stats)."""
    ctx = make_ctx(torch, ia, sc, table, mlp, precision, 0.0)
    poses = [S.make_pose(sc, 200 + i) for i in range(16)]
    ia.ia_set_pose(ctx, np.stack([p[0] for p in poses]), np.stack([p[1] for p in poses]))
    for i in range(16):
        ia.ia_update_occupancy(ctx, i, ia.IA_OCC_UNION)
    if prop is not None:
        pc = S.proposal_config()
        ia.ia_proposal_init(ctx, ia.make_proposal_config(pc["n_levels"], pc["log2_table"], pc["level_res"],
                                                         pc["top_k"], pc["offset_weight"]))
        ia.ia_proposal_set_params(ctx, prop[0], prop[1])
        ia.ia_set_search(ctx, ia.IA_SEARCH_PROPOSAL)
    rb = S.make_ray_batch(sc, n_rays, 16, seed=3)
    dev = {k: torch.from_numpy(np.ascontiguousarray(rb[k])).cuda() for k in ("origin", "direction", "pose", "target")}
    nt, nm = ia.ia_param_sizes(ctx)
    ns, nbn = ia.ia_grad_sizes(ctx)
    g = dict(table=torch.zeros(nt, device="cuda"), mlp=torch.zeros(nm, device="cuda"),
             skin=torch.zeros(ns, device="cuda"), bones=torch.zeros(nbn, device="cuda"))
    loss = torch.zeros(1, device="cuda")
    for _ in range(2):  # workspaces and culling masks
        ia.ia_train_step(ctx, dev["origin"], dev["direction"], dev["pose"], dev["target"], loss, g,
                         occ_grid=ia.IA_OCC_UNION)
    torch.cuda.synchronize()
    ia.ia_profile_begin()
    for _ in range(steps):
        ia.ia_train_step(ctx, dev["origin"], dev["direction"], dev["pose"], dev["target"], loss, g,
                         occ_grid=ia.IA_OCC_UNION)
    prof = ia.ia_profile_end()
    st = ia.ia_train_stats(ctx)
    ia.ia_destroy(ctx)
    return {k: (n / steps, tot / n) for k, (n, tot, _) in prof.items()}, st


def lbs_residual(sc, N, x_canon, x_posed):
    """|LBS(x*) - x'| in fp64 for canonical points x* [n, 3] and their posed
    points x' [n, 3] (normalised space): trilinear skinning weights of the grid
    (vertices at the canonical box's corners, clamped to the border), the
    pose's fp32 transforms N [nb, 3, 4] as the library stores them."""
    R = sc.skin_res
    W = sc.skin_grid.reshape(R, R, R, sc.n_bones).astype(np.float64)
    lo, hi = sc.canon_min.astype(np.float64), sc.canon_max.astype(np.float64)
    u = np.clip((x_canon - lo) / (hi - lo) * (R - 1), 0, R - 1)
    i0 = np.minimum(np.floor(u).astype(np.int64), R - 2)
    f = u - i0
    w = np.zeros((len(x_canon), sc.n_bones))
    for c in range(8):
        d = np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1])
        wt = np.prod(np.where(d, f, 1 - f), axis=1)
        v = i0 + d
        w += wt[:, None] * W[v[:, 2], v[:, 1], v[:, 0]]
    xh = np.concatenate([x_canon, np.ones((len(x_canon), 1))], axis=1)
    y = np.einsum("nb,bij,nj->ni", w, N.astype(np.float64), xh)
    return np.linalg.norm(y - x_posed, axis=1)


def residual_stats(torch, ia, sc, ctx_plain, ctx_prop, pose, n=32768):
    """Correspondence residual and colour of the selected roots of both searches
    at the same posed points (uniform in the occupied cells of the pose's grid):
    LBS residual of each path's roots, their distance, and the colour and
    density differences between the paths."""
    th, tr = pose
    R = sc.occ_res
    bits = torch.zeros((R ** 3 + 31) // 32, dtype=torch.int32, device="cuda")
    out = {}
    for name, ctx in (("fp32_plain", ctx_plain), ("fp16_proposal", ctx_prop)):
        ia.ia_set_pose(ctx, th[None], tr[None])
        ia.ia_update_occupancy(ctx, 0, ia.IA_OCC_POSE, None, bits)
        if name == "fp32_plain":
            x = occupied_points(bits.cpu().numpy().view(np.uint32), sc, n, np.random.default_rng(99))
            xd = torch.from_numpy(x).cuda()
            N = np.zeros((sc.n_bones, 12), np.float32)
            ia.ia_get_transforms(ctx, 0, N)
        sig, rgb, xc = (torch.zeros(n, device="cuda"), torch.zeros(n, 3, device="cuda"),
                        torch.zeros(n, 3, device="cuda"))
        start = torch.zeros(n, dtype=torch.int32, device="cuda")
        ia.ia_query_posed(ctx, 0, xd, sig, rgb, xc, start)
        torch.cuda.synchronize()
        out[name] = dict(sigma=sig.cpu().numpy(), rgb=rgb.cpu().numpy(), xc=xc.cpu().numpy().astype(np.float64),
                         has=start.cpu().numpy() >= 0)
    a, b = out["fp32_plain"], out["fp16_proposal"]
    both = a["has"] & b["has"]
    res = {}
    for name, o in out.items():
        r = lbs_residual(sc, N.reshape(-1, 3, 4), o["xc"][o["has"]], x.astype(np.float64)[o["has"]])
        res[name] = {"mean": float(r.mean()), "max": float(r.max()), "p99": float(np.quantile(r, 0.99)),
                     "with_root": int(o["has"].sum())}
    dx = np.linalg.norm(a["xc"][both] - b["xc"][both], axis=1)
    drgb = np.abs(a["rgb"][both] - b["rgb"][both]).max(axis=1)
    return {"points": n, "lbs_residual_m": res, "root_presence_differs": int((a["has"] != b["has"]).sum()),
            "root_distance_m": {"mean": float(dx.mean()), "p99": float(np.quantile(dx, 0.99)), "max": float(dx.max()),
                                "over_1e-4": int((dx > 1e-4).sum())},
            "colour_abs_diff": {"mean": float(drgb.mean()), "p99": float(np.quantile(drgb, 0.99))},
            "what": "posed points uniform in the occupied cells of one pose's grid; selected roots of the plain "
                    "fp32 24-start search and of the fp16 + proposal search (ia_query_posed), residual "
                    "|LBS(x*) - x'| in fp64 with the stored fp32 transforms"}


def roofline_entry(kernel, bound, work, unit_work, ms, peak, peak_unit, peak_source, what):
    """work per launch (bytes or FLOPs) over the measured launch time, against a peak."""
    achieved = work / (ms * 1e-3) / (1e9 if peak_unit == "GB/s" else 1e12)
    return {"kernel": kernel, "bound": bound, "achieved": round(achieved, 2), "peak": round(peak, 2),
            "unit": peak_unit, "frac": round(achieved / peak, 4), "work_per_launch": round(work),
            "work_unit": unit_work, "ms_per_launch": round(ms, 4), "peak_source": peak_source, "work": what}


def frame_gather_bytes(st, hash_bytes, prop=False):
    """Algorithmic gather bytes of a posed-field pass from its counters: one LBS
    evaluation per start and Broyden step, per distinct root its polish (one
    more LBS) and hash encoding, per proposed sample the proposal's encoding."""
    b = GATHER_LBS * (st["starts"] + st["broyden_iters"]) + (GATHER_LBS + hash_bytes) * st["roots"]
    return b + (GATHER_PROP * st["proposed"] if prop else 0)




def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2212_10550_b300 as ia

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    sc = S.make_scene("full", 0)
    table, mlp = S.make_field(sc, 0)
    poses = [S.make_pose(sc, (rank * N_POSES + i) % 1024) for i in range(N_POSES)]
    cam = S.make_camera(sc)
    icam = ia.make_camera(cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["width"], cam["height"], cam["c2w"])
    W, H = cam["width"], cam["height"]
    rgb = torch.zeros(W * H, 3, device=dev)
    alpha = torch.zeros(W * H, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    if args.only == "proposal":
        ctx16 = make_ctx(torch, ia, sc, table, mlp, 1, EARLY_T)
        pt = train_proposal(torch, ia, ctx16, sc, n_poses=64, steps=400)
        ia.ia_set_search(ctx16, ia.IA_SEARCH_PROPOSAL)
        step16, render16 = time_frames(torch, ia, ctx16, poses, icam, rgb, alpha, flush, args.steps, args.warmup,
                                       stream)
        ia.ia_destroy(ctx16)
        if rank != 0:
            return None
        return {"metric": METRIC, "partial": "fp16 + proposal frames only (proposal trained on 64 poses)",
                "ms_per_step": round(statistics.mean(step16), 4), "render_ms": round(statistics.mean(render16), 4),
                "proposal_training": pt}

    if args.only == "ablation":
        ab = skip_ablation(torch, ia, sc, table, mlp, icam, rgb, alpha, stream, poses)
        return {"metric": METRIC, "partial": "skip ablation only", "skip_ablation": ab} if rank == 0 else None

    if args.only == "profile":
        # per-kernel launch times of the frames and train steps (launch tracing), short
        ctx = make_ctx(torch, ia, sc, table, mlp, 0, EARLY_T)
        frame_stats(ia, ctx, poses[:2], icam, rgb, alpha)
        pf = profile_frames(ia, ctx, poses, icam, rgb, alpha, max(4, args.steps))
        ia.ia_destroy(ctx)
        ctx16 = make_ctx(torch, ia, sc, table, mlp, 1, EARLY_T)
        pt = train_proposal(torch, ia, ctx16, sc, n_poses=64, steps=400)
        ia.ia_set_search(ctx16, ia.IA_SEARCH_PROPOSAL)
        frame_stats(ia, ctx16, poses[:2], icam, rgb, alpha)
        pf16 = profile_frames(ia, ctx16, poses, icam, rgb, alpha, max(4, args.steps))
        pnt, pnm = ia.ia_proposal_param_sizes(ctx16)
        pp = (torch.zeros(pnt, device=dev), torch.zeros(pnm, device=dev))
        ia.ia_proposal_get_params(ctx16, *pp)
        ia.ia_destroy(ctx16)
        tr = {n: profile_train(torch, ia, sc, table, mlp, 5, 32768, prec, q)[0]
              for n, prec, q in (("fp32", 0, None), ("fp16", 1, None), ("fp16_proposal", 1, pp))}
        if rank != 0:
            return None
        fmt = lambda d: {k: [round(n, 2), round(ms, 4)] for k, (n, ms) in d.items()}  # noqa: E731
        return {"metric": METRIC, "partial": "per-kernel launch times ([launches per unit, ms per launch])",
                "frame_fp32": fmt(pf), "frame_fp16_proposal": fmt(pf16),
                "train_step_32768": {n: fmt(d) for n, d in tr.items()}, "proposal_training": pt}

    if args.only == "quality":
        q = train_quality(torch, ia, sc, table, mlp, None, iters=max(50, args.steps), eval_every=100)
        q_off = train_quality(torch, ia, sc, table, mlp, None, iters=max(50, args.steps), eval_every=100, skip=False,
                              stop_db=50.0)
        return ({"metric": METRIC, "partial": "training quality only", "train_quality": q,
                 "train_quality_no_skip": q_off} if rank == 0 else None)


    if args.only == "train":
        tsteps = max(3, args.steps)
        res = {name: time_train_step(torch, ia, sc, table, mlp, flush, tsteps, args.warmup, stream,
                                     n_rays=args.train_rays, precision=prec) for name, prec in (("fp32", 0), ("fp16", 1))}
        if rank != 0:
            return None
        return {"metric": METRIC, "value": res["fp16"]["ms"], "unit": f"ms per fp16 training step ({args.train_rays} rays)",
                "n_gpus": world, "steps": tsteps, "warmup": args.warmup, "higher_is_better": False,
                "train_step_32768": res, "partial": "training steps only"}

    # ---- plain fp32 multi-start (the headline workload)
    ctx = make_ctx(torch, ia, sc, table, mlp, 0, EARLY_T)
    per_frame, occ_per_frame = frame_stats(ia, ctx, poses, icam, rgb, alpha)
    ref_rgb = []
    for th, tr in poses[:4]:
        ia.ia_set_pose(ctx, th[None], tr[None])
        ia.ia_update_occupancy(ctx, 0)
        ia.ia_render(ctx, 0, icam, rgb, alpha)
        ref_rgb.append((rgb.clone(), alpha.clone()))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    t0 = time.perf_counter()
    step_ms, render_ms = time_frames(torch, ia, ctx, poses, icam, rgb, alpha, flush, args.steps, args.warmup,
                                     stream)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    local_total_s = sum(step_ms) / 1e3
    prof_plain = profile_frames(ia, ctx, poses, icam, rgb, alpha, 8)

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
    occ_cull_ms = time_occupancy(torch, ia, ctx, poses, flush, 16, stream, True)
    occ_full_ms = time_occupancy(torch, ia, ctx, poses, flush, 16, stream, False)

    if args.only == "plain":
        ia.ia_destroy(ctx)
        total = sum(step_ms) / 1e3
        if rank == 0:
            return {"metric": METRIC, "value": round(args.steps / total, 3), "unit": "frames/s",
                    "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                    "ms_per_step": round(1e3 * total / args.steps, 4), "higher_is_better": True,
                    "render_ms": round(statistics.mean(render_ms), 4),
                    "kernels_per_frame": {k: [round(n, 2), round(ms, 4)] for k, (n, ms) in prof_plain.items()},
                    "occupancy_refresh": {"culled_ms": round(occ_cull_ms, 4), "full_search_ms": round(occ_full_ms, 4)},
                    "partial": "plain fp32 frames only"}
        return None

    # ---- fp16 + learned proposal on the same sequence (proposal trained on other poses)
    ctx16 = make_ctx(torch, ia, sc, table, mlp, 1, EARLY_T)
    prop_train = train_proposal(torch, ia, ctx16, sc)
    ia.ia_set_search(ctx16, ia.IA_SEARCH_PROPOSAL)
    per_frame16, occ16 = frame_stats(ia, ctx16, poses, icam, rgb, alpha)
    differ = hit = 0
    for (th, tr), (r0, a0) in zip(poses[:4], ref_rgb):
        ia.ia_set_pose(ctx16, th[None], tr[None])
        ia.ia_update_occupancy(ctx16, 0)
        ia.ia_render(ctx16, 0, icam, rgb, alpha)
        torch.cuda.synchronize()
        d = ((rgb - r0).abs() > 2e-3 * r0.abs() + 2e-4).any(dim=1) | ((alpha - a0).abs() > 2e-3 * a0.abs() + 2e-4)
        differ += int(d.sum().item())
        hit += int((a0 > 0).sum().item())
    step16, render16 = time_frames(torch, ia, ctx16, poses, icam, rgb, alpha, flush, args.steps, args.warmup,
                                   stream)
    prof16 = profile_frames(ia, ctx16, poses, icam, rgb, alpha, 8)
    residual = residual_stats(torch, ia, sc, ctx, ctx16, poses[1])
    pnt, pnm = ia.ia_proposal_param_sizes(ctx16)
    prop_params = (torch.zeros(pnt, device=dev), torch.zeros(pnm, device=dev))
    ia.ia_proposal_get_params(ctx16, *prop_params)
    ia.ia_destroy(ctx16)
    ia.ia_destroy(ctx)

    # ---- fwd+bwd training steps: fp32 at 8192 rays; fp32 / fp16 / bf16 / fp16+proposal at 32768 rays
    tsteps = max(5, args.steps // 10)
    train = {"fp32_8192": time_train_step(torch, ia, sc, table, mlp, flush, tsteps, 3, stream)}
    for name, prec, pp in (("fp32", 0, None), ("fp16", 1, None), ("bf16", 2, None), ("fp16_proposal", 1, prop_params)):
        train[name] = time_train_step(torch, ia, sc, table, mlp, flush, tsteps, 3, stream, n_rays=32768,
                                      precision=prec, prop=pp)
    prof_train = {name: profile_train(torch, ia, sc, table, mlp, 5, 32768, prec, pp)
                  for name, prec, pp in (("fp32", 0, None), ("fp16_proposal", 1, prop_params))}
    quality = train_quality(torch, ia, sc, table, mlp, prop_params, iters=2000, eval_every=100)
    quality_off = train_quality(torch, ia, sc, table, mlp, prop_params, iters=1000, eval_every=100, skip=False,
                                stop_db=50.0)
    ablation = skip_ablation(torch, ia, sc, table, mlp, icam, rgb, alpha, stream, poses)
    ablation["train_time_to_psnr"] = {"skip": quality["time_to_psnr"], "no_skip": quality_off["time_to_psnr"],
                                      "no_skip_curve": quality_off["psnr_curve"],
                                      "no_skip_iters_per_s": quality_off["iters_per_s"]}
    ablation["train_time_ratio"] = {
        db: (round(quality_off["time_to_psnr"][db]["seconds"] / quality["time_to_psnr"][db]["seconds"], 2)
             if quality_off["time_to_psnr"][db] and quality["time_to_psnr"][db] else None)
        for db in ("30dB", "40dB", "50dB")}

    fps, total_s = job_rate(args.steps, local_total_s, world, dev)
    if rank != 0:
        return None
    ms_per_step = 1e3 * total_s / args.steps
    peaks, peak_kind = load_peaks()
    sm_mhz = peaks.get("sm_max_mhz", 2032.0)
    peak = fp32_peak_tflops(sm_mhz)
    r_ms = statistics.mean(render_ms)
    r16_ms = statistics.mean(render16)
    pcfg = S.proposal_config()
    peaks_g = gather_peaks(torch, ia, stream, torch.cuda.get_device_properties(0).multi_processor_count,
                           hash_entries=sc.n_table_entries(),
                           prop_entries=table_entries(pcfg["level_res"], pcfg["log2_table"]),
                           skin_floats=sc.skin_res ** 3 * sc.n_bones)
    hash_src = ("ia_gather_probe: random {b}-byte records from a table of the field's {n:,} hash entries "
                "({mb:.1f} MB), measured in this run")
    prop_src = "ia_gather_probe: random 8-byte records from a table of the proposal's hash entries, measured in this run"
    l1_src = "ia_gather_probe: random 48-byte records from a 64 KiB table (L1), measured in this run"
    hbm = peaks.get("hbm_gbs", 6400.0)
    hbm_src = f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else \
        "fallback HBM figure"
    tc = peaks.get("bf16_tflops", 1800.0)
    # ---- the dominant kernel of the plain fp32 frame: the correspondence search
    search_bytes = GATHER_LBS * (per_frame["starts"] + per_frame["broyden_iters"])
    s_ms = prof_plain["wf_search_kernel"][1]
    s_achieved = search_bytes / (s_ms * 1e-3) / 1e9
    # the gathers actually issued: an evaluation in the cell of the item's previous one reuses its records
    issued_bytes = GATHER_LBS * per_frame.get("grid_gathers", 0)
    roofline_gather = {"kernel": "wf_search_kernel", "bound": "l1-gather", "achieved": round(s_achieved, 1),
                       "peak": peaks_g["l1"], "unit": "GB/s", "frac": round(s_achieved / peaks_g["l1"], 4),
                       "traffic": None, "bytes_per_launch": round(search_bytes), "ms_per_launch": round(s_ms, 4),
                       "peak_l2_random": peaks_g["l2"], "peak_source": l1_src,
                       "work": "48 B x 8 corners per LBS evaluation x (starts + Broyden steps) of the frame",
                       "gathered_bytes_per_launch": round(issued_bytes),
                       "gathered_frac": round(issued_bytes / (s_ms * 1e-3) / 1e9 / peaks_g["l1"], 4),
                       "gathered_note": "the gathers issued: evaluations in the cell of the item's previous "
                                        "evaluation reuse the corner records it holds in registers",
                       "traffic_note": "DRAM bytes per launch come from an ncu capture, not from this run"}
    # ---- the whole render (all its kernels) against the same gather peak
    render_roofline = {}
    for name, st, hb, pr, ms in (("fp32", per_frame, GATHER_HASH, False, r_ms),
                                 ("fp16_proposal", per_frame16, GATHER_HASH_H, True, r16_ms)):
        gb = frame_gather_bytes(st, hb, pr)
        ach = gb / (ms * 1e-3) / 1e9
        render_roofline[name] = {"bound": "l1-gather", "achieved": round(ach, 1), "peak": peaks_g["l1"],
                                 "unit": "GB/s", "frac": round(ach / peaks_g["l1"], 4), "bytes_per_frame": round(gb),
                                 "render_ms": round(ms, 4)}
    render_roofline["what"] = ("ia_render's algorithmic gather bytes (search, polish, hash encoding, proposal "
                               "encoding) over its CUDA-event time, all its kernels and the sample-count read-back")
    # ---- fp32 field kernel: polish + hash encoding + per-lane fp32 MLP per root
    f_ms = prof_plain["wf_field_kernel<fp32>"][1]
    flop_field = FLOP_ROOT * per_frame["roots"]
    achieved = flop_field / (f_ms * 1e-3) / 1e12
    # ---- per-kernel rooflines: work per launch from the counters, time per launch from launch tracing
    kern = {}

    def add(name, prof, bound, work, unit_work, pk, pk_unit, pk_src, what):
        if name in prof:
            kern[name] = roofline_entry(name, bound, work, unit_work, prof[name][1], pk, pk_unit, pk_src, what)

    def wavefront(prof, st, hash_b, prop, tag, label):
        """Rooflines of the wavefront kernels of one caller (tag: the launch-name
        suffix, "" for the render): the search (both waves summed when the
        proposal runs; the counters do not split them), the field and the
        proposal network."""
        def mine(k, base):
            return k.startswith(base) and (k.endswith(tag) if tag else "[" not in k)

        sk = [k for k in prof if mine(k, "wf_search_kernel")]
        if sk:
            kern[f"wf_search_kernel ({label})"] = roofline_entry(
                " + ".join(sk), "l1-gather", GATHER_LBS * (st["starts"] + st["broyden_iters"]), "B",
                sum(prof[k][1] * prof[k][0] for k in sk), peaks_g["l1"], "GB/s", l1_src,
                "48 B x 8 corners x (starts + Broyden steps); time: all its launches per frame (step)")
        fk = [k for k in prof if mine(k, "wf_field_kernel")]
        if fk:
            rb = hash_b // 128  # bytes of one hash entry: 8 (fp32) or 4 (fp16 shadow)
            kern[f"{fk[0]} ({label})"] = roofline_entry(
                fk[0], "hash-gather", hash_b * st["roots"], "B", prof[fk[0]][1] * prof[fk[0]][0],
                peaks_g[f"hash{rb}"], "GB/s",
                hash_src.format(b=rb, n=sc.n_table_entries(), mb=sc.n_table_entries() * rb / 1e6),
                f"per distinct root: {hash_b} B of hash gathers (16 levels x 8 corners x {rb} B); the polish's "
                "8 x 48 B blended-grid gathers, the merge and the MLP run in the same time and are not counted")
        pk = [k for k in prof if mine(k, "wf_propose_kernel")]
        if pk and prop:
            kern[f"{pk[0]} ({label})"] = roofline_entry(
                pk[0], "hash-gather", GATHER_PROP * st["proposed"], "B", prof[pk[0]][1] * prof[pk[0]][0],
                peaks_g["prop8"], "GB/s", prop_src,
                "512 B of proposal-encoding gathers per sample (8 levels x 8 corners x 8 B); its network "
                "runs in the same time and is not counted")

    wavefront(prof_plain, per_frame, GATHER_HASH, False, "", "render, fp32")
    wavefront(prof16, per_frame16, GATHER_HASH_H, True, "", "render, fp16 + proposal")
    wavefront(prof_plain, occ_per_frame, GATHER_HASH, False, " [occupancy]", "occupancy, fp32")
    wavefront(prof16, occ16, GATHER_HASH_H, True, " [occupancy]", "occupancy, fp16 + proposal")
    V = sc.skin_res ** 3
    add("blend_kernel", prof_plain, "hbm", V * sc.n_bones * 4 + V * 48, "B", hbm, "GB/s", hbm_src,
        "skinning grid read (64^3 x 24 fp32) + blended grid written (64^3 x 48 B)")
    for tname, (tp, tst) in prof_train.items():
        searched = tst["occupied_samples"] - tst["culled"]
        hash_b = GATHER_HASH if tname == "fp32" else GATHER_HASH_H
        wavefront(tp, tst, hash_b, tname != "fp32", " [train]", f"{tname} train step, 32768 rays")
        # per searched sample: table read for dL/dx*, hash-gradient atomics, skinning-grid
        # atomics (8 corners x 24 bones), the Jacobian's blended-grid gather, dL/dfeatures and x*
        rooted = tst.get("rooted_samples", 0)
        if "train_hash_grad_kernel" in tp and rooted:
            kern[f"train_hash_grad_kernel ({tname})"] = roofline_entry(
                "train_hash_grad_kernel", "l2-atomic", rooted * 128 * 8, "B", tp["train_hash_grad_kernel"][1],
                peaks_g["atomic8"], "GB/s",
                "ia_atomic_probe: random float2 atomicAdds on a table of the field's hash entries, measured in "
                "this run",
                "per sample with a root: 16 levels x 8 corners float2 atomics into the table gradient; its table "
                "reads for dL/dx* run in the same time and are not counted")
        if "train_ift_kernel" in tp and rooted:
            kern[f"train_ift_kernel ({tname})"] = roofline_entry(
                "train_ift_kernel", "l2-atomic", rooted * 8 * sc.n_bones * 4, "B", tp["train_ift_kernel"][1],
                peaks_g["atomic16"], "GB/s",
                "ia_atomic_probe: random float4 atomicAdds on a skinning-grid-sized table, measured in this run",
                "per sample with a root: 8 corners x 24 bones fp32 of skinning-grid gradient as float4 atomics; "
                "the Jacobian's gathers and the bone-gradient reduction run in the same time and are not counted")
        if tname != "fp32":
            add("wgrad_tc_kernel", tp, "hbm", WGRAD_ROW_BYTES * searched, "B", hbm, "GB/s", hbm_src,
                "the 384-row fp16 operand column of every searched sample, streamed once")
            add("train_backward_h_kernel<fp16>", tp, "tensor", FLOP_MLP_BWD * searched, "FLOP", tc, "TFLOP/s",
                f"{peak_kind} dense bf16 tensor peak (fp16 runs at the same rate)",
                "MLP forward recompute + backward per searched sample")
        else:
            add("train_backward_kernel", tp, "alu", FLOP_MLP_BWD * searched, "FLOP", peak, "TFLOP/s",
                f"fp32 FMA: 148 SM x 128 lanes x 2 x {sm_mhz:.0f} MHz", "MLP forward recompute + backward per sample")
    launches_per_frame = sum(n for n, _ in prof_plain.values())
    m16 = statistics.mean(step16)
    line = {
        "metric": METRIC,
        "value": round(fps, 3),
        "unit": "frames/s",
        # headline numbers of the metric's other parts (the FP16 + proposal path and the train steps)
        "fp16_proposal_fps": round(1e3 / m16, 3),
        "fp16_proposal_speedup": round(statistics.mean(step_ms) / m16, 3),
        "samples_per_s": round(per_frame["occupied_samples"] * fps, 1),
        "fp16_proposal_samples_per_s": round(per_frame16["occupied_samples"] * 1e3 / m16, 1),
        "marched_slots_per_s": round(per_frame["marched_slots"] * fps, 1),
        "train_step_ms_fp32_8192": train["fp32_8192"]["ms"],
        "train_step_ms_fp32_32768": train["fp32"]["ms"],
        "train_step_ms_fp16_proposal_32768": train["fp16_proposal"]["ms"],
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "flushed (256 MiB write) before every timed step",
                   "parallelism": f"replicas x{world}", "precision": "fp32", "starts": "all 24 bones",
                   "value": "540x540 frames/s, pose + occupancy refresh + render, plain fp32"},
        "roofline": roofline_gather,
        "render_roofline": render_roofline,
        "roofline_alu": {"kernel": "wf_field_kernel<fp32>", "bound": "alu", "achieved": round(achieved, 3),
                         "peak": round(peak, 2), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                         "peak_source": f"fp32 FMA: 148 SM x 128 lanes x 2 x {sm_mhz:.0f} MHz ({peak_kind} max clock)",
                         "flop_per_launch": round(flop_field),
                         "work": "per distinct root: Newton polish, hash encoding, fp32 MLP 32-64-64-4, activations"},
        "rooflines": kern,
        "probe_peaks": dict(peaks_g, unit="GB/s", what="useful bytes per second of random records: 48-byte "
                            "gathers from L1- and L2-sized tables, 4/8-byte gathers from hash-table-sized tables, "
                            "8/16-byte vector atomics (ia_gather_probe, ia_atomic_probe)"),
        "correspondence": residual,
        "render_only_fps": round(1e3 / r_ms, 3),
        "mean_broyden_iters_per_sample": round(per_frame["broyden_iters"] / per_frame["occupied_samples"], 2),
        "per_frame": {k: round(v, 1) for k, v in per_frame.items()},
        "occupancy_per_frame": {k: round(v, 1) for k, v in occ_per_frame.items()},
        "kernels_per_frame": {"fp32": {k: [round(n, 2), round(ms, 4)] for k, (n, ms) in prof_plain.items()},
                              "fp16_proposal": {k: [round(n, 2), round(ms, 4)] for k, (n, ms) in prof16.items()},
                              "what": "[launches per frame, ms per launch] from launch tracing over 8 frames"},
        "kernels_per_train_step": {n: {k: [round(c, 2), round(ms, 4)] for k, (c, ms) in tp.items()}
                                   for n, (tp, _) in prof_train.items()},
        "occupancy_refresh": {
            "culled_ms": round(occ_cull_ms, 4), "full_search_ms": round(occ_full_ms, 4),
            "speedup": round(occ_full_ms / occ_cull_ms, 2),
            "searched_cells": round(occ_per_frame["starts"] / (sc.n_bones * sc.occ_res ** 3), 4),
            "what": "ia_update_occupancy of one 64^3 grid, plain fp32, culling on vs off (same densities)"},
        "step_ms": {"mean": round(statistics.mean(step_ms), 4), "min": round(min(step_ms), 4),
                    "max": round(max(step_ms), 4)},
        "render_ms": {"mean": round(r_ms, 4), "min": round(min(render_ms), 4)},
        "wall_s": round(wall, 3),
        "fp16_proposal": {
            "frames_per_s": round(1e3 / m16, 3), "ms_per_step": round(m16, 4),
            "render_only_fps": round(1e3 / statistics.mean(render16), 3),
            "samples_per_s": round(per_frame16["occupied_samples"] * 1e3 / m16, 1),
            "mean_broyden_iters_per_sample": round(per_frame16["broyden_iters"] / per_frame16["occupied_samples"], 2),
            "mean_starts_per_sample": round(per_frame16["starts"] / per_frame16["occupied_samples"], 2),
            "fallback_rate": round(per_frame16["fallbacks"] / max(per_frame16["proposed"], 1), 4),
            "point_culled_rate": round(per_frame16.get("point_culled", 0) / max(per_frame16["proposed"], 1), 4),
            "miss_rate_rays": round(differ / max(hit, 1), 5),
            "miss_definition": "hit rays of 4 frames whose colour or opacity differs from plain fp32 by more "
                               "than 2e-3 relative + 2e-4",
            "speedup_vs_plain_fp32": round(statistics.mean(step_ms) / m16, 3),
            "proposal_training": prop_train,
            "per_frame": {k: round(v, 1) for k, v in per_frame16.items()},
        },
        "train_step_fp32": dict(train["fp32_8192"], what="forward + hand-written backward (all gradients), "
                                "no optimiser, L2 flushed before each step"),
        "train_step_32768": {
            "fp32_ms": train["fp32"]["ms"], "fp16_ms": train["fp16"]["ms"], "bf16_ms": train["bf16"]["ms"],
            "fp16_proposal_ms": train["fp16_proposal"]["ms"],
            "speedup_fp16_proposal_vs_fp32": round(train["fp32"]["ms"] / train["fp16_proposal"]["ms"], 3),
            "speedup_fp16_vs_fp32": round(train["fp32"]["ms"] / train["fp16"]["ms"], 3),
            "detail": {k: train[k] for k in ("fp32", "fp16", "bf16", "fp16_proposal")},
            "what": "32768 rays over 16 poses, <=128 slots, forward + hand-written backward, fp32 master "
                    "gradients; fp16 with dynamic loss scaling, weight gradients on tcgen05"},
        "train_quality": quality,
        "skip_ablation": ablation,
        "e2e": {"value": round(1.0 / statistics.mean(e2e_s), 3), "unit": "frames/s",
                "h2d_bytes_per_step": int(sc.n_bones * 3 * 8 + 3 * 8),
                "d2h_bytes_per_step": int(W * H * 4 * 4)},
        "gpu_launches": int(round(launches_per_frame * args.steps)),
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
    2-row stripe of the image).  ms_per_step is the measured time of that
    work; value (frames/s) divides the part's frame fraction by it, each of
    the two parts scaled by its own fraction of the frame."""
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
        rows = [r for r in range(H) if (r // 2) % n_parts == part]
        pix = np.concatenate([np.arange(r * W, (r + 1) * W) for r in rows]).astype(np.int32)
        t0 = time.perf_counter()
        om.occupancy_cells(p, cells, nthreads)
        t1 = time.perf_counter()
        om.render_pixels(p, cam, bits, pix, nthreads)
        t2 = time.perf_counter()
        frame_s = (t1 - t0) * (R ** 3) / len(cells) + (t2 - t1) * H / len(rows)
        return t2 - t0, frame_s

    for i in range(args.warmup):
        one(i)
    step_s, frame_s = [], []
    t0 = time.perf_counter()
    for i in range(args.steps):
        a, b = one(args.warmup + i)
        step_s.append(a)
        frame_s.append(b)
    wall = time.perf_counter() - t0
    fps = 1.0 / statistics.mean(frame_s)
    return {"impl": "reference", "metric": METRIC, "value": round(fps, 5), "unit": "frames/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * statistics.mean(step_s), 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "host caches, not flushed (the oracle runs on the CPU)",
                       "parallelism": f"{nthreads} host threads", "precision": "fp64", "starts": "all 24 bones",
                       "value": "540x540 frames/s, pose + occupancy refresh + render, fp64 oracle"},
            "work_per_step": f"1/{n_parts} of a frame: one z-slab of the 64^3 occupancy grid and every "
                             f"{n_parts}th 2-row stripe of the 540 x 540 image",
            "frame_ms_extrapolated": round(1e3 * statistics.mean(frame_s), 1),
            "wall_s": round(wall, 2),
            "cpu_baseline": {"value": round(fps, 5), "unit": "frames/s", "cores": nthreads, "kind": "oracle",
                             "sample": f"pose 0; per step 1/{n_parts} of the occupancy grid (a z-slab) and of "
                                       "the image rows (2-row stripes), each part's time divided by its fraction "
                                       "of the frame"},
            "e2e": {"value": round(fps, 5), "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--train-rays", type=int, default=32768, help="rays per step of --only train")
    ap.add_argument("--only", default="all", choices=["all", "plain", "train", "quality", "ablation", "proposal",
                                                      "profile"],
                    help="plain: time only the plain fp32 frames; train: only the fp32 and fp16 training "
                         "steps (both used for profiling captures); profile: per-kernel launch times")
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
