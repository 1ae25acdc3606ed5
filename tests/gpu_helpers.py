"""Shared set-up for the GPU parity tests: a library context and an oracle model
built from the same seeded synthetic inputs."""
import numpy as np

import oracle as O
import synthetic as S

# Tolerances.  Colour and opacity: 1e-5 relative (plus a 1e-6 absolute floor for
# values near zero, i.e. 1e-6 of full scale).  The fp32 path's sample positions,
# roots (after one Newton polish) and field agree with fp64 to ~1e-7 relative;
# the field's log-density slope (<= ~150 / m for the fixture) turns a 1e-7 m
# root difference into ~1.5e-5 relative density, so density and canonical roots
# get the looser bounds below.
RTOL_RGB, ATOL_RGB = 1e-5, 1e-6
RTOL_SIGMA = 1e-4
ATOL_XSTAR = 2e-5


def make_ctx(ia, torch, sc, table, mlp, early_T=0.0, max_samples=None, precision=0):
    cfg = ia.make_config(n_levels=sc.n_levels, log2_table=sc.log2_table, level_res=sc.level_res,
                         max_samples=sc.max_samples if max_samples is None else max_samples,
                         broyden_max_iter=sc.broyden_max_iter, broyden_tol=sc.broyden_tol,
                         occ_res=sc.occ_res, occ_tau=sc.occ_tau, occ_dilate=sc.occ_dilate,
                         early_stop_T=early_T, precision=precision)
    ctx = ia.ia_create(cfg)
    ia.ia_set_skeleton(ctx, sc.parents, sc.rest_joints, sc.skin_grid, sc.canon_min, sc.canon_max,
                       sc.norm_min, sc.norm_max)
    ia.ia_set_params(ctx, torch.from_numpy(np.ascontiguousarray(table)).cuda(),
                     torch.from_numpy(S.pack_mlp(mlp)).cuda())
    torch.cuda.synchronize()
    return ctx


def camera(ia, cam):
    return ia.make_camera(cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["width"], cam["height"], cam["c2w"])


def close(gpu, ref, rtol, atol):
    gpu, ref = np.asarray(gpu, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    return np.abs(gpu - ref) <= rtol * np.abs(ref) + atol


def err_report(name, gpu, ref):
    gpu, ref = np.asarray(gpu, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    d = np.abs(gpu - ref)
    rel = d / np.maximum(np.abs(ref), 1e-30)
    big = np.abs(ref) > 1e-3
    print(f"{name}: max abs {d.max() if d.size else 0:.3e}  max rel (|ref|>1e-3) "
          f"{rel[big].max() if big.any() else 0:.3e}  n={ref.size}")


def points_near_body(sc, om, p, n, seed):
    """Posed (normalised-space) points: canonical points near the capsules, skinned."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        s = rng.integers(len(sc.seg_a))
        t = rng.uniform()
        c = sc.seg_a[s] + t * (sc.seg_b[s] - sc.seg_a[s]) + rng.normal(0, 0.06, 3)
        if np.all(c > sc.canon_min) and np.all(c < sc.canon_max):
            out.append(om.lbs(p, c))
    return np.array(out, dtype=np.float32)


def bits_to_bool(bits, n):
    return np.unpackbits(np.asarray(bits, dtype=np.uint32).view(np.uint8), bitorder="little")[:n].astype(bool)
