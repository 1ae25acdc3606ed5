"""Reduced-precision field (fp16 hash features, fp16 / bf16 tensor-core MLP with
fp32 accumulation) against the fp64 oracle.

Tolerances: fp16 colour and opacity 2e-3 relative (plus 2e-4 of full scale for
values near zero), the bound stated for the fp16 MLP.  bf16 keeps 8 mantissa
bits (unit roundoff 2^-9 = 2e-3 per rounding, three roundings deep through the
network), so its bound is 5x looser: 1e-2 relative (+1e-3).  Density is
exp(o0): an absolute error e in o0 is a relative error e in density, bounded
here by 2e-2 (fp16) and 1e-1 (bf16).  Root finding stays fp32, so the sample set
and the canonical roots are those of the fp32 path; the oracle's occupancy bits
are installed so both sides evaluate the same samples.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from gpu_helpers import camera, close, err_report, make_ctx

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {1: dict(rgb=(2e-3, 2e-4), sigma=2e-2), 2: dict(rgb=(1e-2, 1e-3), sigma=1e-1)}
NAMES = {1: "fp16", 2: "bf16"}


@pytest.fixture(scope="module")
def ia():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_10550_b300 as ia
    ia.lib()
    return ia


def _ctx(ia, sc, table, mlp, prec, early_T=0.0):
    cfg = ia.make_config(n_levels=sc.n_levels, log2_table=sc.log2_table, level_res=sc.level_res,
                         max_samples=sc.max_samples, occ_res=sc.occ_res, occ_tau=sc.occ_tau,
                         occ_dilate=sc.occ_dilate, early_stop_T=early_T, precision=prec)
    ctx = ia.ia_create(cfg)
    ia.ia_set_skeleton(ctx, sc.parents, sc.rest_joints, sc.skin_grid, sc.canon_min, sc.canon_max,
                       sc.norm_min, sc.norm_max)
    ia.ia_set_params(ctx, torch.from_numpy(table).cuda(), torch.from_numpy(S.pack_mlp(mlp)).cuda())
    return ctx


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("config", ["tiny", "full"])
def test_canonical_field_reduced_precision(ia, prec, config):
    sc = S.make_scene(config, 0)
    table, mlp = S.make_field(sc, 0)
    ctx = _ctx(ia, sc, table, mlp, prec)
    om = O.OracleModel(sc, table, mlp)
    rng = np.random.default_rng(3)
    s = rng.integers(len(sc.seg_a), size=3000)
    t = rng.uniform(size=(3000, 1))
    x = np.clip(sc.seg_a[s] + t * (sc.seg_b[s] - sc.seg_a[s]) + rng.normal(0, 0.05, (3000, 3)),
                sc.canon_min, sc.canon_max).astype(np.float32)
    x = np.concatenate([x, S.random_points(sc, 1000, seed=4, box="canon")])
    sig = torch.zeros(len(x), device="cuda")
    rgb = torch.zeros(len(x), 3, device="cuda")
    ia.ia_query_canonical(ctx, torch.from_numpy(x).cuda(), sig, rgb)
    torch.cuda.synchronize()
    ref = [om.field(p) for p in x.astype(np.float64)]
    rs, rc = np.array([r[0] for r in ref]), np.array([r[1] for r in ref])
    err_report(f"{NAMES[prec]} canonical sigma", sig.cpu().numpy(), rs)
    err_report(f"{NAMES[prec]} canonical rgb", rgb.cpu().numpy(), rc)
    assert close(sig.cpu().numpy(), rs, TOL[prec]["sigma"], 1e-7).all()
    assert close(rgb.cpu().numpy(), rc, *TOL[prec]["rgb"]).all()
    ia.ia_destroy(ctx)


@pytest.mark.parametrize("prec", [1, 2])
def test_render_reduced_precision(ia, prec):
    for config in ("tiny", "full"):
        sc = S.make_scene(config, 0)
        table, mlp = S.make_field(sc, 0)
        om = O.OracleModel(sc, table, mlp)
        th, tr = S.make_pose(sc, 2)
        p = om.pose(th, tr)
        _, occ = om.occupancy(p)
        ctx = _ctx(ia, sc, table, mlp, prec)
        ia.ia_set_pose(ctx, th[None], tr[None])
        ia.ia_set_occupancy(ctx, occ)
        cam = S.make_camera(sc)
        W, H = cam["width"], cam["height"]
        rgb = torch.zeros(W * H, 3, device="cuda")
        alpha = torch.zeros(W * H, device="cuda")
        stats = ia.ia_render(ctx, 0, camera(ia, cam), rgb, alpha, stats=True)
        if config == "tiny":
            pix = np.arange(W * H)
        else:
            pix = np.random.default_rng(5).choice(W * H, 3000, replace=False)
        ref = om.render_pixels(p, cam, occ, pix)
        if config == "tiny":
            assert stats["occupied_samples"] == int(ref["nsamp"].sum())
        ok = ref["flags"] == 0
        g_rgb, g_a = rgb.cpu().numpy()[pix], alpha.cpu().numpy()[pix]
        err_report(f"{NAMES[prec]} {config} rgb", g_rgb[ok], ref["rgb"][ok])
        err_report(f"{NAMES[prec]} {config} alpha", g_a[ok], ref["alpha"][ok])
        good = close(g_rgb[ok], ref["rgb"][ok], *TOL[prec]["rgb"]).all(axis=1) & \
            close(g_a[ok], ref["alpha"][ok], *TOL[prec]["rgb"])
        # a density change of this size can move the max-density choice between
        # two roots of close density; such rays are rare and counted
        print(f"{NAMES[prec]} {config}: {np.sum(~good)} of {ok.sum()} rays outside tolerance")
        assert np.sum(~good) <= 0.002 * ok.sum() + 1
        ia.ia_destroy(ctx)
