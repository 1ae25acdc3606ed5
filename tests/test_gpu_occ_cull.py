"""Exact culling of the occupancy queries, render samples and training samples
(searched only where a root can exist): with culling on, densities, frames and
training steps are those of the full search (bit-identical: every sample's
search items are merged in start order whichever other samples are searched),
the culled cells are the ones without a root (same root and convergence counts),
and the search work drops.  The full search itself is checked against the
oracle in test_gpu_parity.py; this file checks that culling changes nothing."""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from gpu_helpers import make_ctx

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ia():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_10550_b300 as ia
    ia.lib()
    return ia


def _ctx(ia, sc, table, mlp, precision):
    if precision == "fp32":
        return make_ctx(ia, torch, sc, table, mlp)
    cfg = ia.make_config(n_levels=sc.n_levels, log2_table=sc.log2_table, level_res=sc.level_res,
                         max_samples=sc.max_samples, broyden_max_iter=sc.broyden_max_iter,
                         broyden_tol=sc.broyden_tol, occ_res=sc.occ_res, occ_tau=sc.occ_tau,
                         occ_dilate=sc.occ_dilate, early_stop_T=0.0, precision=ia.IA_FP16)
    ctx = ia.ia_create(cfg)
    ia.ia_set_skeleton(ctx, sc.parents, sc.rest_joints, sc.skin_grid, sc.canon_min, sc.canon_max,
                       sc.norm_min, sc.norm_max)
    ia.ia_set_params(ctx, torch.from_numpy(np.ascontiguousarray(table)).cuda(),
                     torch.from_numpy(S.pack_mlp(mlp)).cuda())
    torch.cuda.synchronize()
    return ctx


def _densities(ia, ctx, pose, R, cull):
    ia.ia_set_occupancy_culling(ctx, cull)
    sig = torch.full((R ** 3,), -1.0, device="cuda")
    bits = torch.zeros((R ** 3 + 31) // 32, dtype=torch.int32, device="cuda")
    st = ia.ia_update_occupancy(ctx, pose, ia.IA_OCC_POSE, sig, bits, stats=True)
    torch.cuda.synchronize()
    return sig.cpu().numpy(), bits.cpu().numpy(), st


@pytest.mark.parametrize("config", ["tiny", "full"])
@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_culling_keeps_every_density(ia, config, precision):
    sc = S.make_scene(config, 0)
    table, mlp = S.make_field(sc, 0)
    ctx = _ctx(ia, sc, table, mlp, precision)
    seeds = [1, 2, 5]
    poses = [S.make_pose(sc, s) for s in seeds]
    ia.ia_set_pose(ctx, np.stack([p[0] for p in poses]), np.stack([p[1] for p in poses]))
    R = sc.occ_res
    for i in range(len(seeds)):
        s_off, b_off, st_off = _densities(ia, ctx, i, R, False)
        s_on, b_on, st_on = _densities(ia, ctx, i, R, True)
        print(f"{config} {precision} pose {i}: starts {st_on['starts']} of {st_off['starts']}, "
              f"roots {st_on['roots']}, rooted cells {(s_off > 0).sum()} of {R ** 3}")
        assert (s_on >= 0).all()  # every cell written
        np.testing.assert_array_equal(s_on, s_off)
        np.testing.assert_array_equal(b_on, b_off)
        assert st_on["roots"] == st_off["roots"]
        assert st_on["converged"] == st_off["converged"]
        assert st_on["starts"] <= st_off["starts"]
        if config == "full":
            assert st_on["starts"] < 0.5 * st_off["starts"]  # most of the grid is culled
    ia.ia_destroy(ctx)


def test_culling_with_jitter_and_static_entry(ia):
    sc = S.make_scene("full", 0)
    table, mlp = S.make_field(sc, 0)
    ctx = make_ctx(ia, torch, sc, table, mlp)
    poses = [S.make_pose(sc, s) for s in (3, 4)]
    ia.ia_set_pose(ctx, np.stack([p[0] for p in poses]), np.stack([p[1] for p in poses]))
    R = sc.occ_res
    out = {}
    for cull in (False, True):
        ia.ia_set_occupancy_culling(ctx, cull)
        dens = torch.zeros(R ** 3, device="cuda")
        for i in range(2):
            jit = torch.from_numpy(S.occupancy_jitter(sc, 10 + i)).cuda()
            # decay 0 on the first frame restarts the running density
            ia.ia_update_occupancy_ema(ctx, i, jit, 0.0 if i == 0 else 0.9, dens, None)
        # points outside their cells (u outside [0, 1)) are searched as well
        u = np.random.default_rng(7).uniform(-0.5, 1.5, size=(R ** 3, 3)).astype(np.float32)
        ia.ia_update_occupancy_ema(ctx, 1, torch.from_numpy(u).cuda(), 0.5, dens, None)
        static_bits = torch.zeros((R ** 3 + 31) // 32, dtype=torch.int32, device="cuda")
        ia.ia_update_occupancy_static(ctx, 0, static_bits)
        torch.cuda.synchronize()
        out[cull] = (dens.cpu().numpy(), static_bits.cpu().numpy())
    np.testing.assert_array_equal(out[True][0], out[False][0])
    np.testing.assert_array_equal(out[True][1], out[False][1])
    assert (out[True][0] > 0).any()
    ia.ia_destroy(ctx)


def test_culled_search_against_oracle(ia):
    """Against the fp64 oracle at every cell of one full-size pose, the culled
    search differs only where the full search does: a cell where one side finds
    a marginal root and the other none (at most 0.1 % of the cells, as in the
    occupancy parity tests).  The bound itself is pinned against the oracle's
    roots on the CPU (test_occ_cull_bound.py)."""
    sc = S.make_scene("full", 0)
    table, mlp = S.make_field(sc, 0)
    ctx = make_ctx(ia, torch, sc, table, mlp)
    th, tr = S.make_pose(sc, 6)
    ia.ia_set_pose(ctx, th[None], tr[None])
    R = sc.occ_res
    s_off, _, _ = _densities(ia, ctx, 0, R, False)
    s_on, _, st = _densities(ia, ctx, 0, R, True)
    om = O.OracleModel(sc, table, mlp)
    ref, _ = om.occupancy(om.pose(th, tr))
    diff_on = (s_on > 0) != (ref > 0)
    diff_off = (s_off > 0) != (ref > 0)
    print(f"oracle rooted cells {(ref > 0).sum()}, searched {st['starts'] / sc.n_bones:.0f} of {R ** 3}, "
          f"rooted on one side only {diff_on.sum()}")
    assert (diff_on != diff_off).sum() <= 2
    assert diff_on.sum() <= 1e-3 * R ** 3
    ia.ia_destroy(ctx)


def _render(ia, ctx, pose, icam, n, cull):
    ia.ia_set_occupancy_culling(ctx, cull)
    ia.ia_update_occupancy(ctx, pose)
    rgb = torch.zeros(n, 3, device="cuda")
    alpha = torch.zeros(n, device="cuda")
    st = ia.ia_render(ctx, pose, icam, rgb, alpha, stats=True)
    torch.cuda.synchronize()
    return rgb.cpu().numpy(), alpha.cpu().numpy(), st


@pytest.mark.parametrize("mode", ["fp32", "fp16_proposal"])
def test_render_culling_keeps_every_pixel(ia, mode):
    """Samples whose point can have no root are not searched; the frame is
    bit-identical to the one that searches them (with early termination on, as
    in the frame benchmark).  The proposal mode uses an untrained network, so
    most proposals fail and the fallback search runs often."""
    from gpu_helpers import camera
    sc = S.make_scene("full", 0)
    table, mlp = S.make_field(sc, 0)
    prec = ia.IA_FP32 if mode == "fp32" else ia.IA_FP16
    cfg = ia.make_config(n_levels=sc.n_levels, log2_table=sc.log2_table, level_res=sc.level_res,
                         max_samples=sc.max_samples, occ_res=sc.occ_res, occ_tau=sc.occ_tau,
                         occ_dilate=sc.occ_dilate, early_stop_T=1e-4, precision=prec)
    ctx = ia.ia_create(cfg)
    ia.ia_set_skeleton(ctx, sc.parents, sc.rest_joints, sc.skin_grid, sc.canon_min, sc.canon_max,
                       sc.norm_min, sc.norm_max)
    ia.ia_set_params(ctx, torch.from_numpy(table).cuda(), torch.from_numpy(S.pack_mlp(mlp)).cuda())
    poses = [S.make_pose(sc, s) for s in (2, 9)]
    ia.ia_set_pose(ctx, np.stack([p[0] for p in poses]), np.stack([p[1] for p in poses]))
    if mode == "fp16_proposal":
        pc = S.proposal_config()
        ia.ia_proposal_init(ctx, ia.make_proposal_config(pc["n_levels"], pc["log2_table"], pc["level_res"],
                                                         pc["top_k"], pc["offset_weight"]))
        pt, pm = S.proposal_init(sc, pc, 3)
        ia.ia_proposal_set_params(ctx, torch.from_numpy(pt).cuda(), torch.from_numpy(S.pack_proposal(pm)).cuda())
        ia.ia_set_search(ctx, ia.IA_SEARCH_PROPOSAL)
    cam = S.make_camera(sc)
    icam = camera(ia, cam)
    n = cam["width"] * cam["height"]
    for pose in range(2):
        r0, a0, st0 = _render(ia, ctx, pose, icam, n, False)
        r1, a1, st1 = _render(ia, ctx, pose, icam, n, True)
        print(f"{mode} pose {pose}: culled {st1['culled']} of {st1['occupied_samples']} samples, "
              f"starts {st1['starts']} vs {st0['starts']}, fallbacks {st1['fallbacks']} vs {st0['fallbacks']}")
        np.testing.assert_array_equal(r1, r0)
        np.testing.assert_array_equal(a1, a0)
        assert st0["culled"] == 0 and st1["culled"] > 0
        assert st1["starts"] < st0["starts"]
        if mode == "fp16_proposal":
            # a culled or point-culled sample has no root, so its proposed starts
            # fail: without culling it falls back
            assert st0["point_culled"] == 0 and st1["point_culled"] > 0
            assert st0["fallbacks"] == st1["fallbacks"] + st1["culled"] + st1["point_culled"]
        assert st1["roots"] == st0["roots"]
        assert (a1 > 0).sum() > 0.05 * n
    # the masks belong to the pose of the last occupancy update: rendering another
    # pose (here with that pose's grid) culls nothing
    ia.ia_update_occupancy(ctx, 0)
    rgb = torch.zeros(n, 3, device="cuda")
    alpha = torch.zeros(n, device="cuda")
    st = ia.ia_render(ctx, 1, icam, rgb, alpha, stats=True)
    assert st["culled"] == 0
    # so does a grid whose pose's blended grid has changed since
    ia.ia_set_pose(ctx, np.stack([p[0] for p in poses]), np.stack([p[1] for p in poses]))
    st = ia.ia_render(ctx, 0, icam, rgb, alpha, stats=True)
    assert st["culled"] == 0
    ia.ia_destroy(ctx)


@pytest.mark.parametrize("prec", ["fp32", "fp16", "fp16_proposal"])
def test_training_culling_keeps_the_step(ia, prec):
    """The training step skips samples (and regulariser points) whose point can
    have no root in their own pose, and with the proposal search the samples
    whose proposed starts failed and whose point lies in no grown image box of
    their pose's canonical cells: per-ray colours are bit-identical, loss and
    gradients equal up to the order of their fp32 atomic sums."""
    sc = S.make_scene("full", 0)
    table, mlp = S.make_field(sc, 0)
    cfg = ia.make_config(n_levels=sc.n_levels, log2_table=sc.log2_table, level_res=sc.level_res,
                         max_samples=sc.max_samples, occ_res=sc.occ_res, occ_tau=sc.occ_tau,
                         occ_dilate=sc.occ_dilate, early_stop_T=0.0,
                         precision=ia.IA_FP32 if prec == "fp32" else ia.IA_FP16)
    ctx = ia.ia_create(cfg)
    ia.ia_set_skeleton(ctx, sc.parents, sc.rest_joints, sc.skin_grid, sc.canon_min, sc.canon_max,
                       sc.norm_min, sc.norm_max)
    ia.ia_set_params(ctx, torch.from_numpy(table).cuda(), torch.from_numpy(S.pack_mlp(mlp)).cuda())
    if prec == "fp16_proposal":
        pc = S.proposal_config()
        ia.ia_proposal_init(ctx, ia.make_proposal_config(pc["n_levels"], pc["log2_table"], pc["level_res"],
                                                         pc["top_k"], pc["offset_weight"]))
        pt, pm = S.proposal_init(sc, pc, 3)
        ia.ia_proposal_set_params(ctx, torch.from_numpy(pt).cuda(), torch.from_numpy(S.pack_proposal(pm)).cuda())
        ia.ia_set_search(ctx, ia.IA_SEARCH_PROPOSAL)
    n_poses = 8
    poses = [S.make_pose(sc, i) for i in range(n_poses)]
    ia.ia_set_pose(ctx, np.stack([p[0] for p in poses]), np.stack([p[1] for p in poses]))
    for i in range(n_poses):
        ia.ia_update_occupancy(ctx, i, ia.IA_OCC_UNION)
    rb = S.make_ray_batch(sc, 8192, n_poses, seed=4)
    dev = {k: torch.from_numpy(np.ascontiguousarray(rb[k])).cuda() for k in ("origin", "direction", "pose", "target")}
    rng = np.random.default_rng(5)
    reg_x = torch.from_numpy(S.random_points(sc, 8192, seed=6)).cuda()
    reg_pose = torch.from_numpy(rng.integers(0, n_poses, 8192).astype(np.int32)).cuda()
    nt, nm = ia.ia_param_sizes(ctx)
    out = {}
    for cull in (False, True):
        ia.ia_set_occupancy_culling(ctx, cull)
        g = dict(table=torch.zeros(nt, device="cuda"), mlp=torch.zeros(nm, device="cuda"),
                 skin=torch.zeros(sc.skin_res ** 3 * sc.n_bones, device="cuda"),
                 bones=torch.zeros(n_poses * sc.n_bones * 12, device="cuda"))
        loss = torch.zeros(1, device="cuda")
        rgb = torch.zeros(8192, 3, device="cuda")
        # (the proposal variant without regulariser points: culled points are not
        # counted in the stats, so the fallback identity below covers ray samples)
        reg = {} if prec == "fp16_proposal" else dict(reg_x=reg_x, reg_pose=reg_pose, reg_weight=0.1)
        ia.ia_train_step(ctx, dev["origin"], dev["direction"], dev["pose"], dev["target"], loss, g,
                         occ_grid=ia.IA_OCC_UNION, rgb_out=rgb, **reg)
        st = ia.ia_train_stats(ctx)
        torch.cuda.synchronize()
        out[cull] = (float(loss.item()), rgb.cpu().numpy(), {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()},
                     st)
    (l0, r0, g0, s0), (l1, r1, g1, s1) = out[False], out[True]
    print(f"{prec}: culled {s1['culled']} of {s1['occupied_samples']} samples, starts {s1['starts']} vs {s0['starts']}, "
          f"loss {l1:.8e} vs {l0:.8e}")
    assert s0["culled"] == 0 and s1["culled"] > 0
    assert s1["occupied_samples"] == s0["occupied_samples"]
    assert s1["starts"] < s0["starts"]
    if prec == "fp16_proposal":
        print(f"fallbacks {s1['fallbacks']} + culled {s1['culled']} + point-culled {s1['point_culled']} "
              f"(culling off: {s0['fallbacks']})")
        assert s0["point_culled"] == 0 and s1["point_culled"] > 0
        assert s0["fallbacks"] == s1["fallbacks"] + s1["culled"] + s1["point_culled"]
    np.testing.assert_array_equal(r1, r0)
    assert abs(l1 - l0) <= 1e-6 * abs(l0)
    for k in ("table", "mlp", "skin", "bones"):
        rel = np.linalg.norm(g1[k] - g0[k]) / max(np.linalg.norm(g0[k]), 1e-30)
        print(f"grad {k}: rel L2 {rel:.2e}")
        assert np.count_nonzero(g0[k]) > 0
        assert rel <= 1e-5, k
    ia.ia_destroy(ctx)
