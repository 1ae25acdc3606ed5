"""The learned correspondence proposal on the GPU.

* its training gradient against the oracle's (fp32 vs fp64),
* its training pairs (label = dominant bone at the selected root, start offset)
  against the oracle,
* after training on the GPU with the library's own kernels: the proposal-mode
  search against the oracle's proposal-mode search with the same weights, and
  what the network gains over the plain search on held-out poses (fewer
  Broyden starts and iterations at a small miss rate).
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from gpu_helpers import camera, close, err_report, points_near_body
from oracle import prop as PP

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_TRAIN, N_TEST, PER = 32, 4, 8192


@pytest.fixture(scope="module")
def ia():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_10550_b300 as ia
    ia.lib()
    return ia


def _ctx(ia, sc, table, mlp, prec, poses):
    cfg = ia.make_config(n_levels=sc.n_levels, log2_table=sc.log2_table, level_res=sc.level_res,
                         max_samples=sc.max_samples, occ_res=sc.occ_res, occ_tau=sc.occ_tau,
                         occ_dilate=sc.occ_dilate, early_stop_T=0.0, precision=prec)
    ctx = ia.ia_create(cfg)
    ia.ia_set_skeleton(ctx, sc.parents, sc.rest_joints, sc.skin_grid, sc.canon_min, sc.canon_max,
                       sc.norm_min, sc.norm_max)
    ia.ia_set_params(ctx, torch.from_numpy(table).cuda(), torch.from_numpy(S.pack_mlp(mlp)).cuda())
    ia.ia_set_pose(ctx, np.stack([p[0] for p in poses]), np.stack([p[1] for p in poses]))
    pc = S.proposal_config()
    ia.ia_proposal_init(ctx, ia.make_proposal_config(pc["n_levels"], pc["log2_table"], pc["level_res"],
                                                     pc["top_k"], pc["offset_weight"]))
    return ctx, pc


def occupied_points(bits, sc, n, rng):
    """Uniform points inside the occupied cells of a packed grid (input sampling)."""
    R = sc.occ_res
    occ = np.unpackbits(np.asarray(bits).view(np.uint8), bitorder="little")[:R ** 3].astype(bool)
    c = rng.choice(np.nonzero(occ)[0], n)
    ijk = np.stack([c % R, (c // R) % R, c // (R * R)], -1)
    cs = (sc.norm_max.astype(np.float64) - sc.norm_min) / R
    return (sc.norm_min + (ijk + rng.uniform(size=(n, 3))) * cs).astype(np.float32)


def test_proposal_gradient_matches_oracle(ia):
    sc = S.make_scene("full", 0)
    table, mlp = S.make_field(sc, 0)
    poses = [S.make_pose(sc, i) for i in range(3)]
    ctx, pc = _ctx(ia, sc, table, mlp, 1, poses)
    pt, pm = S.proposal_init(sc, pc, 2)
    rng = np.random.default_rng(11)
    pt = pt + rng.normal(0, 0.05, pt.shape).astype(np.float32)
    pm = {k: v + (0.05 * rng.normal(size=v.shape)).astype(np.float32) for k, v in pm.items()}
    ia.ia_proposal_set_params(ctx, torch.from_numpy(pt).cuda(), torch.from_numpy(S.pack_proposal(pm)).cuda())
    n = 512
    x = S.random_points(sc, n, seed=12)
    pid = rng.integers(0, 3, n).astype(np.int32)
    lab = rng.integers(0, sc.n_bones, n).astype(np.int32)
    tgt = rng.normal(0, 0.02, (n, 3)).astype(np.float32)
    nt, nm = ia.ia_proposal_param_sizes(ctx)
    gt, gm, loss = (torch.zeros(nt, device="cuda"), torch.zeros(nm, device="cuda"), torch.zeros(1, device="cuda"))
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    ia.ia_proposal_grad(ctx, d(x), d(pid), d(lab), d(tgt), loss, gt, gm)
    torch.cuda.synchronize()
    om = O.OracleModel(sc, table, mlp)
    pr = PP.PropModel(om, pc, pt, pm)
    thetas = np.stack([p[0] for p in poses])
    rl, rt, rm = pr.loss_grad(x, pid, thetas, lab, tgt.astype(np.float64))
    print(f"proposal loss gpu {loss.item():.7e} oracle {rl:.7e}")
    assert abs(loss.item() - rl) <= 1e-5 * rl
    for name, g, r in (("table", gt.cpu().numpy(), rt.reshape(-1)), ("mlp", gm.cpu().numpy(), rm)):
        rel = np.linalg.norm(g - r) / np.linalg.norm(r)
        print(f"proposal grad {name}: rel L2 {rel:.2e}")
        assert rel < 1e-4
        assert np.abs(g - r).max() <= 1e-4 * np.abs(r).max()
    ia.ia_destroy(ctx)


def test_training_pairs_match_oracle(ia):
    sc = S.make_scene("full", 0)
    table, mlp = S.make_field(sc, 0)
    poses = [S.make_pose(sc, 5)]
    ctx, pc = _ctx(ia, sc, table, mlp, 1, poses)
    om = O.OracleModel(sc, table, mlp)
    pr = PP.PropModel(om, pc, *S.proposal_init(sc, pc, 0))
    p = om.pose(*poses[0])
    x = np.concatenate([points_near_body(sc, om, p, 800, 13), S.random_points(sc, 200, seed=14)])
    lab = torch.zeros(len(x), dtype=torch.int32, device="cuda")
    off = torch.zeros(len(x), 3, device="cuda")
    ia.ia_proposal_pairs(ctx, 0, torch.from_numpy(x).cuda(), lab, off)
    torch.cuda.synchronize()
    g_lab, g_off = lab.cpu().numpy(), off.cpu().numpy()
    checked = 0
    for i, xn in enumerate(x.astype(np.float64)):
        s = om.posed_field(p, xn)
        if s["flags"]:
            continue
        if s["start"] < 0:
            assert g_lab[i] == -1
            continue
        w = om.skin_weights(s["xstar"])
        top2 = np.sort(w)[-2:]
        if top2[1] - top2[0] < 1e-4:  # near-tie of the dominant bone: either label is right
            continue
        k, ref_off = pr.label(p, s["xstar"], xn)
        assert g_lab[i] == k
        np.testing.assert_allclose(g_off[i], ref_off, atol=2e-5)
        checked += 1
    assert checked > 600
    ia.ia_destroy(ctx)


def _train_proposal(ia, ctx, sc, pc, n_poses, per, steps, rng):
    """Pairs from the plain search at points in the occupied cells of poses
    0..n_poses-1 of the context, then the library's own training kernels."""
    pt, pm = S.proposal_init(sc, pc, 0)
    ia.ia_proposal_set_params(ctx, torch.from_numpy(pt).cuda(), torch.from_numpy(S.pack_proposal(pm)).cuda())
    R = sc.occ_res
    bits = torch.zeros((R ** 3 + 31) // 32, dtype=torch.int32, device="cuda")
    X, P, L, T = [], [], [], []
    for i in range(n_poses):
        ia.ia_update_occupancy(ctx, i, ia.IA_OCC_POSE, None, bits)
        x = torch.from_numpy(occupied_points(bits.cpu().numpy().view(np.uint32), sc, per, rng)).cuda()
        lab = torch.zeros(per, dtype=torch.int32, device="cuda")
        off = torch.zeros(per, 3, device="cuda")
        ia.ia_proposal_pairs(ctx, i, x, lab, off)
        X.append(x); P.append(torch.full((per,), i, dtype=torch.int32, device="cuda")); L.append(lab); T.append(off)
    X, P, L, T = (torch.cat(a) for a in (X, P, L, T))
    keep = torch.nonzero(L >= 0).squeeze(1)
    perm = keep[torch.from_numpy(rng.permutation(len(keep))).cuda()]
    X, P, L, T = (a[perm].contiguous() for a in (X, P, L, T))
    losses = torch.zeros(steps, device="cuda")
    ia.ia_proposal_train(ctx, X, P, L, T, steps, 8192, 2e-3, losses)
    torch.cuda.synchronize()
    ls = losses.cpu().numpy()
    print(f"proposal training: {len(perm)} pairs, loss {ls[0]:.3f} -> {ls[-20:].mean():.3f}")
    assert ls[-20:].mean() < 0.25 * ls[0]


@pytest.fixture(scope="module")
def trained(ia):
    """A proposal trained on the GPU (library kernels) on pairs from N_TRAIN poses."""
    sc = S.make_scene("full", 0)
    table, mlp = S.make_field(sc, 0)
    poses = [S.make_pose(sc, 100 + i) for i in range(N_TRAIN)] + [S.make_pose(sc, i) for i in range(N_TEST)]
    ctx, pc = _ctx(ia, sc, table, mlp, 1, poses)
    _train_proposal(ia, ctx, sc, pc, N_TRAIN, PER, 400, np.random.default_rng(15))
    yield sc, table, mlp, ctx, pc, poses
    ia.ia_destroy(ctx)


def test_trained_proposal_gains_over_plain_search(ia, trained):
    sc, table, mlp, ctx, pc, poses = trained
    cam = S.make_camera(sc)
    W, H = cam["width"], cam["height"]
    miss_tot = has_tot = 0
    for i in range(N_TRAIN, N_TRAIN + N_TEST):  # held-out poses
        ia.ia_set_search(ctx, ia.IA_SEARCH_ALL_BONES)
        ia.ia_update_occupancy(ctx, i)
        res = {}
        for mode in (ia.IA_SEARCH_ALL_BONES, ia.IA_SEARCH_PROPOSAL):
            ia.ia_set_search(ctx, mode)
            rgb = torch.zeros(W * H, 3, device="cuda")
            a = torch.zeros(W * H, device="cuda")
            st = ia.ia_render(ctx, i, camera(ia, cam), rgb, a, stats=True)
            res[mode] = (st, rgb.cpu().numpy(), a.cpu().numpy())
        sp, rp, ap = res[ia.IA_SEARCH_PROPOSAL]
        s0, r0, a0 = res[ia.IA_SEARCH_ALL_BONES]
        work0 = s0["starts"] + s0["broyden_iters"]
        work1 = sp["starts"] + sp["broyden_iters"]
        diff = ~(close(rp, r0, 2e-3, 2e-4).all(axis=1) & close(ap, a0, 2e-3, 2e-4))
        hit = a0 > 0
        print(f"pose {i}: search work plain {work0} -> proposal {work1} ({work0 / work1:.1f}x), "
              f"fallbacks {sp['fallbacks']}/{sp['proposed']}, rays differing {diff.sum()}/{hit.sum()}")
        # every searched sample takes the proposal (culled ones have no root and are not searched)
        assert sp["proposed"] == s0["occupied_samples"] - s0["culled"]
        assert sp["culled"] == s0["culled"]
        assert work0 >= 4 * work1
        miss_tot += diff.sum()
        has_tot += hit.sum()
    assert miss_tot <= 0.02 * has_tot
    ia.ia_set_search(ctx, ia.IA_SEARCH_ALL_BONES)


def test_proposal_search_matches_oracle(ia, trained):
    sc, table, mlp, ctx, pc, poses = trained
    nt, nm = ia.ia_proposal_param_sizes(ctx)
    pt, pmf = np.zeros(nt, np.float32), np.zeros(nm, np.float32)
    ia.ia_proposal_get_params(ctx, pt, pmf)
    nb = sc.n_bones
    nin = 2 * pc["n_levels"] + 3 * nb
    shapes = [("W1", (64, nin)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (64, 64)), ("b3", (64,)),
              ("W4", (nb + 3, 64)), ("b4", (nb + 3,))]
    pm, o = {}, 0
    for k, shp in shapes:
        n = int(np.prod(shp))
        pm[k] = pmf[o:o + n].reshape(shp)
        o += n
    om = O.OracleModel(sc, table, mlp)
    pr = PP.PropModel(om, pc, pt.reshape(-1, 2), pm)
    i = N_TRAIN
    th, tr = poses[i]
    p = om.pose(th, tr)
    x = points_near_body(sc, om, p, 600, 16)
    ia.ia_set_search(ctx, ia.IA_SEARCH_PROPOSAL)
    sig = torch.zeros(len(x), device="cuda")
    rgb = torch.zeros(len(x), 3, device="cuda")
    xc = torch.zeros(len(x), 3, device="cuda")
    st = torch.zeros(len(x), dtype=torch.int32, device="cuda")
    ia.ia_query_posed(ctx, i, torch.from_numpy(x).cuda(), sig, rgb, xc, st)
    torch.cuda.synchronize()
    ia.ia_set_search(ctx, ia.IA_SEARCH_ALL_BONES)
    g_sig, g_rgb, g_xc, g_st = sig.cpu().numpy(), rgb.cpu().numpy(), xc.cpu().numpy(), st.cpu().numpy()
    ok = []
    for j, xn in enumerate(x.astype(np.float64)):
        r = pr.posed_field(p, th, xn)
        if r["flags"]:
            continue
        assert (g_st[j] >= 0) == (r["start"] >= 0)
        if r["start"] >= 0:
            ok.append((j, r))
    assert len(ok) > 500
    idx = np.array([j for j, _ in ok])
    ref_x = np.array([r["xstar"] for _, r in ok])
    ref_s = np.array([r["sigma"] for _, r in ok])
    ref_c = np.array([r["rgb"] for _, r in ok])
    err_report("proposal x*", g_xc[idx], ref_x)
    assert np.all(np.abs(g_xc[idx] - ref_x) <= 2e-5)
    assert close(g_sig[idx], ref_s, 2e-2, 1e-7).all()
    assert close(g_rgb[idx], ref_c, 2e-3, 2e-4).all()


def _round_fp16(x):
    return np.asarray(x, np.float32).astype(np.float16).astype(np.float32)


def _oracle_fp16(ia, ctx, sc, table, mlp, pc, early_T):
    """The oracle on the operands the fp16 field and proposal read: the hash
    table rounded to fp16, the MLP weights rounded to fp16 (biases fp32); the
    proposal's weights rounded to fp16 except its layer-1 pose columns, which
    the library folds into an fp32 per-pose bias.  The proposal's weights are
    the ones trained on the GPU (an input both sides read)."""
    om = O.OracleModel(sc, _round_fp16(table), {k: (_round_fp16(v) if k.startswith("W") else v)
                                                 for k, v in mlp.items()}, early_T=early_T)
    nt, nm = ia.ia_proposal_param_sizes(ctx)
    pt, pmf = np.zeros(nt, np.float32), np.zeros(nm, np.float32)
    ia.ia_proposal_get_params(ctx, pt, pmf)
    nb = sc.n_bones
    nin = 2 * pc["n_levels"] + 3 * nb
    shapes = [("W1", (64, nin)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (64, 64)), ("b3", (64,)),
              ("W4", (nb + 3, 64)), ("b4", (nb + 3,))]
    pm, o = {}, 0
    for k, shp in shapes:
        n = int(np.prod(shp))
        pm[k] = pmf[o:o + n].reshape(shp).copy()
        o += n
    pm_op = {k: (_round_fp16(v) if k.startswith("W") else v) for k, v in pm.items()}
    nf = 2 * pc["n_levels"]
    pm_op["W1"][:, nf:] = pm["W1"][:, nf:]
    return om, PP.PropModel(om, pc, pt.reshape(-1, 2), pm_op), (pt, pmf)


def _proposal_frame(ia, sc, table, mlp, pc, params, pose, cam, early_T, om, pr, pix, path=1):
    """fp16 + proposal frame of one pose on the GPU (render_kernel with the
    proposal search and root culling, over the oracle's occupancy bits) and the
    oracle's proposal-mode render of the listed pixels."""
    th, tr = pose
    p = om.pose(th, tr)
    _, bits = om.occupancy(p)
    cfg = ia.make_config(n_levels=sc.n_levels, log2_table=sc.log2_table, level_res=sc.level_res,
                         max_samples=sc.max_samples, occ_res=sc.occ_res, occ_tau=sc.occ_tau,
                         occ_dilate=sc.occ_dilate, early_stop_T=early_T, precision=ia.IA_FP16)
    ctx = ia.ia_create(cfg)
    ia.ia_set_skeleton(ctx, sc.parents, sc.rest_joints, sc.skin_grid, sc.canon_min, sc.canon_max,
                       sc.norm_min, sc.norm_max)
    ia.ia_set_params(ctx, torch.from_numpy(table).cuda(), torch.from_numpy(S.pack_mlp(mlp)).cuda())
    ia.ia_set_pose(ctx, th[None], tr[None])
    ia.ia_proposal_init(ctx, ia.make_proposal_config(pc["n_levels"], pc["log2_table"], pc["level_res"],
                                                     pc["top_k"], pc["offset_weight"]))
    ia.ia_proposal_set_params(ctx, torch.from_numpy(params[0]).cuda(), torch.from_numpy(params[1]).cuda())
    ia.ia_set_search(ctx, ia.IA_SEARCH_PROPOSAL)
    ia.ia_update_occupancy(ctx, 0)  # the pose's root-culling masks
    ia.ia_set_occupancy(ctx, bits)  # the grid: the oracle's
    ia.ia_set_render_path(ctx, path)
    W, H = cam["width"], cam["height"]
    rgb = torch.zeros(W * H, 3, device="cuda")
    a = torch.zeros(W * H, device="cuda")
    st = ia.ia_render(ctx, 0, camera(ia, cam), rgb, a, stats=True)
    torch.cuda.synchronize()
    ia.ia_destroy(ctx)
    ref = pr.render_pixels(p, th, cam, bits, pix)
    return st, rgb.cpu().numpy()[pix], a.cpu().numpy()[pix], ref


def _check_frame(name, st, rgb, alpha, ref):
    hit = ref["nsamp"] > 0
    flagged = hit & (ref["flags"] != 0)
    ok = hit & ~flagged
    bad = ok & ~(close(rgb, ref["rgb"], 2e-3, 2e-4).all(axis=1) & close(alpha, ref["alpha"], 2e-3, 2e-4))
    err_report(f"{name} colour", rgb[ok], ref["rgb"][ok])
    err_report(f"{name} opacity", alpha[ok], ref["alpha"][ok])
    bits = {b: int(np.sum(hit & ((ref["flags"] & b) != 0))) for b in (1, 2, 4, 8, 16, 32, 64)}
    print(f"{name}: rays flagged per oracle flag bit {bits}")
    print(f"{name}: {hit.sum()} rays with samples, {flagged.sum()} flagged by the oracle and excluded "
          f"({flagged.sum() / max(hit.sum(), 1):.2%}), {bad.sum()} outside 2e-3; fallbacks gpu {st['fallbacks']} "
          f"+ culled {st['culled']} + point-culled {st['point_culled']}, oracle {int(ref['fallbacks'].sum())}")
    assert hit.sum() > 500
    assert flagged.sum() <= 0.01 * hit.sum()
    assert bad.sum() == 0
    assert np.all(alpha[~hit] == 0) and np.all(ref["alpha"][~hit] == 0)


@pytest.fixture(scope="module")
def trained_tiny(ia):
    """A proposal trained on the GPU for the tiny scene (16 poses)."""
    sc = S.make_scene("tiny", 0)
    table, mlp = S.make_field(sc, 0)
    poses = [S.make_pose(sc, 200 + i) for i in range(16)] + [S.make_pose(sc, 3)]
    ctx, pc = _ctx(ia, sc, table, mlp, 1, poses)
    _train_proposal(ia, ctx, sc, pc, 16, PER, 300, np.random.default_rng(25))
    yield sc, table, mlp, ctx, pc, poses
    ia.ia_destroy(ctx)


@pytest.mark.parametrize("path", ["wavefront", "fused"])
def test_proposal_frame_matches_oracle_tiny(ia, trained_tiny, path):
    """The product path's frame, fp16 with the proposal search, on the whole
    64 x 64 tiny frame of a held-out pose (parity mode: no early termination)
    against the oracle's proposal-mode render (or_render_pixels_prop) with the
    same GPU-trained proposal: colour and opacity of every ray within the fp16
    bound (2e-3 relative + 2e-4), rays the oracle flags as marginal excluded
    (at most 1 %), and the frame's fallback count (samples whose proposed
    starts found no root; the GPU does not search samples that root culling
    proves rootless, so those count on its side as culled, or as point-culled
    when their point lies in no canonical cell's image box) equal to the
    oracle's up to a few marginal samples."""
    sc, table, mlp, ctx, pc, poses = trained_tiny
    om, pr, params = _oracle_fp16(ia, ctx, sc, table, mlp, pc, 0.0)
    cam = S.make_camera(sc)
    pix = np.arange(cam["width"] * cam["height"], dtype=np.int32)
    st, rgb, alpha, ref = _proposal_frame(ia, sc, table, mlp, pc, params, poses[-1], cam, 0.0, om, pr, pix,
                                          {"wavefront": 1, "fused": 0}[path])
    _check_frame(f"tiny fp16+proposal frame ({path})", st, rgb, alpha, ref)
    fb = int(ref["fallbacks"].sum())
    assert st["proposed"] == st["occupied_samples"] - st["culled"] > 0
    assert abs(st["fallbacks"] + st["culled"] + st["point_culled"] - fb) <= max(3, 0.005 * fb)


def test_proposal_frame_matches_oracle_full(ia, trained):
    """The same at full size with the proposal of the 540 x 540 workload:
    (a) a whole 135 x 135 frame of a held-out pose (the 540 x 540 camera at a
    quarter of the resolution) in parity mode, with the fallback count;
    (b) 4000 pixels, drawn from those whose rays reach an occupied cell of the
    oracle's grid, of the 540 x 540 frame with early termination at T < 1e-4
    (the benchmark's configuration; rays whose transmittance ends within
    1e-3 of the threshold are flagged by the oracle and excluded)."""
    sc, table, mlp, ctx, pc, poses = trained
    pose = poses[N_TRAIN]
    om, pr, params = _oracle_fp16(ia, ctx, sc, table, mlp, pc, 0.0)
    cam = S.make_camera(sc, 135, 135)
    pix = np.arange(135 * 135, dtype=np.int32)
    st, rgb, alpha, ref = _proposal_frame(ia, sc, table, mlp, pc, params, pose, cam, 0.0, om, pr, pix)
    _check_frame("135^2 fp16+proposal frame", st, rgb, alpha, ref)
    fb = int(ref["fallbacks"].sum())
    assert st["proposed"] == st["occupied_samples"] - st["culled"] > 0
    assert abs(st["fallbacks"] + st["culled"] + st["point_culled"] - fb) <= max(3, 0.005 * fb)

    om, pr, params = _oracle_fp16(ia, ctx, sc, table, mlp, pc, 1e-4)
    cam = S.make_camera(sc)
    p = om.pose(*pose)
    _, bits = om.occupancy(p)
    reach = np.nonzero(om.march_mask(p, cam, bits).any(axis=1))[0]
    pix = np.sort(np.random.default_rng(31).choice(reach, 4000, replace=False)).astype(np.int32)
    st, rgb, alpha, ref = _proposal_frame(ia, sc, table, mlp, pc, params, pose, cam, 1e-4, om, pr, pix)
    _check_frame("540^2 fp16+proposal frame, 4000 pixels, early termination", st, rgb, alpha, ref)
