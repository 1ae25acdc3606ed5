"""GPU parity: the CUDA path through the C ABI against the fp64 oracle.

Bit-exact: bone transforms as stored (fp32 casts of the fp64 chain), occupancy
bits from a shared density array, the per-ray set of evaluated slots.
Within tolerance (gpu_helpers): canonical field, posed field, occupancy
densities, rendered colour and opacity.  Rays or samples the oracle flags as
marginal (an fp decision within rounding of its threshold) are excluded from
the strict comparison and counted.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from gpu_helpers import (ATOL_RGB, ATOL_XSTAR, RTOL_RGB, RTOL_SIGMA, bits_to_bool, camera, close,
                         err_report, make_ctx, points_near_body)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ia():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_10550_b300 as ia
    ia.lib()
    return ia


@pytest.fixture(scope="module", params=["tiny", "full"])
def scene(request):
    sc = S.make_scene(request.param, 0)
    table, mlp = S.make_field(sc, 0)
    return sc, table, mlp


def _pose_ctx(ia, sc, table, mlp, seeds, early_T=0.0, precision=0):
    ctx = make_ctx(ia, torch, sc, table, mlp, early_T=early_T, precision=precision)
    poses = [S.make_pose(sc, s) for s in seeds]
    ia.ia_set_pose(ctx, np.stack([p[0] for p in poses]), np.stack([p[1] for p in poses]))
    return ctx, poses


def test_transforms_bit_exact(ia, scene):
    """The fp64 pose chain's fp32 results on 256 seeded poses.  Both sides
    take the same rounded fp64 operations in the same order, the joint
    angles' cosine and sine included (each side sums their Maclaurin series
    term by term, with the series reciprocals formed the same way, rather
    than calling a math library), so every fp32 value must match bit for bit.
    Differing elements are counted and reported before the assertion."""
    sc, table, mlp = scene
    seeds = list(range(256))
    ctx, poses = _pose_ctx(ia, sc, table, mlp, seeds)
    om = O.OracleModel(sc, table, mlp)
    nb = sc.n_bones
    differ = checked = 0
    for i, (th, tr) in enumerate(poses):
        N = np.zeros((nb, 12), np.float32)
        Ni = np.zeros((nb, 12), np.float32)
        B0 = np.zeros(12, np.float32)
        ia.ia_get_transforms(ctx, i, N, Ni, B0)
        T = om.transforms(om.pose(th, tr))
        for got, ref in ((N, T["N"].reshape(nb, 12).astype(np.float32)),
                         (Ni, T["Ninv"].reshape(nb, 12).astype(np.float32)), (B0, T["B0inv"].reshape(12))):
            differ += int(np.sum(got.view(np.int32) != ref.view(np.int32)))
            checked += got.size
    print(f"pose chain: {checked} fp32 values over {len(poses)} poses, {differ} differing")
    assert differ == 0
    ia.ia_destroy(ctx)


def test_canonical_field(ia, scene):
    sc, table, mlp = scene
    ctx = make_ctx(ia, torch, sc, table, mlp)
    om = O.OracleModel(sc, table, mlp)
    x = S.random_points(sc, 2048, seed=1, box="canon")
    # and points near the body, where the field varies
    rng = np.random.default_rng(2)
    s = rng.integers(len(sc.seg_a), size=2048)
    t = rng.uniform(size=(2048, 1))
    near = (sc.seg_a[s] + t * (sc.seg_b[s] - sc.seg_a[s]) + rng.normal(0, 0.05, (2048, 3)))
    near = np.clip(near, sc.canon_min, sc.canon_max).astype(np.float32)
    x = np.concatenate([x, near])
    xd = torch.from_numpy(x).cuda()
    sig = torch.zeros(len(x), device="cuda")
    rgb = torch.zeros(len(x), 3, device="cuda")
    ia.ia_query_canonical(ctx, xd, sig, rgb)
    torch.cuda.synchronize()
    ref = [om.field(p) for p in x.astype(np.float64)]
    rs = np.array([r[0] for r in ref])
    rc = np.array([r[1] for r in ref])
    err_report("canonical sigma", sig.cpu().numpy(), rs)
    err_report("canonical rgb", rgb.cpu().numpy(), rc)
    assert close(sig.cpu().numpy(), rs, RTOL_SIGMA, 1e-9).all()
    assert close(rgb.cpu().numpy(), rc, RTOL_RGB, ATOL_RGB).all()
    ia.ia_destroy(ctx)


def test_posed_field(ia, scene):
    sc, table, mlp = scene
    ctx, poses = _pose_ctx(ia, sc, table, mlp, [3])
    om = O.OracleModel(sc, table, mlp)
    p = om.pose(*poses[0])
    n = 1500 if sc.name == "full" else 3000
    pts = np.concatenate([points_near_body(sc, om, p, n, 5), S.random_points(sc, n // 3, seed=6)])
    xd = torch.from_numpy(pts).cuda()
    sig = torch.zeros(len(pts), device="cuda")
    rgb = torch.zeros(len(pts), 3, device="cuda")
    xc = torch.zeros(len(pts), 3, device="cuda")
    st = torch.zeros(len(pts), dtype=torch.int32, device="cuda")
    ia.ia_query_posed(ctx, 0, xd, sig, rgb, xc, st)
    torch.cuda.synchronize()
    ref = om.posed_field_many(p, pts)
    ok = ref["flags"] == 0
    print(f"posed field: {len(pts)} points, {np.sum(~ok)} flagged marginal, "
          f"{np.sum(ref['start'] >= 0)} with a root, {np.sum(ref['n_unique'] > 1)} with several")
    g_start = st.cpu().numpy()
    assert np.sum(~ok) <= 0.01 * len(pts)
    # a root exists on both sides or on neither
    np.testing.assert_array_equal(g_start[ok] >= 0, ref["start"][ok] >= 0)
    has = ok & (ref["start"] >= 0)
    g_sig, g_rgb, g_xc = sig.cpu().numpy(), rgb.cpu().numpy(), xc.cpu().numpy()
    err_report("posed sigma", g_sig[has], ref["sigma"][has])
    err_report("posed rgb", g_rgb[has], ref["rgb"][has])
    err_report("posed x*", g_xc[has], ref["xstar"][has])
    assert np.all(np.abs(g_xc[has] - ref["xstar"][has]) <= ATOL_XSTAR)
    assert close(g_sig[has], ref["sigma"][has], RTOL_SIGMA, 1e-9).all()
    # colour: the stated fp32 bound (1e-5 relative)
    n_over = int((~close(g_rgb[has], ref["rgb"][has], RTOL_RGB, ATOL_RGB)).any(axis=1).sum())
    print(f"posed field: {n_over} of {has.sum()} colours beyond 1e-5 relative")
    assert n_over == 0
    assert np.all(g_sig[ok & (ref["start"] < 0)] == 0)
    # the start label names the first start that reached the selected root; when
    # an earlier start converges only marginally the label may move to a later
    # start reaching the same root (x* compared above)
    relabel = has & (g_start != ref["start"])
    print(f"posed field: {relabel.sum()} roots reached first from another start")
    assert relabel.sum() <= 0.01 * has.sum()
    ia.ia_destroy(ctx)


def test_occupancy_bits_from_shared_density_bit_exact(ia):
    sc = S.make_scene("tiny", 0)
    table, mlp = S.make_field(sc, 0)
    ctx = make_ctx(ia, torch, sc, table, mlp)
    R = sc.occ_res
    rng = np.random.default_rng(7)
    sig = (sc.occ_tau * np.exp(rng.normal(-3.0, 2.0, R ** 3))).astype(np.float32)
    sig[rng.integers(R ** 3, size=50)] = np.float32(sc.occ_tau)  # exactly at the threshold: not occupied
    bits = torch.zeros((R ** 3 + 31) // 32, dtype=torch.int32, device="cuda")
    ia.ia_occupancy_from_density(ctx, torch.from_numpy(sig).cuda(), bits)
    torch.cuda.synchronize()
    ref = O.occ_bits_f32(R, sc.occ_dilate, sc.occ_tau, sig)
    np.testing.assert_array_equal(bits.cpu().numpy().view(np.uint32), ref)
    ia.ia_destroy(ctx)


def test_occupancy_end_to_end(ia, scene):
    sc, table, mlp = scene
    ctx, poses = _pose_ctx(ia, sc, table, mlp, [1])
    om = O.OracleModel(sc, table, mlp)
    p = om.pose(*poses[0])
    R = sc.occ_res
    sig = torch.zeros(R ** 3, device="cuda")
    bits = torch.zeros((R ** 3 + 31) // 32, dtype=torch.int32, device="cuda")
    stats = ia.ia_update_occupancy(ctx, 0, ia.IA_OCC_POSE, sig, bits, stats=True)
    ref_sig, ref_bits = om.occupancy(p)
    g_sig = sig.cpu().numpy()
    pos = ref_sig > 0
    err_report("occupancy sigma", g_sig[pos], ref_sig[pos])
    print("occupancy stats", stats)
    # densities agree where the oracle sees a root; bits agree except where a cell's
    # dilation neighbourhood holds a density within 1e-3 relative of tau
    near = _ambiguous_cells(sc, ref_sig)
    g_occ = bits_to_bool(bits.cpu().numpy().view(np.uint32), R ** 3)
    r_occ = bits_to_bool(ref_bits, R ** 3)
    mism = (g_occ != r_occ) & ~near
    print(f"occupancy: {g_occ.sum()} occupied, {near.sum()} cells excluded as ambiguous")
    assert mism.sum() == 0
    assert g_occ.sum() > 0
    ia.ia_destroy(ctx)


def _render_case(ia, sc, table, mlp, seed, early_T, width=None, height=None):
    """A context and the oracle on one pose, both over the oracle's occupancy
    grid: the GPU builds its own grid first (which also builds the pose's
    root-culling masks that the render uses), then the oracle's bits replace it."""
    ctx, poses = _pose_ctx(ia, sc, table, mlp, [seed], early_T=early_T)
    om = O.OracleModel(sc, table, mlp, early_T=early_T)
    p = om.pose(*poses[0])
    ia.ia_update_occupancy(ctx, 0, ia.IA_OCC_POSE)
    _, occ = om.occupancy(p)
    ia.ia_set_occupancy(ctx, occ)
    cam = S.make_camera(sc, width, height)
    return ctx, om, p, occ, cam


def _ambiguous_cells(sc, ref_sig):
    """Cells whose dilation neighbourhood holds a density within 1e-3
    relative of tau: their occupancy bit is an fp32-vs-fp64 coin flip."""
    R, d = sc.occ_res, sc.occ_dilate
    amb3 = (np.abs(ref_sig - sc.occ_tau) < 1e-3 * sc.occ_tau).reshape(R, R, R)
    near = np.zeros_like(amb3)
    for dz in range(-d, d + 1):
        for dy in range(-d, d + 1):
            for dx in range(-d, d + 1):
                near |= np.roll(amb3, (dz, dy, dx), axis=(0, 1, 2))
    return near.reshape(-1)


def test_render_end_to_end_chain(ia, scene):
    """The whole chain on each side with nothing shared but the inputs: the
    GPU's pose chain, occupancy grid (its own densities, threshold, dilation;
    root culling on) and frame, against the oracle's pose chain, occupancy grid
    and frame.  The two grids must agree except in cells whose dilation
    neighbourhood holds a density within 1e-3 of tau; rays crossing such a cell
    are excluded (reported), as are rays the oracle flags.  Tiny: the whole
    frame without early termination; full size: 4000 sampled pixels of the
    540 x 540 frame with early termination at T < 1e-4."""
    sc, table, mlp = scene
    early = 0.0 if sc.name == "tiny" else 1e-4
    ctx, poses = _pose_ctx(ia, sc, table, mlp, [6], early_T=early)
    om = O.OracleModel(sc, table, mlp, early_T=early)
    p = om.pose(*poses[0])
    R = sc.occ_res
    bits = torch.zeros((R ** 3 + 31) // 32, dtype=torch.int32, device="cuda")
    ia.ia_update_occupancy(ctx, 0, ia.IA_OCC_POSE, None, bits)
    cam = S.make_camera(sc)
    W, H = cam["width"], cam["height"]
    rgb = torch.zeros(H * W, 3, device="cuda")
    alpha = torch.zeros(H * W, device="cuda")
    ia.ia_render(ctx, 0, camera(ia, cam), rgb, alpha)
    torch.cuda.synchronize()
    ref_sig, ref_bits = om.occupancy(p)
    near = _ambiguous_cells(sc, ref_sig)
    g_occ = bits_to_bool(bits.cpu().numpy().view(np.uint32), R ** 3)
    r_occ = bits_to_bool(ref_bits, R ** 3)
    assert np.sum((g_occ != r_occ) & ~near) == 0
    near_bits = np.packbits(near.astype(np.uint8), bitorder="little").view(np.uint32)
    crosses = om.march_mask(p, cam, near_bits).any(axis=1)
    if sc.name == "tiny":
        pix = np.arange(W * H)
    else:
        pix = np.random.default_rng(9).choice(W * H, 4000, replace=False)
    ref = om.render_pixels(p, cam, ref_bits, pix)
    ok = (ref["flags"] == 0) & ~crosses[pix]
    print(f"end-to-end {sc.name}: {near.sum()} ambiguous cells, {(g_occ != r_occ).sum()} differing bits; "
          f"{crosses[pix].sum()} of {len(pix)} rays cross an ambiguous cell, {(ref['flags'] != 0).sum()} flagged")
    g_rgb, g_a = rgb.cpu().numpy()[pix], alpha.cpu().numpy()[pix]
    err_report(f"end-to-end {sc.name} rgb", g_rgb[ok], ref["rgb"][ok])
    assert ok.sum() >= 0.98 * len(pix)
    assert (ref["alpha"][ok] > 0.01).sum() >= 100
    assert close(g_rgb[ok], ref["rgb"][ok], RTOL_RGB, ATOL_RGB).all()
    assert close(g_a[ok], ref["alpha"][ok], RTOL_RGB, ATOL_RGB).all()
    ia.ia_destroy(ctx)


def test_march_mask_bit_exact(ia, scene):
    sc, table, mlp = scene
    ctx, om, p, occ, cam = _render_case(ia, sc, table, mlp, 2, 0.0)
    W, H = cam["width"], cam["height"]
    words = (sc.max_samples + 31) // 32
    mask = torch.zeros(H * W * words, dtype=torch.int32, device="cuda")
    ia.ia_march_mask(ctx, 0, camera(ia, cam), mask)
    torch.cuda.synchronize()
    ref = om.march_mask(p, cam, occ)
    got = mask.cpu().numpy().view(np.uint32).reshape(H * W, words)
    print(f"march mask: {np.unpackbits(ref.view(np.uint8)).sum()} occupied samples over {H * W} rays")
    np.testing.assert_array_equal(got, ref)
    ia.ia_destroy(ctx)


PATHS = {"wavefront": 1, "fused": 0}


@pytest.mark.parametrize("path", list(PATHS))
def test_render_tiny_full_frame(ia, path):
    sc = S.make_scene("tiny", 0)
    table, mlp = S.make_field(sc, 0)
    for seed in (0, 1):
        ctx, om, p, occ, cam = _render_case(ia, sc, table, mlp, seed, 0.0)
        ia.ia_set_render_path(ctx, PATHS[path])
        W, H = cam["width"], cam["height"]
        rgb = torch.zeros(H * W, 3, device="cuda")
        alpha = torch.zeros(H * W, device="cuda")
        stats = ia.ia_render(ctx, 0, camera(ia, cam), rgb, alpha, stats=True)
        ref = om.render(p, cam, occ)
        ok = ref["flags"] == 0
        print("render stats", stats, "flagged rays", np.sum(~ok))
        assert stats["occupied_samples"] == int(ref["nsamp"].sum())
        assert stats["rays"] == W * H
        g_rgb, g_a = rgb.cpu().numpy(), alpha.cpu().numpy()
        err_report("tiny rgb", g_rgb[ok], ref["rgb"][ok])
        err_report("tiny alpha", g_a[ok], ref["alpha"][ok])
        assert np.sum(~ok) <= 0.01 * W * H
        assert close(g_rgb[ok], ref["rgb"][ok], RTOL_RGB, ATOL_RGB).all()
        assert close(g_a[ok], ref["alpha"][ok], RTOL_RGB, ATOL_RGB).all()
        ia.ia_destroy(ctx)


@pytest.mark.parametrize("path", list(PATHS))
def test_render_early_termination(ia, scene, path):
    sc, table, mlp = scene
    early = 1e-4
    if sc.name == "tiny":
        ctx, om, p, occ, cam = _render_case(ia, sc, table, mlp, 4, early)
        pix = np.arange(cam["width"] * cam["height"])
    else:
        # full 540 x 540 frame in the benchmark's configuration; pixels sampled
        ctx, om, p, occ, cam = _render_case(ia, sc, table, mlp, 4, early)
        rng = np.random.default_rng(8)
        pix = rng.choice(cam["width"] * cam["height"], 4000, replace=False)
    ia.ia_set_render_path(ctx, PATHS[path])
    W, H = cam["width"], cam["height"]
    rgb = torch.zeros(H * W, 3, device="cuda")
    alpha = torch.zeros(H * W, device="cuda")
    stats = ia.ia_render(ctx, 0, camera(ia, cam), rgb, alpha, stats=True)
    print("render stats", stats)
    ref = om.render_pixels(p, cam, occ, pix)
    if sc.name == "full":  # the sampled pixels should include plenty of hits
        hit = ref["alpha"] > 0.01
        assert hit.sum() >= 100, hit.sum()
    ok = ref["flags"] == 0
    g_rgb, g_a = rgb.cpu().numpy()[pix], alpha.cpu().numpy()[pix]
    err_report(f"{sc.name} rgb (early stop)", g_rgb[ok], ref["rgb"][ok])
    err_report(f"{sc.name} alpha (early stop)", g_a[ok], ref["alpha"][ok])
    assert np.sum(~ok) <= 0.01 * len(pix)
    assert close(g_rgb[ok], ref["rgb"][ok], RTOL_RGB, ATOL_RGB).all()
    assert close(g_a[ok], ref["alpha"][ok], RTOL_RGB, ATOL_RGB).all()
    ia.ia_destroy(ctx)


@pytest.mark.parametrize("size", [(1, 1), (37, 23), (17, 64)])
def test_render_ragged_sizes(ia, size):
    sc = S.make_scene("tiny", 0)
    table, mlp = S.make_field(sc, 0)
    W, H = size
    ctx, om, p, occ, _ = _render_case(ia, sc, table, mlp, 0, 0.0)
    cam = S.make_camera(sc)
    cam = dict(cam, width=W, height=H, cx=np.float32(cam["cx"] * W / 64), cy=np.float32(cam["cy"] * H / 64))
    rgb = torch.full((H * W, 3), -1.0, device="cuda")
    alpha = torch.full((H * W,), -1.0, device="cuda")
    stats = ia.ia_render(ctx, 0, camera(ia, cam), rgb, alpha, stats=True)
    ref = om.render(p, cam, occ)
    assert stats["rays"] == W * H
    ok = ref["flags"] == 0
    assert close(rgb.cpu().numpy()[ok], ref["rgb"][ok], RTOL_RGB, ATOL_RGB).all()
    assert close(alpha.cpu().numpy()[ok], ref["alpha"][ok], RTOL_RGB, ATOL_RGB).all()
    ia.ia_destroy(ctx)


def test_render_paths_agree(ia):
    """The wavefront schedule (kernels over arrays) and the fused one (one
    persistent kernel) compute every sample with the same device functions and
    the same explicitly rounded search arithmetic, so the 540 x 540 frames are
    bit-identical with the plain search, fp32 and fp16, and with the
    learned proposal (untrained here, so the fallback wave is large) equal but
    for the fused fallback queue's merge order, early termination on.  One context renders a small frame first and switches the
    search mode, so the sample arrays grow and are re-laid out between calls."""
    sc = S.make_scene("full", 0)
    table, mlp = S.make_field(sc, 0)
    for prec in (ia.IA_FP32, ia.IA_FP16):
        ctx, poses = _pose_ctx(ia, sc, table, mlp, [6], early_T=1e-4, precision=prec)
        ia.ia_update_occupancy(ctx, 0, ia.IA_OCC_POSE)
        small, cam = S.make_camera(sc, 64, 64), S.make_camera(sc)
        modes = [ia.IA_SEARCH_ALL_BONES]
        if prec == ia.IA_FP16:
            pc = S.proposal_config()
            ia.ia_proposal_init(ctx, ia.make_proposal_config(pc["n_levels"], pc["log2_table"], pc["level_res"],
                                                             pc["top_k"], pc["offset_weight"]))
            pt, pm = S.proposal_init(sc, pc, 3)
            ia.ia_proposal_set_params(ctx, torch.from_numpy(pt).cuda(), torch.from_numpy(S.pack_proposal(pm)).cuda())
            modes.append(ia.IA_SEARCH_PROPOSAL)
        for mode in modes:
            ia.ia_set_search(ctx, mode)
            out = {}
            for path in ("wavefront", "fused"):
                ia.ia_set_render_path(ctx, PATHS[path])
                for c in (small, cam):
                    n = c["width"] * c["height"]
                    rgb = torch.full((n, 3), -1.0, device="cuda")
                    alpha = torch.full((n,), -1.0, device="cuda")
                    st = ia.ia_render(ctx, 0, camera(ia, c), rgb, alpha, stats=True)
                out[path] = (rgb.cpu().numpy(), alpha.cpu().numpy(), st)
            (r1, a1, s1), (r0, a0, s0) = out["wavefront"], out["fused"]
            d = np.abs(r1 - r0).max()
            print(f"precision {prec} search {mode}: max |rgb diff| {d:.3g}, alpha {np.abs(a1 - a0).max():.3g}; "
                  f"samples wavefront {s1['occupied_samples']} fused {s0['occupied_samples']}")
            assert (a0 >= 0).all() and (a1 >= 0).all()
            if mode == ia.IA_SEARCH_ALL_BONES:
                # each lane of the fused kernel runs its sample's starts in
                # order, the same merge as the wavefront's: bit-identical
                np.testing.assert_array_equal(r1, r0)
                np.testing.assert_array_equal(a1, a0)
            else:
                # the fused kernel runs the fallback starts through a shared
                # queue, whose merge order may keep another start's position of
                # a root (polished to the same root within fp16 rounding)
                np.testing.assert_allclose(r1, r0, rtol=2e-3, atol=2e-4)
                np.testing.assert_allclose(a1, a0, rtol=2e-3, atol=2e-4)
                assert (r1 != r0).any(axis=1).sum() <= 1e-3 * (a0 > 0).sum()
            # the wavefront marches whole rays; the fused kernel stops marching a ray
            # at early termination
            assert s1["rays"] == s0["rays"] == cam["width"] * cam["height"]
            assert s1["early_stopped"] == s0["early_stopped"] > 0
            assert s1["occupied_samples"] >= s0["occupied_samples"]
            assert s1["marched_slots"] == s1["hit_rays"] * sc.max_samples
            # the fused search gathers at every evaluation; a wavefront item
            # gathers at its start and then only when a step leaves its cell
            assert s0["grid_gathers"] == s0["starts"] + s0["broyden_iters"]
            assert s1["starts"] <= s1["grid_gathers"] < s1["starts"] + s1["broyden_iters"]
            # samples with a selected root: counted by the wavefront's field kernel
            assert 0 < s1["rooted_samples"] <= min(s1["roots"], s1["occupied_samples"] - s1["culled"])
            assert s0["rooted_samples"] == 0
        with pytest.raises(ia.IAError) as e:
            ia.ia_set_render_path(ctx, 7)
        assert e.value.status == ia.IA_ERR_ARG
        ia.ia_destroy(ctx)


def test_render_paths_agree_over_chunks(ia):
    """A 540 x 540 frame over a full occupancy grid (culling off): every slot of
    every hit ray is a sample, far more than one chunk of the wavefront's search
    (2^21 samples), so the search and field kernels run chunk after chunk; the
    frame is bit-identical to the fused kernel's."""
    sc = S.make_scene("full", 0)
    table, mlp = S.make_field(sc, 0)
    ctx, poses = _pose_ctx(ia, sc, table, mlp, [11], early_T=1e-4)
    ia.ia_set_occupancy_culling(ctx, False)
    R = sc.occ_res
    ia.ia_set_occupancy(ctx, np.full((R ** 3 + 31) // 32, 0xFFFFFFFF, np.uint32))
    cam = S.make_camera(sc)
    n = cam["width"] * cam["height"]
    out = {}
    for path in ("wavefront", "fused"):
        ia.ia_set_render_path(ctx, PATHS[path])
        rgb = torch.full((n, 3), -1.0, device="cuda")
        alpha = torch.full((n,), -1.0, device="cuda")
        st = ia.ia_render(ctx, 0, camera(ia, cam), rgb, alpha, stats=True)
        out[path] = (rgb.cpu().numpy(), alpha.cpu().numpy(), st)
    (r1, a1, s1), (r0, a0, s0) = out["wavefront"], out["fused"]
    print(f"samples wavefront {s1['occupied_samples']} fused {s0['occupied_samples']}, "
          f"max |rgb diff| {np.abs(r1 - r0).max():.3g}")
    assert s1["occupied_samples"] == s1["hit_rays"] * sc.max_samples > 3 * 2 ** 21
    np.testing.assert_array_equal(r1, r0)
    np.testing.assert_array_equal(a1, a0)
    assert (a1 > 0).sum() > 0.05 * n
    ia.ia_destroy(ctx)


def test_render_more_slots_than_the_march_mask(ia):
    """Rays of 300 slots: more than the march's per-ray register mask holds
    (128), so the march counts and emits in two full passes.  The frame matches
    the oracle on the tiny scene (parity mode) and the fused kernel bit for bit."""
    sc = S.make_scene("tiny", 0)
    sc.max_samples = 300
    table, mlp = S.make_field(sc, 0)
    ctx, om, p, occ, cam = _render_case(ia, sc, table, mlp, 5, 0.0)
    W, H = cam["width"], cam["height"]
    out = {}
    for path in ("wavefront", "fused"):
        ia.ia_set_render_path(ctx, PATHS[path])
        rgb = torch.zeros(H * W, 3, device="cuda")
        alpha = torch.zeros(H * W, device="cuda")
        st = ia.ia_render(ctx, 0, camera(ia, cam), rgb, alpha, stats=True)
        out[path] = (rgb.cpu().numpy(), alpha.cpu().numpy(), st)
    (r1, a1, s1), (r0, a0, s0) = out["wavefront"], out["fused"]
    np.testing.assert_array_equal(r1, r0)
    np.testing.assert_array_equal(a1, a0)
    assert s1["marched_slots"] == s1["hit_rays"] * 300
    ref = om.render(p, cam, occ)
    ok = ref["flags"] == 0
    assert s1["occupied_samples"] == int(ref["nsamp"].sum())
    assert np.sum(~ok) <= 0.01 * W * H
    assert (ref["alpha"][ok] > 0.01).sum() >= 100
    assert close(r1[ok], ref["rgb"][ok], RTOL_RGB, ATOL_RGB).all()
    assert close(a1[ok], ref["alpha"][ok], RTOL_RGB, ATOL_RGB).all()
    ia.ia_destroy(ctx)


def test_render_degenerate_cases(ia):
    sc = S.make_scene("tiny", 0)
    table, mlp = S.make_field(sc, 0)
    ctx, om, p, occ, cam = _render_case(ia, sc, table, mlp, 0, 1e-4)
    W, H = cam["width"], cam["height"]
    rgb = torch.full((H * W, 3), -1.0, device="cuda")
    alpha = torch.full((H * W,), -1.0, device="cuda")
    # camera looking away from the subject: every ray misses the box
    away = dict(cam, c2w=cam["c2w"] * np.array([[1, 1, -1, 1]] * 3, dtype=np.float32))
    st = ia.ia_render(ctx, 0, camera(ia, away), rgb, alpha, stats=True)
    assert st["hit_rays"] == 0 and st["occupied_samples"] == 0
    assert torch.all(rgb == 0) and torch.all(alpha == 0)
    # an empty occupancy grid: every slot is skipped
    R = sc.occ_res
    ia.ia_set_occupancy(ctx, np.zeros((R ** 3 + 31) // 32, np.uint32))
    st = ia.ia_render(ctx, 0, camera(ia, cam), rgb, alpha, stats=True)
    assert st["occupied_samples"] == 0 and torch.all(alpha == 0)
    # a full grid: every slot of every hit ray is a sample
    ia.ia_set_occupancy(ctx, np.full((R ** 3 + 31) // 32, 0xFFFFFFFF, np.uint32))
    st = ia.ia_render(ctx, 0, camera(ia, cam), rgb, alpha, stats=True)
    assert st["marched_slots"] >= st["occupied_samples"] > 0
    ia.ia_destroy(ctx)


def test_render_into_host_buffers(ia):
    sc = S.make_scene("tiny", 0)
    table, mlp = S.make_field(sc, 0)
    ctx, om, p, occ, cam = _render_case(ia, sc, table, mlp, 1, 1e-4)
    W, H = cam["width"], cam["height"]
    rgb = torch.zeros(H * W, 3, device="cuda")
    alpha = torch.zeros(H * W, device="cuda")
    ia.ia_render(ctx, 0, camera(ia, cam), rgb, alpha)
    h_rgb = np.zeros((H * W, 3), np.float32)
    h_a = np.zeros(H * W, np.float32)
    ia.ia_render(ctx, 0, camera(ia, cam), h_rgb, h_a)
    np.testing.assert_array_equal(h_rgb, rgb.cpu().numpy())
    np.testing.assert_array_equal(h_a, alpha.cpu().numpy())
    ia.ia_destroy(ctx)


def test_errors_are_status_codes(ia):
    sc = S.make_scene("tiny", 0)
    table, mlp = S.make_field(sc, 0)
    ctx = make_ctx(ia, torch, sc, table, mlp)
    cam = camera(ia, S.make_camera(sc))
    rgb = torch.zeros(64 * 64, 3, device="cuda")
    a = torch.zeros(64 * 64, device="cuda")
    with pytest.raises(ia.IAError) as e:
        ia.ia_render(ctx, 0, cam, rgb, a)
    assert e.value.status == ia.IA_ERR_STATE  # no pose yet
    th, tr = S.make_pose(sc, 0)
    bad = th.copy()
    bad[2, 1] = np.nan
    with pytest.raises(ia.IAError) as e:
        ia.ia_set_pose(ctx, bad[None], tr[None])
    assert e.value.status == ia.IA_ERR_ARG
    ia.ia_set_pose(ctx, th[None], tr[None])
    with pytest.raises(ia.IAError) as e:
        ia.ia_render(ctx, 0, cam, rgb, a)
    assert e.value.status == ia.IA_ERR_STATE  # no occupancy grid yet
    with pytest.raises(ia.IAError) as e:
        ia.ia_update_occupancy(ctx, 3)
    assert e.value.status == ia.IA_ERR_ARG
    parents = sc.parents.copy()
    parents[3] = 5  # child before parent
    with pytest.raises(ia.IAError) as e:
        ia.ia_set_skeleton(ctx, parents, sc.rest_joints, sc.skin_grid, sc.canon_min, sc.canon_max,
                           sc.norm_min, sc.norm_max)
    assert e.value.status == ia.IA_ERR_ARG
    ia.ia_destroy(ctx)


def test_measurement_probes(ia):
    """The bench's roofline denominators: random gathers of every record size
    run and leave the table alone; random vector atomics add their count times
    the increment to the table's total (to fp32 rounding)."""
    sink = torch.zeros(1, device="cuda")
    for rb in (4, 8, 16, 48):
        table = torch.rand(4096 * rb // 4, device="cuda")
        before = table.clone()
        ia.ia_gather_probe(table, 4096, 16, 4, sink, record_bytes=rb)
        torch.cuda.synchronize()
        assert torch.equal(table, before)
    for rb in (8, 16):
        table = torch.zeros(1000 * rb // 4, device="cuda")
        ia.ia_atomic_probe(table, 1000, 16, 4, record_bytes=rb)
        torch.cuda.synchronize()
        total = float(table.double().sum().item())
        expect = 4 * 256 * 16 * (rb // 4) * 1e-7
        assert abs(total - expect) <= 1e-3 * expect
    with pytest.raises(ia.IAError) as e:
        ia.ia_gather_probe(torch.zeros(16, device="cuda"), 4, 1, 1, sink, record_bytes=12)
    assert e.value.status == ia.IA_ERR_ARG
