"""GPU training step (ia_train_step) against the fp64 oracle's loss and gradient.

Both sides composite every occupied sample (no early termination) over the same
occupancy grid (the oracle's union over the batch's poses, installed on the GPU
as the render grid) and the same seeded rays.  Rays the oracle flags as marginal
are removed from the batch before the comparison.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from gpu_helpers import ATOL_RGB, RTOL_RGB, camera, close, make_ctx, points_near_body
from oracle import grad as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# Gradient tolerance: fp32 accumulation in a different order (atomics) and fp32
# roots/activations against fp64; compared per parameter group as a relative L2
# error and per element against the group's scale.
GRAD_REL_L2 = 2e-3
GRAD_ELEM = 1e-3


@pytest.fixture(scope="module")
def ia():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_10550_b300 as ia
    ia.lib()
    return ia


def _case(config, n_poses, n_rays):
    sc = S.make_scene(config, 0)
    table, mlp = S.make_field(sc, 0)
    om = O.OracleModel(sc, table, mlp)
    poses = [S.make_pose(sc, i) for i in range(n_poses)]
    op = [om.pose(*p) for p in poses]
    occ = np.zeros((sc.occ_res ** 3 + 31) // 32, np.uint32)
    for p in op:
        occ |= om.occupancy(p)[1]
    rb = S.make_ray_batch(sc, n_rays, n_poses, seed=2)
    _, _, flags, _ = G.train(om, op, occ, rb["origin"], rb["direction"], rb["pose"], rb["target"], grad=False)
    keep = flags == 0
    rays = {k: rb[k][keep] for k in ("origin", "direction", "pose", "target")}
    return sc, table, mlp, om, poses, op, occ, rays, int((~keep).sum())


def _run_gpu(ia, sc, table, mlp, poses, occ, rays):
    ctx = make_ctx(ia, torch, sc, table, mlp)
    ia.ia_set_pose(ctx, np.stack([p[0] for p in poses]), np.stack([p[1] for p in poses]))
    ia.ia_set_occupancy(ctx, occ)
    nt, nm = ia.ia_param_sizes(ctx)
    g = dict(table=torch.zeros(nt, device="cuda"), mlp=torch.zeros(nm, device="cuda"),
             skin=torch.zeros(sc.skin_res ** 3 * sc.n_bones, device="cuda"),
             bones=torch.zeros(len(poses) * sc.n_bones * 12, device="cuda"))
    dev = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in rays.items()}
    loss = torch.zeros(1, device="cuda")
    rgb = torch.zeros(len(rays["pose"]), 3, device="cuda")
    ia.ia_train_step(ctx, dev["origin"], dev["direction"], dev["pose"], dev["target"], loss, g,
                     occ_grid=ia.IA_OCC_POSE, rgb_out=rgb)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}
    # a second step on the same inputs overwrites the gradients with the same values
    loss2 = torch.zeros(1, device="cuda")
    ia.ia_train_step(ctx, dev["origin"], dev["direction"], dev["pose"], dev["target"], loss2, g,
                     occ_grid=ia.IA_OCC_POSE)
    torch.cuda.synchronize()
    again = {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}
    ia.ia_destroy(ctx)
    return float(loss.item()), float(loss2.item()), rgb.cpu().numpy(), out, again


def _compare(sc, om, op, occ, rays, gpu):
    loss, loss2, rgb, g, g2 = gpu
    ref_loss, ref_rgb, _, ref = G.train(om, op, occ, rays["origin"], rays["direction"], rays["pose"],
                                        rays["target"])
    print(f"loss gpu {loss:.8e} oracle {ref_loss:.8e}")
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    assert abs(loss2 - loss) <= 1e-6 * loss
    assert close(rgb, ref_rgb, RTOL_RGB, ATOL_RGB).all()
    ref_flat = {k: v.reshape(-1) for k, v in ref.items()}
    for k in ("table", "mlp", "skin", "bones"):
        a, b = g[k], ref_flat[k]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        worst = np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)
        print(f"grad {k}: rel L2 {rel:.2e}, worst element / scale {worst:.2e}, nonzero {np.count_nonzero(b)}")
        assert np.count_nonzero(b) > 0
        assert rel <= GRAD_REL_L2, k
        assert worst <= GRAD_ELEM, k
        np.testing.assert_allclose(g2[k], a, rtol=1e-3, atol=1e-6 * max(np.abs(b).max(), 1e-30))


def test_train_step_tiny(ia):
    sc, table, mlp, om, poses, op, occ, rays, dropped = _case("tiny", 2, 3000)
    print(f"{len(rays['pose'])} rays, {dropped} flagged rays dropped")
    _compare(sc, om, op, occ, rays, _run_gpu(ia, sc, table, mlp, poses, occ, rays))


def test_train_step_full_size(ia):
    sc, table, mlp, om, poses, op, occ, rays, dropped = _case("full", 4, 2048)
    print(f"{len(rays['pose'])} rays, {dropped} flagged rays dropped")
    _compare(sc, om, op, occ, rays, _run_gpu(ia, sc, table, mlp, poses, occ, rays))


def test_train_step_bad_pose_index_is_an_empty_ray(ia):
    sc, table, mlp, om, poses, op, occ, rays, _ = _case("tiny", 2, 500)
    rays = {k: v.copy() for k, v in rays.items()}
    rays["pose"][:10] = 7  # only poses 0 and 1 exist
    _, _, rgb, _, _ = _run_gpu(ia, sc, table, mlp, poses, occ, rays)
    assert np.all(rgb[:10] == 0)


def _round_fp16(x):
    return np.asarray(x, np.float32).astype(np.float16).astype(np.float32)


@pytest.mark.parametrize("config,n_poses,n_rays,prec", [("tiny", 2, 1500, 0), ("full", 4, 2048, 0),
                                                        ("tiny", 2, 1500, 1)])
def test_autograd_backward_of_a_torch_loss(ia, config, n_poses, n_rays, prec):
    """A loss built in torch on the differentiable render (autograd.render_rays:
    ia_train_forward, then ia_train_backward with the incoming dL/drgb and
    dL/dalpha): a weighted L1 of the colour to a target plus a weighted squared
    error of the opacity, back-propagated by loss.backward(), against the
    oracle's backward of the same loss (or_train_upstream given that loss's
    dL/dC and dL/dalpha at the oracle's own forward).  The targets sit at least
    0.05 from the oracle's colour in every channel, so the L1 signs are the same
    on both sides.  fp32 at the fp32 gradient bounds; fp16 (fp16 shadow of the
    caller's table, fp16 MLP operands, loss scaling) against the oracle on the
    fp16-rounded operands at the fp16 bound (1e-2 relative L2)."""
    from paper_2212_10550_b300.autograd import Field, render_rays
    sc, table, mlp, om, poses, op, occ, rays, _ = _case(config, n_poses, n_rays)
    if prec:
        t_op = _round_fp16(table)
        m_op = {k: (_round_fp16(v) if k.startswith("W") else v) for k, v in mlp.items()}
        om = O.OracleModel(sc, t_op, m_op)
        op = [om.pose(*p) for p in poses]
    n = len(rays["pose"])
    rng = np.random.default_rng(21)
    ref_rgb, ref_a, flags, _ = G.train_upstream(om, op, occ, rays["origin"], rays["direction"], rays["pose"])
    assert np.all(flags == 0)
    tgt = ref_rgb + rng.choice([-1.0, 1.0], size=(n, 3)) * rng.uniform(0.05, 0.3, size=(n, 3))
    mask = rng.uniform(0, 1, n)
    w = rng.uniform(0.5, 2.0, size=(n, 3)) / n
    v = rng.uniform(0.5, 2.0, size=n) / n
    up_rgb = w * np.sign(ref_rgb - tgt)
    up_a = 2 * v * (ref_a - mask)
    _, _, _, ref = G.train_upstream(om, op, occ, rays["origin"], rays["direction"], rays["pose"], up_rgb, up_a)

    cfg = ia.make_config(n_levels=sc.n_levels, log2_table=sc.log2_table, level_res=sc.level_res,
                         max_samples=sc.max_samples, broyden_max_iter=sc.broyden_max_iter,
                         broyden_tol=sc.broyden_tol, occ_res=sc.occ_res, occ_tau=sc.occ_tau,
                         occ_dilate=sc.occ_dilate, early_stop_T=0.0, precision=prec)
    ctx = ia.ia_create(cfg)
    ia.ia_set_skeleton(ctx, sc.parents, sc.rest_joints, sc.skin_grid, sc.canon_min, sc.canon_max,
                       sc.norm_min, sc.norm_max)
    zeros_t, zeros_m = np.zeros_like(table), np.zeros_like(S.pack_mlp(mlp))
    ia.ia_set_params(ctx, torch.from_numpy(zeros_t).cuda(), torch.from_numpy(zeros_m).cuda())  # unused
    ia.ia_set_pose(ctx, np.stack([p[0] for p in poses]), np.stack([p[1] for p in poses]))
    ia.ia_set_occupancy(ctx, occ)
    field = Field(ctx, ia.IA_OCC_POSE)
    dev = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in rays.items()}
    t = torch.from_numpy(np.ascontiguousarray(table).reshape(-1)).cuda().requires_grad_()
    m = torch.from_numpy(S.pack_mlp(mlp)).cuda().requires_grad_()
    ns, nbn = ia.ia_grad_sizes(ctx)
    skin = torch.zeros(ns, device="cuda", requires_grad=True)
    bones = torch.zeros(nbn, device="cuda", requires_grad=True)
    rgb, alpha = render_rays(field, t, m, skin, bones, dev["origin"], dev["direction"], dev["pose"])
    T = {k: torch.from_numpy(x).cuda().float() for k, x in (("tgt", tgt), ("mask", mask), ("w", w), ("v", v))}
    loss = (T["w"] * (rgb - T["tgt"]).abs()).sum() + (T["v"] * (alpha - T["mask"]) ** 2).sum()
    loss.backward(retain_graph=True)
    got = {"table": t.grad.clone(), "mlp": m.grad.clone(), "skin": skin.grad.clone(), "bones": bones.grad.clone()}
    # a second backward of the same forward gives the same gradients
    for x in (t, m, skin, bones):
        x.grad = None
    loss.backward(retain_graph=True)
    again = {"table": t.grad, "mlp": m.grad, "skin": skin.grad, "bones": bones.grad}
    torch.cuda.synchronize()
    rtol = RTOL_RGB if prec == 0 else 2e-3
    atol = ATOL_RGB if prec == 0 else 2e-4
    assert close(rgb.detach().cpu().numpy(), ref_rgb, rtol, atol).all()
    assert close(alpha.detach().cpu().numpy(), ref_a, rtol, atol).all()
    tol_rel, tol_elem = (GRAD_REL_L2, GRAD_ELEM) if prec == 0 else (1e-2, 2e-2)
    for k in ("table", "mlp", "skin", "bones"):
        a = got[k].cpu().numpy().astype(np.float64)
        b = ref[k].reshape(-1)
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        worst = np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)
        print(f"{config} prec {prec} autograd grad {k}: rel L2 {rel:.2e}, worst element / scale {worst:.2e}")
        assert np.count_nonzero(b) > 0
        assert rel <= tol_rel, k
        assert worst <= tol_elem, k
        np.testing.assert_allclose(again[k].cpu().numpy(), a, rtol=1e-3, atol=1e-6 * np.abs(b).max())
    # the per-sample state belongs to the latest forward: a backward of an older one is refused
    rgb2, alpha2 = render_rays(field, t, m, skin, bones, dev["origin"], dev["direction"], dev["pose"])
    with pytest.raises(ia.IAError):
        rgb.sum().backward()
    rgb2.sum().backward()
    ia.ia_destroy(ctx)


def test_loss_set_matches_oracle(ia):
    """Huber colour loss (Eq. 9), alpha L1 to a mask (Eq. 10) and the hard-surface
    term (Eq. 11) together, against the oracle's loss set."""
    sc, table, mlp, om, poses, op, occ, rays, _ = _case("tiny", 2, 3000)
    alpha_gt = np.random.default_rng(12).uniform(0, 1, len(rays["pose"]))
    cfg = dict(huber=1, delta=0.8, w_rgb=1.0, w_alpha=0.7, w_hard=0.3, alpha_target=alpha_gt)
    ref_loss, _, _, ref = G.train(om, op, occ, rays["origin"], rays["direction"], rays["pose"], rays["target"],
                                  loss=cfg)
    ctx = make_ctx(ia, torch, sc, table, mlp)
    ia.ia_set_pose(ctx, np.stack([p[0] for p in poses]), np.stack([p[1] for p in poses]))
    ia.ia_set_occupancy(ctx, occ)
    ia.ia_set_loss(ctx, ia.IA_LOSS_HUBER, 0.8, 1.0, 0.7, 0.3)
    nt, nm = ia.ia_param_sizes(ctx)
    g = dict(table=torch.zeros(nt, device="cuda"), mlp=torch.zeros(nm, device="cuda"),
             skin=torch.zeros(sc.skin_res ** 3 * sc.n_bones, device="cuda"),
             bones=torch.zeros(len(poses) * sc.n_bones * 12, device="cuda"))
    dev = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in rays.items()}
    loss = torch.zeros(1, device="cuda")
    ia.ia_train_step(ctx, dev["origin"], dev["direction"], dev["pose"], dev["target"], loss, g,
                     occ_grid=ia.IA_OCC_POSE, alpha_target=torch.from_numpy(alpha_gt.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    ia.ia_destroy(ctx)
    print(f"loss set: gpu {loss.item():.8e} oracle {ref_loss:.8e}")
    assert abs(loss.item() - ref_loss) <= 1e-5 * ref_loss
    for k in ("table", "mlp", "skin", "bones"):
        a, b = g[k].cpu().numpy().astype(np.float64), ref[k].reshape(-1)
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        worst = np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)
        print(f"grad {k}: rel L2 {rel:.2e}, worst element / scale {worst:.2e}")
        assert rel <= GRAD_REL_L2 and worst <= GRAD_ELEM, k


@pytest.mark.parametrize("prec", [0, 1])
def test_adam_step_matches_its_definition(ia, prec):
    """Two Adam steps on the context's table and MLP against the update rule
    written out in numpy (fp64)."""
    sc = S.make_scene("tiny", 0)
    table, mlp = S.make_field(sc, 0)
    cfg = ia.make_config(n_levels=sc.n_levels, log2_table=sc.log2_table, level_res=sc.level_res,
                         max_samples=sc.max_samples, precision=prec)
    ctx = ia.ia_create(cfg)
    ia.ia_set_skeleton(ctx, sc.parents, sc.rest_joints, sc.skin_grid, sc.canon_min, sc.canon_max,
                       sc.norm_min, sc.norm_max)
    p0 = [np.ascontiguousarray(table).reshape(-1).astype(np.float64), S.pack_mlp(mlp).astype(np.float64)]
    ia.ia_set_params(ctx, torch.from_numpy(np.ascontiguousarray(table)).cuda(), torch.from_numpy(S.pack_mlp(mlp)).cuda())
    rng = np.random.default_rng(7)
    grads = [[rng.normal(0, s, p.shape) for p, s in zip(p0, (1e-3, 1e-2))] for _ in range(2)]
    lr, b1, b2, eps = 1e-2, 0.9, 0.99, 1e-15
    for gt, gm in grads:
        ia.ia_adam_step(ctx, torch.from_numpy(gt.astype(np.float32)).cuda(), torch.from_numpy(gm.astype(np.float32)).cuda(),
                        lr, b1, b2, eps)
    nt, nm = ia.ia_param_sizes(ctx)
    t_out, m_out = np.zeros(nt, np.float32), np.zeros(nm, np.float32)
    ia.ia_get_params(ctx, t_out, m_out)
    ia.ia_destroy(ctx)
    for p, out, gs in ((p0[0], t_out, [g[0] for g in grads]), (p0[1], m_out, [g[1] for g in grads])):
        m = np.zeros_like(p)
        v = np.zeros_like(p)
        x = p.copy()
        for t, gg in enumerate(gs, start=1):
            gg = gg.astype(np.float32).astype(np.float64)
            m = b1 * m + (1 - b1) * gg
            v = b2 * v + (1 - b2) * gg * gg
            x = x - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
        np.testing.assert_allclose(out, x, rtol=1e-5, atol=1e-6 * lr)


def test_skinning_grid_step_before_any_pose(ia):
    """An Adam step on the skinning grid before any pose is set updates the grid
    and leaves the context whole: no blended grid to rebuild yet, and setting a
    pose afterwards builds it from the updated weights (the render then runs)."""
    sc = S.make_scene("tiny", 0)
    table, mlp = S.make_field(sc, 0)
    ctx = make_ctx(ia, torch, sc, table, mlp)
    nt, nm = ia.ia_param_sizes(ctx)
    ns, _ = ia.ia_grad_sizes(ctx)
    gs = np.random.default_rng(4).normal(0, 1e-3, ns).astype(np.float32)
    ia.ia_adam_step(ctx, torch.zeros(nt, device="cuda"), torch.zeros(nm, device="cuda"), 1e-3, 0.9, 0.99, 1e-15,
                    g_skin=torch.from_numpy(gs).cuda())
    torch.cuda.synchronize()
    pose = S.make_pose(sc, 3)
    ia.ia_set_pose(ctx, pose[0][None], pose[1][None])
    ia.ia_update_occupancy(ctx, 0)
    cam = S.make_camera(sc)
    n = cam["width"] * cam["height"]
    rgb, alpha = torch.zeros(n, 3, device="cuda"), torch.zeros(n, device="cuda")
    st = ia.ia_render(ctx, 0, camera(ia, cam), rgb, alpha, stats=True)
    torch.cuda.synchronize()
    assert st["rays"] == n and (alpha > 0).any()
    ia.ia_destroy(ctx)


def test_learnable_skinning_grid(ia):
    """With g_skin the Adam step moves the skinning-weight grid (checked against
    the update rule) and rebuilds the blended grids: a posed query afterwards
    equals the oracle's on the updated weights."""
    sc = S.make_scene("tiny", 0)
    table, mlp = S.make_field(sc, 0)
    pose = S.make_pose(sc, 3)
    ctx = make_ctx(ia, torch, sc, table, mlp)
    ia.ia_set_pose(ctx, pose[0][None], pose[1][None])
    nt, nm = ia.ia_param_sizes(ctx)
    ns, _ = ia.ia_grad_sizes(ctx)
    rng = np.random.default_rng(9)
    gs = rng.normal(0, 1e-3, ns)
    lr = 2e-3
    ia.ia_adam_step(ctx, torch.zeros(nt, device="cuda"), torch.zeros(nm, device="cuda"), lr, 0.9, 0.99, 1e-15,
                    g_skin=torch.from_numpy(gs.astype(np.float32)).cuda())
    # one bias-corrected Adam step moves every weight by -lr * g / (|g| + eps / ...) = -lr * sign(g)
    skin_new = (sc.skin_grid.reshape(-1).astype(np.float64) - lr * np.sign(gs)).reshape(sc.skin_grid.shape)
    om = O.OracleModel(sc, table, mlp, skin=skin_new)
    p = om.pose(*pose)
    x = points_near_body(sc, om, p, 1500, 21)
    sig = torch.zeros(len(x), device="cuda")
    xc = torch.zeros(len(x), 3, device="cuda")
    st = torch.zeros(len(x), dtype=torch.int32, device="cuda")
    ia.ia_query_posed(ctx, 0, torch.from_numpy(x).cuda(), sig, None, xc, st)
    torch.cuda.synchronize()
    ia.ia_destroy(ctx)
    g_xc, g_st = xc.cpu().numpy(), st.cpu().numpy()
    n_ok = 0
    for j in range(len(x)):
        r = om.posed_field(p, x[j].astype(np.float64))
        if r["flags"] or r["start"] < 0:
            continue
        assert g_st[j] >= 0
        assert np.all(np.abs(g_xc[j] - r["xstar"]) <= 2e-5), j
        n_ok += 1
    print(f"{n_ok} posed queries on the updated skinning grid match the oracle")
    assert n_ok > 100


def test_gradient_buffer_alignment(ia):
    """A skinning-grid gradient buffer 4 bytes off a 16-byte boundary takes the
    one-bone-at-a-time scatter: same gradients as the four-bone vector atomics
    up to summation order.  A hash-table gradient buffer that is not 8-byte
    aligned is refused before any launch."""
    sc, table, mlp, om, poses, op, occ, rays, _ = _case("full", 2, 1024)
    ctx = make_ctx(ia, torch, sc, table, mlp)
    ia.ia_set_pose(ctx, np.stack([p[0] for p in poses]), np.stack([p[1] for p in poses]))
    ia.ia_set_occupancy(ctx, occ)
    nt, nm = ia.ia_param_sizes(ctx)
    ns, nbn = ia.ia_grad_sizes(ctx)
    dev = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in rays.items()}
    out = []
    for shift in (0, 1):
        skin_buf = torch.zeros(ns + 4, device="cuda")
        g = dict(table=torch.zeros(nt, device="cuda"), mlp=torch.zeros(nm, device="cuda"),
                 skin=skin_buf[shift:shift + ns], bones=torch.zeros(nbn, device="cuda"))
        loss = torch.zeros(1, device="cuda")
        ia.ia_train_step(ctx, dev["origin"], dev["direction"], dev["pose"], dev["target"], loss, g,
                         occ_grid=ia.IA_OCC_POSE)
        torch.cuda.synchronize()
        out.append({k: v.cpu().numpy().astype(np.float64) for k, v in g.items()})
    for k in ("table", "mlp", "skin", "bones"):
        a, b = out[1][k], out[0][k]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        print(f"{k}: rel L2 {rel:.2e}")
        assert np.count_nonzero(b) > 0 and rel <= 1e-5, k
    bad = torch.zeros(nt + 1, device="cuda")
    g = dict(table=bad[1:], mlp=torch.zeros(nm, device="cuda"), skin=torch.zeros(ns, device="cuda"),
             bones=torch.zeros(nbn, device="cuda"))
    with pytest.raises(ia.IAError) as e:
        ia.ia_train_step(ctx, dev["origin"], dev["direction"], dev["pose"], dev["target"], torch.zeros(1, device="cuda"),
                         g, occ_grid=ia.IA_OCC_POSE)
    assert e.value.status == ia.IA_ERR_ARG
    ia.ia_destroy(ctx)
