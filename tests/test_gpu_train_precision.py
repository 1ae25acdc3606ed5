"""Reduced-precision training step (fp16 / bf16 MLP operands and fp16 hash
features, fp32 accumulation, fp32 master gradients, loss scaling) against the
fp64 oracle's loss and gradient.

The oracle runs on the parameters the reduced-precision forward actually reads:
the hash table rounded to fp16 (the shadow table) and the MLP weights rounded to
the operand type (biases stay fp32).  What remains is the rounding of the
features, the two hidden activations and the three scaled gradients (dO, dH2,
dH1): six roundings of unit roundoff u (2^-11 fp16, 2^-8 bf16) on the path of
every gradient.  Density is exp(o0), so a relative error e in o0's inputs gives
~e |o0| (|o0| <= ~6 here) relative density error, and every compositing weight
of the ray inherits it: about 6 * 6u ~ 2e-2 (fp16) and 1.4e-1 (bf16) per sample
at worst, far less in an L2 norm over many samples.  The bounds below are 1e-2
relative L2 (fp16) and 6e-2 (bf16) per parameter group, and the loss within
5e-3 / 3e-2.  Root finding and skinning stay fp32, so the samples and roots are
those of the fp32 path.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from gpu_helpers import close, make_ctx
from oracle import grad as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NAMES = {1: "fp16", 2: "bf16"}
TOL = {1: dict(loss=5e-3, grad=1e-2), 2: dict(loss=3e-2, grad=6e-2)}


@pytest.fixture(scope="module")
def ia():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_10550_b300 as ia
    ia.lib()
    return ia


def _round_fp16(x):
    return np.asarray(x, np.float32).astype(np.float16).astype(np.float32)


def _round_bf16(x):
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def _operands(table, mlp, prec):
    rw = _round_fp16 if prec == 1 else _round_bf16
    m = {k: (rw(v) if k.startswith("W") else np.asarray(v, np.float32)) for k, v in mlp.items()}
    return _round_fp16(table), m


def _ctx(ia, sc, table, mlp, prec):
    cfg = ia.make_config(n_levels=sc.n_levels, log2_table=sc.log2_table, level_res=sc.level_res,
                         max_samples=sc.max_samples, broyden_max_iter=sc.broyden_max_iter,
                         broyden_tol=sc.broyden_tol, occ_res=sc.occ_res, occ_tau=sc.occ_tau,
                         occ_dilate=sc.occ_dilate, early_stop_T=0.0, precision=prec)
    ctx = ia.ia_create(cfg)
    ia.ia_set_skeleton(ctx, sc.parents, sc.rest_joints, sc.skin_grid, sc.canon_min, sc.canon_max,
                       sc.norm_min, sc.norm_max)
    ia.ia_set_params(ctx, torch.from_numpy(np.ascontiguousarray(table)).cuda(),
                     torch.from_numpy(S.pack_mlp(mlp)).cuda())
    return ctx


def _grads(ia, ctx, sc, n_poses):
    nt, nm = ia.ia_param_sizes(ctx)
    return dict(table=torch.zeros(nt, device="cuda"), mlp=torch.zeros(nm, device="cuda"),
                skin=torch.zeros(sc.skin_res ** 3 * sc.n_bones, device="cuda"),
                bones=torch.zeros(n_poses * sc.n_bones * 12, device="cuda"))


def _dev(rays):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in rays.items()}


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("config,n_poses,n_rays", [("tiny", 2, 3000), ("full", 4, 2048)])
def test_train_step_reduced_precision(ia, prec, config, n_poses, n_rays):
    sc = S.make_scene(config, 0)
    table, mlp = S.make_field(sc, 0)
    t_op, m_op = _operands(table, mlp, prec)
    om = O.OracleModel(sc, t_op, m_op)
    poses = [S.make_pose(sc, i) for i in range(n_poses)]
    op = [om.pose(*p) for p in poses]
    occ = np.zeros((sc.occ_res ** 3 + 31) // 32, np.uint32)
    for p in op:
        occ |= om.occupancy(p)[1]
    rb = S.make_ray_batch(sc, n_rays, n_poses, seed=2)
    _, _, flags, _ = G.train(om, op, occ, rb["origin"], rb["direction"], rb["pose"], rb["target"], grad=False)
    keep = flags == 0
    rays = {k: rb[k][keep] for k in ("origin", "direction", "pose", "target")}

    ctx = _ctx(ia, sc, table, mlp, prec)  # fp32 master parameters
    ia.ia_set_pose(ctx, np.stack([p[0] for p in poses]), np.stack([p[1] for p in poses]))
    ia.ia_set_occupancy(ctx, occ)
    g = _grads(ia, ctx, sc, n_poses)
    dev = _dev(rays)
    loss = torch.zeros(1, device="cuda")
    ia.ia_train_step(ctx, dev["origin"], dev["direction"], dev["pose"], dev["target"], loss, g,
                     occ_grid=ia.IA_OCC_POSE)
    scale, skipped = ia.ia_loss_scale(ctx)
    st = ia.ia_train_stats(ctx)
    torch.cuda.synchronize()
    ia.ia_destroy(ctx)
    assert not skipped
    # plain search: every searched sample (occupied and not culled: culled ones can
    # have no root) runs every bone-wise start
    assert st["rays"] == keep.sum() and st["occupied_samples"] > 0
    assert st["starts"] == sc.n_bones * (st["occupied_samples"] - st["culled"])
    assert st["proposed"] == 0 and st["fallbacks"] == 0
    assert scale == (16384.0 if prec == 1 else 1.0)

    ref_loss, _, _, ref = G.train(om, op, occ, rays["origin"], rays["direction"], rays["pose"], rays["target"])
    lg = float(loss.item())
    print(f"{NAMES[prec]} {config}: {keep.sum()} rays, loss gpu {lg:.6e} oracle {ref_loss:.6e} "
          f"rel {abs(lg - ref_loss) / ref_loss:.2e}")
    assert abs(lg - ref_loss) <= TOL[prec]["loss"] * ref_loss
    for k in ("table", "mlp", "skin", "bones"):
        a = g[k].cpu().numpy().astype(np.float64)
        b = ref[k].reshape(-1)
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        print(f"  grad {k}: rel L2 {rel:.2e}")
        assert np.count_nonzero(b) > 0
        assert rel <= TOL[prec]["grad"], k


def test_mlp_weight_gradient_blocks(ia):
    """Each block of the tensor-core weight-gradient GEMM (dW1, db1, dW2, db2,
    dW3, db3) against the oracle separately, fp16, tiny scene."""
    sc = S.make_scene("tiny", 0)
    table, mlp = S.make_field(sc, 0)
    t_op, m_op = _operands(table, mlp, 1)
    om = O.OracleModel(sc, t_op, m_op)
    poses = [S.make_pose(sc, i) for i in range(2)]
    op = [om.pose(*p) for p in poses]
    occ = np.zeros((sc.occ_res ** 3 + 31) // 32, np.uint32)
    for p in op:
        occ |= om.occupancy(p)[1]
    rb = S.make_ray_batch(sc, 3000, 2, seed=5)
    _, _, flags, _ = G.train(om, op, occ, rb["origin"], rb["direction"], rb["pose"], rb["target"], grad=False)
    keep = flags == 0
    rays = {k: rb[k][keep] for k in ("origin", "direction", "pose", "target")}
    ctx = _ctx(ia, sc, table, mlp, 1)
    ia.ia_set_pose(ctx, np.stack([p[0] for p in poses]), np.stack([p[1] for p in poses]))
    ia.ia_set_occupancy(ctx, occ)
    g = _grads(ia, ctx, sc, 2)
    dev = _dev(rays)
    ia.ia_train_step(ctx, dev["origin"], dev["direction"], dev["pose"], dev["target"],
                     torch.zeros(1, device="cuda"), g, occ_grid=ia.IA_OCC_POSE)
    torch.cuda.synchronize()
    ia.ia_destroy(ctx)
    _, _, _, ref = G.train(om, op, occ, rays["origin"], rays["direction"], rays["pose"], rays["target"])
    a, b = g["mlp"].cpu().numpy().astype(np.float64), ref["mlp"].reshape(-1)
    n_in, w = sc.mlp_in(), sc.mlp_width
    sizes = [("W1", w * n_in), ("b1", w), ("W2", w * w), ("b2", w), ("W3", 4 * w), ("b3", 4)]
    off = 0
    for name, n in sizes:
        x, y = a[off:off + n], b[off:off + n]
        rel = np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-30)
        print(f"d{name}: rel L2 {rel:.2e}")
        assert rel <= TOL[1]["grad"], name
        off += n
    assert off == len(b)


def test_overflow_skips_the_step_and_halves_the_scale(ia):
    """A batch whose scaled output gradient leaves the fp16 range: every gradient
    buffer comes back zero, the step reports skipped, and S halves."""
    sc = S.make_scene("tiny", 0)
    table, mlp = S.make_field(sc, 0)
    ctx = _ctx(ia, sc, table, mlp, 1)
    th, tr = S.make_pose(sc, 0)
    ia.ia_set_pose(ctx, th[None], tr[None])
    ia.ia_update_occupancy(ctx, 0)
    rb = S.make_ray_batch(sc, 64, 1, seed=3)
    rays = {k: rb[k] for k in ("origin", "direction", "pose", "target")}
    # one ray's loss gradient dominates: (C - target) ~ -1e4 and n = 64 rays
    rays["target"] = np.full_like(rays["target"], 1e4)
    dev = _dev(rays)
    g = _grads(ia, ctx, sc, 1)
    for v in g.values():
        v.fill_(7.0)
    ia.ia_train_step(ctx, dev["origin"], dev["direction"], dev["pose"], dev["target"],
                     torch.zeros(1, device="cuda"), g, occ_grid=ia.IA_OCC_POSE)
    scale, skipped = ia.ia_loss_scale(ctx)
    assert skipped
    assert scale == 8192.0
    for k, v in g.items():
        assert torch.count_nonzero(v).item() == 0, k
    # a normal batch afterwards is not skipped and keeps the halved scale
    dev = _dev({k: rb[k] for k in ("origin", "direction", "pose", "target")})
    ia.ia_train_step(ctx, dev["origin"], dev["direction"], dev["pose"], dev["target"],
                     torch.zeros(1, device="cuda"), g, occ_grid=ia.IA_OCC_POSE)
    scale, skipped = ia.ia_loss_scale(ctx)
    assert not skipped and scale == 8192.0
    assert torch.count_nonzero(g["mlp"]).item() > 0
    ia.ia_destroy(ctx)


def test_pipeline_wait_limit_skips_the_step(ia):
    """The weight-gradient GEMM's bounded waits, made to run out without any
    fault: with copy withholding injected, each CTA's producer never issues the
    TMA copy of its last operand chunk, so the MMA thread's wait for it expires
    after the (1 ms) wait limit while earlier chunks' MMAs are still in flight.
    The kernel must drain those, free its tensor memory and return: the step is
    reported as IA_ERR_CUDA and skipped (all gradients zero, loss scale kept),
    and the context stays usable -- the next step, without injection, gives the
    same gradients as a clean step before."""
    sc = S.make_scene("full", 0)
    table, mlp = S.make_field(sc, 0)
    ctx = _ctx(ia, sc, table, mlp, 1)
    poses = [S.make_pose(sc, i) for i in range(2)]
    ia.ia_set_pose(ctx, np.stack([p[0] for p in poses]), np.stack([p[1] for p in poses]))
    for i in range(2):
        ia.ia_update_occupancy(ctx, i, ia.IA_OCC_UNION)
    rb = S.make_ray_batch(sc, 12288, 2, seed=9)
    dev = _dev({k: rb[k] for k in ("origin", "direction", "pose", "target")})

    def step():
        g = _grads(ia, ctx, sc, 2)
        for v in g.values():
            v.fill_(7.0)
        ia.ia_train_step(ctx, dev["origin"], dev["direction"], dev["pose"], dev["target"],
                         torch.zeros(1, device="cuda"), g, occ_grid=ia.IA_OCC_UNION)
        return g

    g0 = step()
    assert ia.ia_loss_scale(ctx) == (16384.0, False)
    st = ia.ia_train_stats(ctx)
    assert st["occupied_samples"] - st["culled"] > 2 * 148 * 64  # several chunks per CTA
    ia.ia_set_wait_limit(ctx, 1_000_000)
    ia.ia_set_fault_injection(ctx, ia.IA_INJECT_WITHHOLD_COPY)
    g1 = step()
    with pytest.raises(ia.IAError) as e:
        ia.ia_loss_scale(ctx)
    assert e.value.status == ia.IA_ERR_CUDA and "gave up" in str(e.value)
    for k, v in g1.items():
        assert torch.count_nonzero(v).item() == 0, k
    ia.ia_set_fault_injection(ctx, 0)
    ia.ia_set_wait_limit(ctx, 0)
    g2 = step()
    assert ia.ia_loss_scale(ctx) == (16384.0, False)  # the skipped step left the scale alone
    for k in g0:
        a, b = g2[k].cpu().numpy(), g0[k].cpu().numpy()
        assert np.count_nonzero(b) > 0
        assert np.allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max()), k
    ia.ia_destroy(ctx)


def test_train_step_with_proposal_starts(ia):
    """fp16 step whose correspondence search starts from the proposal's top-2
    bones of each sample's own pose (the batch mixes 4 poses, so every warp
    holds several poses) against the oracle's proposal-start step.  The
    proposal is the seeded initial network with its pose columns amplified, so
    the chosen bones depend strongly on the pose; the oracle reads the same
    fp16-rounded weights (the pose columns are folded in fp32 on both sides).
    Rays the oracle flags (near-tied logits, marginal roots) are dropped."""
    from oracle import prop as PP
    sc = S.make_scene("full", 0)
    table, mlp = S.make_field(sc, 0)
    t_op, m_op = _operands(table, mlp, 1)
    om = O.OracleModel(sc, t_op, m_op)
    n_poses = 4
    poses = [S.make_pose(sc, 20 + i) for i in range(n_poses)]
    theta = np.stack([p[0] for p in poses])
    op = [om.pose(*p) for p in poses]
    occ = np.zeros((sc.occ_res ** 3 + 31) // 32, np.uint32)
    for p in op:
        occ |= om.occupancy(p)[1]
    cfg = S.proposal_config()
    pt, pm = S.proposal_init(sc, cfg, 3)
    nf = 2 * cfg["n_levels"]
    pm["W1"][:, nf:] *= 4.0
    pm_op = {k: (v.copy() if not k.startswith("W") else _round_fp16(v)) for k, v in pm.items()}
    pm_op["W1"][:, nf:] = pm["W1"][:, nf:]  # folded into the fp32 bias, not rounded
    pr = PP.PropModel(om, cfg, pt, pm_op)
    rb = S.make_ray_batch(sc, 2048, n_poses, seed=7)
    args = (om, op, occ, rb["origin"], rb["direction"], rb["pose"], rb["target"])
    _, _, flags, _ = G.train(*args, grad=False, prop=pr, theta=theta)
    keep = flags == 0
    print(f"oracle-flagged rays dropped: {(~keep).sum()} of {keep.size}")
    assert (~keep).sum() <= 0.02 * keep.size  # 24 of 2048 with this seed
    rays = {k: rb[k][keep] for k in ("origin", "direction", "pose", "target")}

    ctx = _ctx(ia, sc, table, mlp, 1)
    ia.ia_set_pose(ctx, theta, np.stack([p[1] for p in poses]))
    ia.ia_set_occupancy(ctx, occ)
    ia.ia_proposal_init(ctx, ia.make_proposal_config(cfg["n_levels"], cfg["log2_table"], cfg["level_res"],
                                                     cfg["top_k"], cfg["offset_weight"]))
    ia.ia_proposal_set_params(ctx, torch.from_numpy(np.ascontiguousarray(pt)).cuda(),
                              torch.from_numpy(S.pack_proposal(pm)).cuda())
    ia.ia_set_search(ctx, ia.IA_SEARCH_PROPOSAL)
    g = _grads(ia, ctx, sc, n_poses)
    dev = _dev(rays)
    loss = torch.zeros(1, device="cuda")
    rgb = torch.zeros(len(rays["pose"]), 3, device="cuda")
    ia.ia_train_step(ctx, dev["origin"], dev["direction"], dev["pose"], dev["target"], loss, g,
                     occ_grid=ia.IA_OCC_POSE, rgb_out=rgb)
    st = ia.ia_train_stats(ctx)
    torch.cuda.synchronize()
    ia.ia_destroy(ctx)

    args = (om, op, occ, rays["origin"], rays["direction"], rays["pose"], rays["target"])
    fb = np.zeros(len(rays["pose"]), np.int32)
    ref_loss, ref_rgb, _, ref = G.train(*args, prop=pr, theta=theta, fallbacks=fb)
    # every ray's colour within the fp16 bound: a sample whose root the GPU missed
    # (or found where the oracle has none) would move its ray far outside it
    bad = ~close(rgb.cpu().numpy(), ref_rgb, 2e-3, 2e-4).all(axis=1)
    print(f"rays outside the fp16 colour bound: {bad.sum()} of {bad.size}")
    assert bad.sum() <= 0.002 * bad.size
    # which samples needed the fallback depends on the bones proposed for each
    # sample's own pose: the counts must agree (a few marginal samples aside)
    # (a culled sample can have no root, so the oracle's search falls back on it)
    print(f"fallbacks gpu {st['fallbacks']} + culled {st['culled']} + point-culled {st['point_culled']}, "
          f"oracle {int(fb.sum())} of "
          f"{st['occupied_samples']} samples")
    assert st["proposed"] == st["occupied_samples"] - st["culled"] > 0
    assert abs(st["fallbacks"] + st["culled"] + st["point_culled"] - int(fb.sum())) <= max(3, 0.005 * fb.sum())
    assert 0 < fb.sum() < st["proposed"]
    plain_loss, _, _, plain = G.train(*args)
    lg = float(loss.item())
    print(f"proposal fp16: {keep.sum()} rays, loss gpu {lg:.6e} oracle {ref_loss:.6e} (plain search {plain_loss:.6e})")
    assert abs(lg - ref_loss) <= TOL[1]["loss"] * ref_loss
    for k in ("table", "mlp", "skin", "bones"):
        a = g[k].cpu().numpy().astype(np.float64)
        b = ref[k].reshape(-1)
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        rel_plain = np.linalg.norm(plain[k].reshape(-1) - b) / max(np.linalg.norm(b), 1e-30)
        print(f"  grad {k}: rel L2 {rel:.2e} (oracle proposal vs oracle plain search: {rel_plain:.2e})")
        assert rel <= TOL[1]["grad"], k
