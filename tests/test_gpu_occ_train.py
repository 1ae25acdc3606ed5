"""Training-mode occupancy (Sec. 3.3, training stage) and the occupancy-based
density regulariser (Eq. 12) on the GPU against the fp64 oracle.

Running density: fp32 against fp64 at the same jittered cell points, the
density tolerance of the posed-field tests (1e-4 relative; a cell where one side
finds a marginal root and the other none may differ, at most 0.1 % of cells);
bits exact outside the dilation neighbourhood of densities within 1e-3 of tau.
Regulariser: the fp32 training step's tolerances (loss 1e-5 relative, gradients
2e-3 relative L2 per group, 1e-3 of the group's scale per element)."""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from gpu_helpers import RTOL_SIGMA, bits_to_bool, make_ctx
from oracle import grad as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ia():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_10550_b300 as ia
    ia.lib()
    return ia


def _near_tau(d, sc):
    R = sc.occ_res
    amb = (np.abs(d - sc.occ_tau) < 1e-3 * sc.occ_tau).reshape(R, R, R)
    near = np.zeros_like(amb)
    k = sc.occ_dilate
    for dz in range(-k, k + 1):
        for dy in range(-k, k + 1):
            for dx in range(-k, k + 1):
                near |= np.roll(amb, (dz, dy, dx), axis=(0, 1, 2))
    return near.reshape(-1)


@pytest.mark.parametrize("config", ["tiny", "full"])
def test_running_density_and_training_grid(ia, config):
    sc = S.make_scene(config, 0)
    table, mlp = S.make_field(sc, 0)
    om = O.OracleModel(sc, table, mlp)
    poses = [S.make_pose(sc, 30 + i) for i in range(3)]
    ctx = make_ctx(ia, torch, sc, table, mlp)
    ia.ia_set_pose(ctx, np.stack([p[0] for p in poses]), np.stack([p[1] for p in poses]))
    R = sc.occ_res
    d_ref = np.zeros(R ** 3)
    dens = torch.zeros(R ** 3, device="cuda")
    bits = torch.zeros((R ** 3 + 31) // 32, dtype=torch.int32, device="cuda")
    for i, decay in enumerate((0.0, 0.95, 0.95)):
        jit = S.occupancy_jitter(sc, i)
        ia.ia_update_occupancy_ema(ctx, i, torch.from_numpy(jit).cuda(), decay, dens, bits)
        ref_bits = om.occupancy_ema(om.pose(*poses[i]), d_ref, jit, decay)
    torch.cuda.synchronize()
    g = dens.cpu().numpy().astype(np.float64)
    off = np.abs(g - d_ref) > RTOL_SIGMA * np.abs(d_ref) + 1e-6 * d_ref.max()
    print(f"{config}: {np.count_nonzero(d_ref)} cells with density, {off.sum()} beyond tolerance")
    assert off.sum() <= 1e-3 * R ** 3
    near = _near_tau(d_ref, sc)
    g_occ = bits_to_bool(bits.cpu().numpy().view(np.uint32), R ** 3)
    r_occ = bits_to_bool(ref_bits, R ** 3)
    mism = (g_occ != r_occ) & ~near
    print(f"{config}: {g_occ.sum()} occupied, {near.sum()} ambiguous cells excluded, {mism.sum()} mismatches")
    assert mism.sum() == 0 and g_occ.sum() > 0
    ia.ia_destroy(ctx)


def test_training_step_reads_the_running_grid(ia):
    """After the updates, a step on the training grid (IA_OCC_UNION) equals a step
    on the same bits installed as the render grid."""
    sc = S.make_scene("tiny", 0)
    table, mlp = S.make_field(sc, 0)
    poses = [S.make_pose(sc, i) for i in range(2)]
    ctx = make_ctx(ia, torch, sc, table, mlp)
    ia.ia_set_pose(ctx, np.stack([p[0] for p in poses]), np.stack([p[1] for p in poses]))
    R = sc.occ_res
    bits = torch.zeros((R ** 3 + 31) // 32, dtype=torch.int32, device="cuda")
    for i in range(2):
        ia.ia_update_occupancy_ema(ctx, i, None, 0.9, None, bits)
    ia.ia_set_occupancy(ctx, bits.cpu().numpy().view(np.uint32).copy())
    rb = S.make_ray_batch(sc, 2000, 2, seed=8)
    dev = {k: torch.from_numpy(np.ascontiguousarray(rb[k])).cuda() for k in ("origin", "direction", "pose", "target")}
    nt, nm = ia.ia_param_sizes(ctx)
    out = []
    for grid in (ia.IA_OCC_UNION, ia.IA_OCC_POSE):
        g = dict(table=torch.zeros(nt, device="cuda"), mlp=torch.zeros(nm, device="cuda"),
                 skin=torch.zeros(sc.skin_res ** 3 * sc.n_bones, device="cuda"),
                 bones=torch.zeros(2 * sc.n_bones * 12, device="cuda"))
        loss = torch.zeros(1, device="cuda")
        ia.ia_train_step(ctx, dev["origin"], dev["direction"], dev["pose"], dev["target"], loss, g, occ_grid=grid)
        out.append((loss.item(), g["mlp"].cpu().numpy()))
    ia.ia_destroy(ctx)
    assert abs(out[0][0] - out[1][0]) <= 1e-6 * out[1][0]
    np.testing.assert_allclose(out[0][1], out[1][1], rtol=1e-4, atol=1e-6 * np.abs(out[1][1]).max())


def test_density_regulariser_matches_oracle(ia):
    sc = S.make_scene("tiny", 0)
    table, mlp = S.make_field(sc, 0)
    om = O.OracleModel(sc, table, mlp)
    poses = [S.make_pose(sc, i) for i in range(2)]
    op = [om.pose(*p) for p in poses]
    occ = om.occupancy(op[0])[1] | om.occupancy(op[1])[1]
    rng = np.random.default_rng(4)
    occ = occ & rng.integers(0, 2 ** 32, size=occ.shape, dtype=np.uint64).astype(np.uint32)  # holes
    rb = S.make_ray_batch(sc, 2000, 2, seed=6)
    _, _, flags, _ = G.train(om, op, occ, rb["origin"], rb["direction"], rb["pose"], rb["target"], grad=False)
    rays = {k: rb[k][flags == 0] for k in ("origin", "direction", "pose", "target")}
    x = S.random_points(sc, 6000, seed=11)
    pid = rng.integers(0, 2, size=len(x)).astype(np.int32)
    _, pflags = G.density_reg(om, op, occ, x, pid, 1.0)
    x, pid = x[pflags == 0], pid[pflags == 0]
    w = 300.0  # the regulariser's share of loss and gradient comparable to the photometric term
    ref_loss, _, _, ref = G.train(om, op, occ, rays["origin"], rays["direction"], rays["pose"], rays["target"])
    photo = {k: v.copy() for k, v in ref.items()}
    reg_loss, _ = G.density_reg(om, op, occ, x, pid, w, ref)
    ref_loss += reg_loss
    share = {k: np.linalg.norm((ref[k] - photo[k]).reshape(-1)) / np.linalg.norm(ref[k].reshape(-1)) for k in ref}
    print("regulariser share of loss %.2f, of gradients %s" % (reg_loss / ref_loss,
                                                              {k: round(float(v), 2) for k, v in share.items()}))
    assert reg_loss > 0.2 * ref_loss and min(share.values()) > 0.1

    ctx = make_ctx(ia, torch, sc, table, mlp)
    ia.ia_set_pose(ctx, np.stack([p[0] for p in poses]), np.stack([p[1] for p in poses]))
    ia.ia_set_occupancy(ctx, occ)
    nt, nm = ia.ia_param_sizes(ctx)
    g = dict(table=torch.zeros(nt, device="cuda"), mlp=torch.zeros(nm, device="cuda"),
             skin=torch.zeros(sc.skin_res ** 3 * sc.n_bones, device="cuda"),
             bones=torch.zeros(2 * sc.n_bones * 12, device="cuda"))
    dev = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in rays.items()}
    loss = torch.zeros(1, device="cuda")
    ia.ia_train_step(ctx, dev["origin"], dev["direction"], dev["pose"], dev["target"], loss, g,
                     occ_grid=ia.IA_OCC_POSE, reg_x=torch.from_numpy(x).cuda(), reg_pose=torch.from_numpy(pid).cuda(),
                     reg_weight=w)
    torch.cuda.synchronize()
    ia.ia_destroy(ctx)
    lg = loss.item()
    print(f"loss gpu {lg:.8e} oracle {ref_loss:.8e} (regulariser {reg_loss:.3e}, {len(x)} points)")
    assert abs(lg - ref_loss) <= 1e-5 * ref_loss
    for k in ("table", "mlp", "skin", "bones"):
        a, b = g[k].cpu().numpy().astype(np.float64), ref[k].reshape(-1)
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        worst = np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)
        print(f"grad {k}: rel L2 {rel:.2e}, worst element / scale {worst:.2e}")
        assert rel <= 2e-3 and worst <= 1e-3, k
