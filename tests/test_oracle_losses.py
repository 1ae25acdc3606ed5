"""Pins of the oracle's loss set of Sec. 3.4 (Huber colour loss Eq. 9, alpha
L1 Eq. 10, hard-surface Eq. 11): central differences of the combined loss,
the Huber function's quadratic limit, and the value on rays that miss."""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from oracle import grad as G

H = 1e-4


@pytest.fixture(scope="module")
def case():
    sc = S.make_scene("tiny", 0)
    table, mlp = S.make_field(sc, 0)
    om = O.OracleModel(sc, table, mlp)
    poses = [om.pose(*S.make_pose(sc, i)) for i in range(2)]
    occ = om.occupancy(poses[0])[1] | om.occupancy(poses[1])[1]
    rb = S.make_ray_batch(sc, 4000, 2, seed=1)
    _, rgb, flags, _ = G.train(om, poses, occ, rb["origin"], rb["direction"], rb["pose"], rb["target"], grad=False)
    hit = np.nonzero((rgb.sum(1) > 1e-3) & (flags == 0))[0][:64]
    rays = {k: rb[k][hit] for k in ("origin", "direction", "pose", "target")}
    alpha_gt = np.random.default_rng(5).uniform(0, 1, len(hit))
    return sc, om, poses, occ, rays, alpha_gt


def _run(om, poses, occ, rays, loss, grad=True):
    return G.train(om, poses, occ, rays["origin"], rays["direction"], rays["pose"], rays["target"], grad=grad,
                   loss=loss)


def test_loss_set_gradient_matches_central_differences(case):
    sc, om, poses, occ, rays, alpha_gt = case
    cfg = dict(huber=1, delta=0.8, w_rgb=1.0, w_alpha=0.7, w_hard=0.3, alpha_target=alpha_gt)
    loss, rgb, _, g = _run(om, poses, occ, rays, cfg)
    err = np.linalg.norm(rgb - rays["target"], axis=1)
    assert np.any(err < 0.8) and np.any(err > 0.8)  # both branches of the Huber function

    def L(pp=poses):
        return _run(om, pp, occ, rays, cfg, grad=False)[0]

    rng = np.random.default_rng(3)
    worst, checks = 0.0, 0
    names = ("W1", "b1", "W2", "b2", "W3", "b3")
    sizes = np.cumsum([0] + [om.mlp[k].size for k in names])
    targets = [(om.table.reshape(-1), g["table"].reshape(-1)), (om.skin.reshape(-1), g["skin"].reshape(-1))]
    for arr, flat in targets:
        nz = np.flatnonzero(np.abs(flat) > 1e-6 * np.abs(flat).max())
        for i in rng.choice(nz, size=8, replace=False):
            old = arr[i]
            arr[i] = old + H
            lp = L()
            arr[i] = old - H
            lm = L()
            arr[i] = old
            fd = (lp - lm) / (2 * H)
            worst = max(worst, abs(flat[i] - fd) / max(abs(fd), abs(flat[i]), 1e-12))
            assert abs(flat[i] - fd) <= 1e-3 * max(abs(fd), abs(flat[i])) + 1e-9
            checks += 1
    nz = np.flatnonzero(np.abs(g["mlp"]) > 1e-6 * np.abs(g["mlp"]).max())
    for i in rng.choice(nz, size=8, replace=False):
        k = int(np.searchsorted(sizes, i, side="right") - 1)
        arr = om.mlp[names[k]].reshape(-1)
        j = i - sizes[k]
        old = arr[j]
        arr[j] = old + H
        lp = L()
        arr[j] = old - H
        lm = L()
        arr[j] = old
        fd = (lp - lm) / (2 * H)
        worst = max(worst, abs(g["mlp"][i] - fd) / max(abs(fd), abs(g["mlp"][i]), 1e-12))
        assert abs(g["mlp"][i] - fd) <= 1e-3 * max(abs(fd), abs(g["mlp"][i])) + 1e-9
        checks += 1
    nz = np.flatnonzero(np.abs(g["bones"].reshape(-1)) > 1e-6 * np.abs(g["bones"]).max())
    for i in rng.choice(nz, size=8, replace=False):
        p, k, e = np.unravel_index(i, g["bones"].shape)
        pp = G.pose_array(poses)
        old = pp[p].N[k][e]
        pp[p].N[k][e] = old + H
        lp = L(pp)
        pp[p].N[k][e] = old - H
        lm = L(pp)
        fd = (lp - lm) / (2 * H)
        assert abs(g["bones"][p, k, e] - fd) <= 1e-3 * max(abs(fd), abs(g["bones"][p, k, e])) + 1e-9
        checks += 1
    print(f"{checks} finite-difference checks of the loss set, worst relative error {worst:.2e}")
    assert checks == 32


def test_huber_with_a_large_threshold_is_half_the_l2_loss(case):
    sc, om, poses, occ, rays, _ = case
    l2, _, _, g2 = _run(om, poses, occ, rays, None)
    lh, _, _, gh = _run(om, poses, occ, rays, dict(huber=1, delta=1e9))
    assert abs(lh - 0.5 * l2) <= 1e-12 * l2
    for k in g2:
        np.testing.assert_allclose(gh[k], 0.5 * g2[k], rtol=1e-12, atol=1e-18)


def test_opacity_terms_on_rays_that_miss(case):
    """alpha = 0 off the body: the hard-surface term is 0 there (its constant
    makes 0 and 1 the minima) and the mask term is the mean target."""
    sc, om, poses, occ, rays, alpha_gt = case
    miss = {k: v.copy() for k, v in rays.items()}
    miss["direction"] = -miss["direction"]
    l_hard, rgb, _, g = _run(om, poses, occ, miss, dict(w_rgb=0.0, w_hard=1.0))
    assert np.all(rgb == 0) and abs(l_hard) < 1e-15
    l_a, _, _, _ = _run(om, poses, occ, miss, dict(w_rgb=0.0, w_alpha=1.0, alpha_target=alpha_gt), grad=False)
    assert abs(l_a - alpha_gt.mean()) <= 1e-12
