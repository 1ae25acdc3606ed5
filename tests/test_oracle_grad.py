"""Pins of the oracle's training-step gradient: central finite differences
(h = 1e-4) of its own fp64 loss on 64 random parameters spread over the hash
table, the MLP, the skinning-weight grid and the bone transforms, plus the
structure the gradient must have (zero where no sample reaches, zero at a zero
residual)."""
import ctypes as C

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
    _, rgb, _, _ = G.train(om, poses, occ, rb["origin"], rb["direction"], rb["pose"], rb["target"], grad=False)
    hit = np.nonzero(rgb.sum(1) > 1e-3)[0][:64]
    rays = {k: rb[k][hit] for k in ("origin", "direction", "pose", "target")}
    return sc, om, poses, occ, rays


def _loss(om, poses, occ, rays):
    return G.train(om, poses, occ, rays["origin"], rays["direction"], rays["pose"], rays["target"],
                   grad=False)[0]


def _fd(om, arr, idx, poses, occ, rays):
    old = arr[idx]
    arr[idx] = old + H
    lp = _loss(om, poses, occ, rays)
    arr[idx] = old - H
    lm = _loss(om, poses, occ, rays)
    arr[idx] = old
    return (lp - lm) / (2 * H)


def _pick(g, n, rng):
    nz = np.flatnonzero(np.abs(g) > 1e-6 * np.abs(g).max())
    return rng.choice(nz, size=min(n, len(nz)), replace=False)


def test_gradient_matches_central_differences(case):
    sc, om, poses, occ, rays = case
    loss, _, flags, g = G.train(om, poses, occ, rays["origin"], rays["direction"], rays["pose"], rays["target"])
    assert np.all(flags == 0) and len(rays["pose"]) >= 32
    rng = np.random.default_rng(0)
    checks = []
    for i in _pick(g["table"].reshape(-1), 16, rng):
        checks.append(("table", g["table"].reshape(-1)[i], _fd(om, om.table.reshape(-1), i, poses, occ, rays)))
    names = ("W1", "b1", "W2", "b2", "W3", "b3")
    sizes = np.cumsum([0] + [om.mlp[k].size for k in names])
    for i in _pick(g["mlp"], 16, rng):
        k = int(np.searchsorted(sizes, i, side="right") - 1)
        checks.append(("mlp." + names[k], g["mlp"][i],
                       _fd(om, om.mlp[names[k]].reshape(-1), i - sizes[k], poses, occ, rays)))
    for i in _pick(g["skin"].reshape(-1), 16, rng):
        checks.append(("skin", g["skin"].reshape(-1)[i], _fd(om, om.skin.reshape(-1), i, poses, occ, rays)))
    for i in _pick(g["bones"].reshape(-1), 16, rng):
        p, k, e = np.unravel_index(i, g["bones"].shape)
        pp = G.pose_array(poses)
        old = pp[p].N[k][e]
        pp[p].N[k][e] = old + H
        lp = _loss(om, pp, occ, rays)
        pp[p].N[k][e] = old - H
        lm = _loss(om, pp, occ, rays)
        checks.append(("bone", g["bones"][p, k, e], (lp - lm) / (2 * H)))
    assert len(checks) == 64
    worst = 0.0
    for name, an, fd in checks:
        worst = max(worst, abs(an - fd) / max(abs(an), abs(fd), 1e-12))
        assert abs(an - fd) <= 1e-3 * max(abs(an), abs(fd)) + 1e-9, (name, an, fd)
    print(f"64 finite-difference checks, worst relative error {worst:.2e}")


def test_gradient_support(case):
    sc, om, poses, occ, rays = case
    miss = {k: v.copy() for k, v in rays.items()}
    miss["direction"] = -miss["direction"]  # rays that leave the box: a loss but no parameter gradient
    loss, rgb, _, g = G.train(om, poses, occ, miss["origin"], miss["direction"], miss["pose"], miss["target"])
    assert np.all(rgb == 0)
    np.testing.assert_allclose(loss, np.mean(np.sum(miss["target"].astype(np.float64) ** 2, axis=1)), rtol=1e-12)
    for v in g.values():
        assert np.all(v == 0)
    _, rgb, _, _ = G.train(om, poses, occ, rays["origin"], rays["direction"], rays["pose"], rays["target"], grad=False)
    loss, _, _, g = G.train(om, poses, occ, rays["origin"], rays["direction"], rays["pose"], rgb)
    assert loss < 1e-28
    for v in g.values():
        assert np.abs(v).max() < 1e-14
