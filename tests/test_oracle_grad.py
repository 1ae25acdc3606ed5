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


def test_proposal_step_gradient_matches_central_differences(case):
    """The same pin for the step whose starts come from the correspondence
    proposal (an untrained, seeded network: many samples take the fallback,
    the others keep the proposed starts' roots).  Whether a proposed start
    converges within the iteration limit is a discrete event that a wide
    stencil can straddle, so the step is h = 3e-5 here (at 1e-4 one bone entry
    of the fixture differs by 1.8e-3 relative; at 3e-5 by 4e-6)."""
    from oracle import prop as PP
    sc, om, poses, occ, rays = case
    cfg = S.proposal_config()
    pt, pm = S.proposal_init(sc, cfg, 3)
    pr = PP.PropModel(om, cfg, pt, pm)
    theta = np.stack([S.make_pose(sc, i)[0] for i in range(2)])

    def loss_of(pp):
        return G.train(om, pp, occ, rays["origin"], rays["direction"], rays["pose"], rays["target"], grad=False,
                       prop=pr, theta=theta)[0]

    loss, _, flags, g = G.train(om, poses, occ, rays["origin"], rays["direction"], rays["pose"], rays["target"],
                                prop=pr, theta=theta)
    keep = flags == 0
    assert keep.sum() >= 32
    rays = {k: v[keep] for k, v in rays.items()}
    loss, _, _, g = G.train(om, poses, occ, rays["origin"], rays["direction"], rays["pose"], rays["target"],
                            prop=pr, theta=theta)
    rng = np.random.default_rng(1)
    h = 3e-5
    worst = 0.0
    for name, arr, flat in (("table", om.table.reshape(-1), g["table"].reshape(-1)),
                            ("skin", om.skin.reshape(-1), g["skin"].reshape(-1)),
                            ("W2", om.mlp["W2"].reshape(-1), None)):
        if flat is None:
            off = om.mlp["W1"].size + om.mlp["b1"].size
            flat = g["mlp"][off:off + arr.size]
        for i in _pick(flat, 8, rng):
            old = arr[i]
            arr[i] = old + h
            lp = loss_of(poses)
            arr[i] = old - h
            lm = loss_of(poses)
            arr[i] = old
            fd = (lp - lm) / (2 * h)
            worst = max(worst, abs(flat[i] - fd) / max(abs(flat[i]), abs(fd), 1e-12))
            assert abs(flat[i] - fd) <= 1e-3 * max(abs(flat[i]), abs(fd)) + 1e-9, (name, flat[i], fd)
    for i in _pick(g["bones"].reshape(-1), 8, rng):
        p, k, e = np.unravel_index(i, g["bones"].shape)
        pp = G.pose_array(poses)
        old = pp[p].N[k][e]
        pp[p].N[k][e] = old + h
        lp = loss_of(pp)
        pp[p].N[k][e] = old - h
        lm = loss_of(pp)
        fd = (lp - lm) / (2 * h)
        worst = max(worst, abs(g["bones"][p, k, e] - fd) / max(abs(fd), 1e-12))
        assert abs(g["bones"][p, k, e] - fd) <= 1e-3 * max(abs(g["bones"][p, k, e]), abs(fd)) + 1e-9
    print(f"32 finite-difference checks (proposal starts), worst relative error {worst:.2e}")


def test_proposal_step_equals_plain_step_when_roots_agree(case):
    """Where the proposal's starts reach the same root as the plain search
    (one root per sample, as on most of the body), the two steps are the same
    function: equal loss and gradient on rays whose samples all agree (up to
    the roots' polish, 1e-12, reached from different starts)."""
    from oracle import prop as PP
    sc, om, poses, occ, rays = case
    cfg = S.proposal_config()
    pt, pm = S.proposal_init(sc, cfg, 3)
    pr = PP.PropModel(om, cfg, pt, pm)
    theta = np.stack([S.make_pose(sc, i)[0] for i in range(2)])
    args = (om, poses, occ, rays["origin"], rays["direction"], rays["pose"], rays["target"])
    _, rgb_a, _, _ = G.train(*args, grad=False)
    _, rgb_b, _, _ = G.train(*args, grad=False, prop=pr, theta=theta)
    same = np.all(np.abs(rgb_a - rgb_b) <= 1e-12, axis=1)
    assert same.sum() >= 16
    sub = {k: v[same] for k, v in rays.items()}
    args = (om, poses, occ, sub["origin"], sub["direction"], sub["pose"], sub["target"])
    la, _, _, ga = G.train(*args)
    lb, _, _, gb = G.train(*args, prop=pr, theta=theta)
    assert abs(la - lb) <= 1e-12 * la
    for k in ga:
        np.testing.assert_allclose(gb[k], ga[k], rtol=1e-6, atol=1e-10 * max(np.abs(ga[k]).max(), 1e-30))


def test_upstream_gradient_matches_central_differences(case):
    """The backward for a loss built outside the step (or_train_upstream, the
    reference of the library's autograd backward): for the linear functional
    L = sum_r w_r . C_r + v_r alpha_r of the rendered colour and opacity, with
    seeded weights given as dL/dC = w, dL/dalpha = v, its gradient matches
    central differences of L computed from the oracle's forward alone, on 32
    parameters over the table, MLP, skinning grid and bone transforms.  The
    weights are O(1) per ray (not the 1/n of an averaged loss), so L's second
    derivatives are ~n times those of the step's loss and the stencil's O(h^2)
    truncation needs h = 1e-5 (measured: at 1e-4 a small bone entry is off by
    2.4e-3, at 1e-5 the checks agree to ~1e-6)."""
    h = 1e-5
    sc, om, poses, occ, rays = case
    n = len(rays["pose"])
    rng = np.random.default_rng(5)
    w = rng.normal(size=(n, 3))
    v = rng.normal(size=n)
    args = (om, poses, occ, rays["origin"], rays["direction"], rays["pose"])
    rgb, alpha, flags, g = G.train_upstream(*args, up_rgb=w, up_alpha=v)
    assert np.all(flags == 0)

    def L(pp=poses):
        r, a, _, _ = G.train_upstream(om, pp, occ, rays["origin"], rays["direction"], rays["pose"])
        return float(np.sum(w * r) + np.sum(v * a))

    assert abs(L() - float(np.sum(w * rgb) + np.sum(v * alpha))) < 1e-12

    def fd(arr, idx):
        old = arr[idx]
        arr[idx] = old + h
        lp = L()
        arr[idx] = old - h
        lm = L()
        arr[idx] = old
        return (lp - lm) / (2 * h)

    checks = []
    for i in _pick(g["table"].reshape(-1), 8, rng):
        checks.append(("table", g["table"].reshape(-1)[i], fd(om.table.reshape(-1), i)))
    names = ("W1", "b1", "W2", "b2", "W3", "b3")
    sizes = np.cumsum([0] + [om.mlp[k].size for k in names])
    for i in _pick(g["mlp"], 8, rng):
        k = int(np.searchsorted(sizes, i, side="right") - 1)
        checks.append(("mlp." + names[k], g["mlp"][i], fd(om.mlp[names[k]].reshape(-1), i - sizes[k])))
    for i in _pick(g["skin"].reshape(-1), 8, rng):
        checks.append(("skin", g["skin"].reshape(-1)[i], fd(om.skin.reshape(-1), i)))
    for i in _pick(g["bones"].reshape(-1), 8, rng):
        p, k, e = np.unravel_index(i, g["bones"].shape)
        pp = G.pose_array(poses)
        old = pp[p].N[k][e]
        pp[p].N[k][e] = old + h
        lp = L(pp)
        pp[p].N[k][e] = old - h
        lm = L(pp)
        checks.append(("bone", g["bones"][p, k, e], (lp - lm) / (2 * h)))
    assert len(checks) == 32
    worst = 0.0
    for name, an, f in checks:
        worst = max(worst, abs(an - f) / max(abs(an), abs(f), 1e-12))
        assert abs(an - f) <= 1e-3 * max(abs(an), abs(f)) + 1e-9, (name, an, f)
    print(f"32 finite-difference checks of the upstream backward, worst relative error {worst:.2e}")
