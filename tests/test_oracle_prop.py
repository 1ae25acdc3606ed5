"""Pins of the oracle's correspondence-proposal network: the MLP against numpy,
the label/offset target in closed form, central finite differences (h = 1e-4) of
its loss, and the search it drives (its roots are roots of the plain search;
no valid proposed root means the plain result)."""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from oracle import prop as PP

H = 1e-6  # small enough that no ReLU of the 40 x 192 hidden units changes side


@pytest.fixture(scope="module")
def setup():
    sc = S.make_scene("full", 0)
    table, mlp = S.make_field(sc, 0)
    om = O.OracleModel(sc, table, mlp)
    cfg = S.proposal_config()
    pt, pm = S.proposal_init(sc, cfg, 1)
    pm = {k: v + np.float32(0.05) * np.random.default_rng(9).normal(size=v.shape).astype(np.float32)
          if k.startswith("b") else v for k, v in pm.items()}  # non-zero biases exercise every term
    return sc, om, cfg, pt, pm


def test_forward_matches_numpy_mlp(setup):
    sc, om, cfg, pt, pm = setup
    pr = PP.PropModel(om, cfg, np.zeros_like(pt), pm)  # zero table: hash features are 0
    th, _ = S.make_pose(sc, 4)
    x = S.random_points(sc, 5, seed=3)
    M = {k: v.astype(np.float64) for k, v in pm.items()}
    for p in x:
        inp = np.concatenate([np.zeros(2 * cfg["n_levels"]), th.reshape(-1)])
        h = inp
        for i in (1, 2, 3):
            h = np.maximum(M[f"W{i}"] @ h + M[f"b{i}"], 0)
        ref = M["W4"] @ h + M["b4"]
        np.testing.assert_allclose(pr.forward(p, th), ref, rtol=1e-12, atol=1e-13)


def test_label_and_offset_closed_form():
    sc = S.make_scene("tiny", 0)
    table, mlp = S.make_field(sc, 0)
    onehot = np.zeros_like(sc.skin_grid, dtype=np.float64)
    onehot[..., 5] = 1.0
    om = O.OracleModel(sc, table, mlp, skin=onehot, quantize_fp32=False)
    cfg = S.proposal_config()
    pt, pm = S.proposal_init(sc, cfg, 0)
    pr = PP.PropModel(om, cfg, pt, pm)
    p = om.pose(*S.make_pose(sc, 2))
    T = om.transforms(p)
    N5 = np.vstack([T["N"][5], [0, 0, 0, 1]])
    for c in S.random_points(sc, 10, seed=1, box="canon").astype(np.float64):
        xn = (N5 @ np.append(c, 1))[:3]
        k, off = pr.label(p, c, xn)
        assert k == 5
        np.testing.assert_allclose(off, 0.0, atol=1e-12)  # x* = N_5^-1 x' exactly


def test_loss_gradient_matches_central_differences(setup):
    sc, om, cfg, pt, pm = setup
    pr = PP.PropModel(om, cfg, pt + np.random.default_rng(2).normal(0, 0.05, pt.shape).astype(np.float32), pm)
    rng = np.random.default_rng(4)
    n_poses = 3
    thetas = np.stack([S.make_pose(sc, i)[0] for i in range(n_poses)])
    x = S.random_points(sc, 40, seed=5)
    pid = rng.integers(0, n_poses, 40).astype(np.int32)
    lab = rng.integers(0, sc.n_bones, 40).astype(np.int32)
    tgt = rng.normal(0, 0.02, (40, 3))
    loss, gt, gm = pr.loss_grad(x, pid, thetas, lab, tgt)
    assert loss > 0
    checks = []
    flat_t = pr.table.reshape(-1)
    nz = np.flatnonzero(np.abs(gt.reshape(-1)) > 1e-8)
    for i in rng.choice(nz, 8, replace=False):
        old = flat_t[i]
        flat_t[i] = old + H
        lp = pr.loss_grad(x, pid, thetas, lab, tgt, grad=False)[0]
        flat_t[i] = old - H
        lm = pr.loss_grad(x, pid, thetas, lab, tgt, grad=False)[0]
        flat_t[i] = old
        checks.append((gt.reshape(-1)[i], (lp - lm) / (2 * H)))
    sizes = np.cumsum([0] + [pr.mlp[k].size for k in PP.NAMES])
    nz = np.flatnonzero(np.abs(gm) > 1e-8)
    for i in rng.choice(nz, 24, replace=False):
        k = int(np.searchsorted(sizes, i, side="right") - 1)
        arr = pr.mlp[PP.NAMES[k]].reshape(-1)
        j = i - sizes[k]
        old = arr[j]
        arr[j] = old + H
        lp = pr.loss_grad(x, pid, thetas, lab, tgt, grad=False)[0]
        arr[j] = old - H
        lm = pr.loss_grad(x, pid, thetas, lab, tgt, grad=False)[0]
        arr[j] = old
        checks.append((gm[i], (lp - lm) / (2 * H)))
    for an, fd in checks:
        assert abs(an - fd) <= 1e-4 * max(abs(an), abs(fd)) + 1e-10, (an, fd)


def test_proposal_search_finds_roots_of_the_plain_search(setup):
    sc, om, cfg, pt, pm = setup
    pr = PP.PropModel(om, cfg, pt, pm)
    th, tr = S.make_pose(sc, 7)
    p = om.pose(th, tr)
    from gpu_helpers import points_near_body
    fallbacks = 0
    for xn in points_near_body(sc, om, p, 60, 8).astype(np.float64):
        s = pr.posed_field(p, th, xn)
        plain = om.posed_field(p, xn)
        if s["fallback"]:
            fallbacks += 1
            assert s["start"] == plain["start"] and s["sigma"] == plain["sigma"]
            continue
        roots, _, _ = om.roots(p, xn)
        assert s["start"] >= 0
        assert np.min(np.linalg.norm(roots - s["xstar"], axis=1)) < 1e-8
    print(f"untrained proposal: {fallbacks} of 60 samples fell back to the plain search")


def test_render_with_every_bone_proposed_is_the_plain_render():
    """Special case of the proposal-mode render (or_render_pixels_prop): a
    network that proposes every bone (top_k = n_bones) with a zero start offset
    starts each sample's search from exactly the paper's bone-wise starts, only
    in the order of its (seeded, sample-dependent) logits, so the root set and
    the max-density root are the plain search's and the frame must equal the
    plain render (or_render_pixels) ray for ray, over the whole 64 x 64 tiny
    frame.  A proposal search only falls back when none of its starts finds a
    root, so with every bone proposed a fallback re-runs the same search: the
    colours stay equal and each ray's fallbacks are at most its samples."""
    sc = S.make_scene("tiny", 0)
    table, mlp = S.make_field(sc, 0)
    om = O.OracleModel(sc, table, mlp)
    cfg = dict(S.proposal_config(), top_k=sc.n_bones)
    pt, pm = S.proposal_init(sc, cfg, 2)
    pm["W4"][sc.n_bones:] = 0.0  # zero start offset
    pm["b4"][sc.n_bones:] = 0.0
    pr = PP.PropModel(om, cfg, pt, pm)
    th, tr = S.make_pose(sc, 3)
    p = om.pose(th, tr)
    _, bits = om.occupancy(p)
    cam = S.make_camera(sc)
    pix = np.arange(cam["width"] * cam["height"], dtype=np.int32)
    plain = om.render_pixels(p, cam, bits, pix)
    prop = pr.render_pixels(p, th, cam, bits, pix)
    np.testing.assert_array_equal(prop["nsamp"], plain["nsamp"])
    assert plain["nsamp"].sum() > 2000 and (plain["alpha"] > 0.01).sum() > 100
    ok = ((prop["flags"] | plain["flags"]) & O.FLAG_TIE) == 0  # exact density ties may pick either root
    assert ok.mean() > 0.99
    np.testing.assert_allclose(prop["rgb"][ok], plain["rgb"][ok], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(prop["alpha"][ok], plain["alpha"][ok], rtol=1e-9, atol=1e-12)
    assert np.all(prop["fallbacks"] <= prop["nsamp"])
