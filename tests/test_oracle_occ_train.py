"""Pins of the oracle's training-mode occupancy (Sec. 3.3, training stage) and of
its occupancy-based density regulariser (Eq. 12)."""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from oracle import grad as G

H = 1e-4


@pytest.fixture(scope="module")
def tiny():
    sc = S.make_scene("tiny", 0)
    table, mlp = S.make_field(sc, 0)
    om = O.OracleModel(sc, table, mlp)
    poses = [om.pose(*S.make_pose(sc, i)) for i in range(2)]
    return sc, om, poses


def test_zero_decay_at_cell_centres_is_the_pose_grid(tiny):
    sc, om, poses = tiny
    d = np.zeros(sc.occ_res ** 3)
    bits = om.occupancy_ema(poses[0], d, None, decay=0.0)
    sigma, ref = om.occupancy(poses[0])
    np.testing.assert_array_equal(d, sigma)
    np.testing.assert_array_equal(bits, ref)
    assert 0 < np.count_nonzero(bits) < len(bits)


def test_no_decay_gives_the_union_of_the_frames(tiny):
    """max is the union of the thresholds, and dilation distributes over union."""
    sc, om, poses = tiny
    d = np.zeros(sc.occ_res ** 3)
    om.occupancy_ema(poses[0], d, None, decay=1.0)
    bits = om.occupancy_ema(poses[1], d, None, decay=1.0)
    s0, b0 = om.occupancy(poses[0])
    s1, b1 = om.occupancy(poses[1])
    np.testing.assert_array_equal(d, np.maximum(s0, s1))
    np.testing.assert_array_equal(bits, b0 | b1)
    assert not np.array_equal(b0, b1)


def test_half_jitter_is_the_centre_and_decay_forgets(tiny):
    sc, om, poses = tiny
    R = sc.occ_res
    d1, d2 = np.zeros(R ** 3), np.zeros(R ** 3)
    om.occupancy_ema(poses[0], d1, np.full((R ** 3, 3), 0.5, np.float32), decay=0.0)
    om.occupancy_ema(poses[0], d2, None, decay=0.0)
    np.testing.assert_array_equal(d1, d2)
    # a jittered update samples other points; with decay 0.5, cells empty in the
    # new query keep half of the old density
    d3 = d1.copy()
    om.occupancy_ema(poses[1], d3, S.occupancy_jitter(sc, 1), decay=0.5)
    s_new = np.zeros(R ** 3)
    om.occupancy_ema(poses[1], s_new, S.occupancy_jitter(sc, 1), decay=0.0)
    np.testing.assert_allclose(d3, np.maximum(0.5 * d1, s_new), rtol=0, atol=0)
    assert np.any(d3 == 0.5 * d1) and np.any(d3 == s_new)


@pytest.fixture(scope="module")
def reg_case(tiny):
    sc, om, poses = tiny
    occ = om.occupancy(poses[0])[1] | om.occupancy(poses[1])[1]
    rng = np.random.default_rng(4)
    holes = occ & rng.integers(0, 2 ** 32, size=occ.shape, dtype=np.uint64).astype(np.uint32)
    x = S.random_points(sc, 4000, seed=9)
    pid = rng.integers(0, 2, size=len(x)).astype(np.int32)
    loss, flags = G.density_reg(om, poses, holes, x, pid, 0.3)
    keep = flags == 0
    return sc, om, poses, holes, x[keep], pid[keep]


def _grads(sc, om, n_poses):
    return dict(table=np.zeros((sc.n_table_entries(), sc.n_features)), mlp=np.zeros(G.mlp_size(sc)),
                skin=np.zeros(om.skin.shape), bones=np.zeros((n_poses, sc.n_bones, 12)))


def test_regulariser_gradient_matches_central_differences(reg_case):
    sc, om, poses, occ, x, pid = reg_case
    g = _grads(sc, om, len(poses))
    loss, _ = G.density_reg(om, poses, occ, x, pid, 0.3, g)
    assert loss > 0

    def L(pp=poses):
        return G.density_reg(om, pp, occ, x, pid, 0.3)[0]

    rng = np.random.default_rng(2)
    worst = 0.0
    checks = 0
    for arr, flat in ((om.table.reshape(-1), g["table"].reshape(-1)), (om.skin.reshape(-1), g["skin"].reshape(-1)),
                      (om.mlp["W1"].reshape(-1), g["mlp"][:om.mlp["W1"].size])):
        nz = np.flatnonzero(np.abs(flat) > 1e-6 * np.abs(flat).max())
        for i in rng.choice(nz, size=min(8, len(nz)), replace=False):
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
    print(f"{checks} finite-difference checks of the regulariser, worst relative error {worst:.2e}")
    assert checks == 32


def test_regulariser_is_zero_where_cells_are_occupied(reg_case):
    sc, om, poses, occ, x, pid = reg_case
    full = np.full_like(occ, 0xFFFFFFFF)
    g = _grads(sc, om, len(poses))
    loss, _ = G.density_reg(om, poses, full, x, pid, 0.3, g)
    assert loss == 0.0
    for v in g.values():
        assert not np.any(v)


def test_regulariser_with_an_empty_grid_is_the_mean_density(reg_case):
    sc, om, poses, occ, x, pid = reg_case
    empty = np.zeros_like(occ)
    loss, _ = G.density_reg(om, poses, empty, x, pid, 0.3)
    sig = [om.posed_field(poses[p], xi.astype(np.float64)) for xi, p in zip(x, pid)]
    ref = 0.3 * np.mean([s["sigma"] if s["start"] >= 0 else 0.0 for s in sig])
    assert abs(loss - ref) <= 1e-12 * ref
