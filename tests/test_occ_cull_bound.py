"""The bound behind the occupancy culling, checked against the fp64 oracle's
roots on the CPU (no GPU).

Inside one cell of the skinning grid the blended LBS map is
f(x) = sum_c w_c (A_c v_c + t_c) + sum_c w_c (A_c - A0)(x - v_c) (trilinear
weights reproduce affine functions), so f(cell) lies in the bounding box of the
corner images grown by max_c sum_j |A_c - A0|_kj h_j per component.  Every cell
of the occupancy grid whose centre has a root in the oracle's search must fall
in one of these boxes (grown by the Broyden tolerance and 1e-4 of the scene's
largest coordinate), or the culled search would drop a root: at the
resolution of the sub-cell masks (a box marks the occupancy cells it meets),
and for the centre queries of the occupancy refresh, point by point (the
centre itself lies in a box).  The CUDA kernels' use of the same boxes is
checked on the GPU (culling on and off give the same densities)."""
import numpy as np
import pytest

import oracle as O
import synthetic as S


def candidate_cells(sc, N, pts=None):
    """Occupancy cells met by some skinning cell's image box, and those whose
    query point (the centre, or pts [R^3][3], one point inside each cell) lies
    in one (fp32 blended grid, bounds in fp64)."""
    Rw = sc.skin_res
    w = sc.skin_grid.reshape(Rw, Rw, Rw, -1).astype(np.float64)  # [z, y, x, bone]
    M = np.einsum("zyxk,kij->zyxij", w, N).astype(np.float32).astype(np.float64)
    cmin, cmax = sc.canon_min.astype(np.float64), sc.canon_max.astype(np.float64)
    nc = Rw - 1
    h = (cmax - cmin) / nc
    R = sc.occ_res
    nmin, nmax = sc.norm_min.astype(np.float64), sc.norm_max.astype(np.float64)
    scale = R / (nmax - nmin)
    L = max(np.abs(cmin).max(), np.abs(cmax).max(), np.abs(nmin).max(), np.abs(nmax).max())
    slack = sc.broyden_tol + 1e-4 * L
    i = np.arange(nc)
    cz, cy, cx = np.meshgrid(i, i, i, indexing="ij")
    lo = np.full((nc, nc, nc, 3), np.inf)
    hi = np.full((nc, nc, nc, 3), -np.inf)
    A = []
    for corner in range(8):
        ox, oy, oz = corner & 1, (corner >> 1) & 1, (corner >> 2) & 1
        Mc = M[cz + oz, cy + oy, cx + ox]
        v = np.stack([cmin[0] + (cx + ox) * h[0], cmin[1] + (cy + oy) * h[1], cmin[2] + (cz + oz) * h[2]], -1)
        img = np.einsum("...ij,...j->...i", Mc[..., :3], v) + Mc[..., 3]
        lo, hi = np.minimum(lo, img), np.maximum(hi, img)
        A.append(Mc[..., :3])
    A = np.stack(A)
    margin = (np.abs(A - A.mean(0)) * h).sum(-1).max(0)
    f0 = np.floor((lo - margin - slack - nmin) * scale)
    f1 = np.floor((hi + margin + slack - nmin) * scale)
    hit = (f1 >= 0).all(-1) & (f0 <= R - 1).all(-1)
    i0 = np.clip(f0, 0, R - 1).astype(int)[hit]
    i1 = np.clip(f1, 0, R - 1).astype(int)[hit]
    blo = (lo - margin - slack)[hit]
    bhi = (hi + margin + slack)[hit]
    mask = np.zeros((R, R, R), bool)
    centre = np.zeros((R, R, R), bool)
    span = (i1 - i0).max(0) + 1
    for dz in range(span[2]):
        for dy in range(span[1]):
            for dx in range(span[0]):
                d = np.array([dx, dy, dz])
                ok = (i0 + d <= i1).all(-1)
                q = i0[ok] + d
                mask[q[:, 2], q[:, 1], q[:, 0]] = True
                cq = q[:, 0] + R * (q[:, 1] + R * q[:, 2])
                xc = nmin + (q + 0.5) / scale if pts is None else pts[cq]
                inside = ((xc >= blo[ok]) & (xc <= bhi[ok])).all(-1)
                qi = q[inside]
                centre[qi[:, 2], qi[:, 1], qi[:, 0]] = True
    return mask.reshape(-1), centre.reshape(-1)


@pytest.mark.parametrize("config,seeds", [("tiny", (1, 2, 3)), ("full", (6,))])
def test_every_rooted_cell_is_a_candidate(config, seeds):
    sc = S.make_scene(config, 0)
    table, mlp = S.make_field(sc, 0)
    om = O.OracleModel(sc, table, mlp)
    for seed in seeds:
        p = om.pose(*S.make_pose(sc, seed))
        cand, centre = candidate_cells(sc, om.transforms(p)["N"])
        sigma, _ = om.occupancy(p)
        rooted = sigma > 0
        print(f"{config} pose {seed}: rooted {rooted.sum()}, centre candidates {centre.sum()}, "
              f"sub-cell candidates {cand.sum()} of {cand.size}")
        assert rooted.any()
        assert not (rooted & ~cand).any()
        assert not (rooted & ~centre).any()
        assert not (centre & ~cand).any()  # the point test only removes candidates
        if config == "full":
            assert cand.sum() < 0.3 * cand.size  # the bound is tight enough to pay


def test_every_rooted_point_is_in_a_box():
    """The render's fallback skips a sample whose point lies in no box: checked
    at one uniformly drawn point inside every occupancy cell of a full-size
    pose (fp32 positions as the GPU forms them), against the oracle's roots."""
    sc = S.make_scene("full", 0)
    table, mlp = S.make_field(sc, 0)
    om = O.OracleModel(sc, table, mlp)
    p = om.pose(*S.make_pose(sc, 7))
    R = sc.occ_res
    u = np.random.default_rng(11).random((R ** 3, 3), dtype=np.float32)
    d = np.zeros(R ** 3)
    om.occupancy_ema(p, d, jitter=u, decay=0.0)  # d = sigma at the drawn points
    c = np.arange(R ** 3)
    ci = np.stack([c % R, (c // R) % R, c // (R * R)], -1).astype(np.float32)
    nmin = sc.norm_min.astype(np.float32)
    cs = ((sc.norm_max - sc.norm_min) / R).astype(np.float32)
    pts = ((ci + u) * cs + nmin).astype(np.float64)  # cell_point: three rounded fp32 operations
    cand, inbox = candidate_cells(sc, om.transforms(p)["N"], pts)
    rooted = d > 0
    print(f"rooted points {rooted.sum()}, in a box {inbox.sum()}, in a met cell {cand.sum()} of {R ** 3}")
    assert rooted.any()
    assert not (rooted & ~inbox).any()
