"""Seeded synthetic inputs for the articulated-avatar render path.

Everything in this module is *input construction*: skeleton topologies and bone
lengths, poses, skinning-weight voxel grids, a radiance-field fixture (hash-table
entries and MLP weights), cameras and ray batches.  No step of the render path
itself (pose chain, skinning, root finding, encoding, MLP, compositing) is
computed here; the CPU oracle and the CUDA library both consume these arrays and
neither is imported from here.

The paper trains on PeopleSnapshot / SURREAL videos with SMPL skinning weights
(Sec. 3.1, Sec. 4.1); none of those are available, so these generators stand in
for them with seeded analytic shapes:

* configuration "tiny":  an 8-bone chain (bone lengths U(0.1, 0.3) m), a union of
  radius-0.06 m capsules, 32^3 x 8 skinning grid, 8 x 2 hash grid (T = 2^14),
  one 64 x 64 pinhole view, <= 32 samples per ray.
* configuration "full":  a 24-joint SMPL-like tree (pelvis, spine, neck/head,
  two arms, two legs), bone lengths U(0.05, 0.4) m, 64^3 x 24 skinning grid,
  16 x 2 hash grid (T = 2^19, resolutions 16 .. 2048), a 540 x 540 pinhole view
  with a 1200 px focal length, <= 128 samples per ray.

Skinning weights are softmax_i(-d_i(v) / 0.05) with d_i the distance from grid
vertex v to the segments of bone i (rows sum to one).  The radiance-field
fixture writes a smoothed signed distance of the capsule union (and a per-bone
colour code) into the dense (coarse) hash levels and builds MLP weights that
turn it into density and colour, so that occupancy, empty-space skipping and
multi-root selection see a body-shaped field instead of noise.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# SMPL kinematic tree (24 joints): parent of each joint, root = -1.
SMPL_PARENTS = np.array(
    [-1, 0, 0, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 9, 9, 12, 13, 14, 16, 17, 18, 19, 20, 21],
    dtype=np.int32)

# Canonical (T-pose) direction of the offset from each joint's parent to the joint.
_SMPL_DIRS = np.array([
    [0, 0, 0],       # 0 pelvis (root)
    [1, -0.4, 0],    # 1 left hip
    [-1, -0.4, 0],   # 2 right hip
    [0, 1, 0],       # 3 spine1
    [0, -1, 0],      # 4 left knee
    [0, -1, 0],      # 5 right knee
    [0, 1, 0],       # 6 spine2
    [0, -1, 0],      # 7 left ankle
    [0, -1, 0],      # 8 right ankle
    [0, 1, 0],       # 9 spine3
    [0, -0.3, 1],    # 10 left foot
    [0, -0.3, 1],    # 11 right foot
    [0, 1, 0],       # 12 neck
    [1, 0.3, 0],     # 13 left collar
    [-1, 0.3, 0],    # 14 right collar
    [0, 1, 0],       # 15 head
    [1, 0, 0],       # 16 left shoulder
    [-1, 0, 0],      # 17 right shoulder
    [1, 0, 0],       # 18 left elbow
    [-1, 0, 0],      # 19 right elbow
    [1, 0, 0],       # 20 left wrist
    [-1, 0, 0],      # 21 right wrist
    [1, 0, 0],       # 22 left hand
    [-1, 0, 0],      # 23 right hand
], dtype=np.float64)

# Capsule radius per SMPL bone (torso and head thicker than limbs).
_SMPL_RADII = np.array([0.14, 0.09, 0.09, 0.15, 0.07, 0.07, 0.15, 0.05, 0.05, 0.13,
                        0.045, 0.045, 0.06, 0.07, 0.07, 0.11, 0.065, 0.065, 0.055, 0.055,
                        0.045, 0.045, 0.04, 0.04])

HASH_PRIMES = (1, 2654435761, 805459861)  # published Instant-NGP spatial-hash primes


@dataclasses.dataclass
class Scene:
    """One synthetic articulated subject plus the sizes of the render path."""
    name: str
    n_bones: int
    parents: np.ndarray          # int32 [nb], -1 for the root, parents precede children
    rest_joints: np.ndarray      # float64 [nb, 3], canonical rest-pose joint positions
    seg_a: np.ndarray            # float64 [S, 3] capsule segment starts (canonical)
    seg_b: np.ndarray            # float64 [S, 3] capsule segment ends
    seg_bone: np.ndarray         # int32 [S] bone owning each segment
    seg_radius: np.ndarray       # float64 [S]
    skin_res: int                # skinning grid vertices per axis
    skin_grid: np.ndarray        # float32 [R, R, R, nb] indexed [z, y, x, i]
    canon_min: np.ndarray        # float32 [3] canonical box (skinning + hash grids)
    canon_max: np.ndarray        # float32 [3]
    norm_min: np.ndarray         # float32 [3] normalised-space box (occupancy + march)
    norm_max: np.ndarray         # float32 [3]
    occ_res: int
    n_levels: int
    n_features: int
    log2_table: int
    level_res: np.ndarray        # int32 [L]
    mlp_width: int
    max_samples: int
    broyden_max_iter: int
    broyden_tol: float
    occ_tau: float
    occ_dilate: int
    pose_angle_max: float
    root_trans_max: float
    image_w: int
    image_h: int
    focal: float

    # ---- storage format of the hash table (documented layout, not arithmetic) ----
    def level_sizes(self) -> np.ndarray:
        T = 1 << self.log2_table
        return np.array([min((int(r) + 1) ** 3, T) for r in self.level_res], dtype=np.int64)

    def level_offsets(self) -> np.ndarray:
        s = self.level_sizes()
        return np.concatenate([[0], np.cumsum(s)[:-1]]).astype(np.int64)

    def n_table_entries(self) -> int:
        return int(self.level_sizes().sum())

    def dense_levels(self) -> list:
        T = 1 << self.log2_table
        return [l for l, r in enumerate(self.level_res) if (int(r) + 1) ** 3 <= T]

    def mlp_in(self) -> int:
        return self.n_levels * self.n_features


def level_resolutions(n_levels: int, base: int, growth: float | None = None,
                      max_res: int | None = None) -> np.ndarray:
    """Per-level grid resolution floor(base * b^l), b from growth or from max_res.

    Computed once on the host and handed to both the oracle and the library so
    that an fp rounding of base*b^l just below an integer cannot split them.
    """
    if growth is None:
        growth = math.exp((math.log(max_res) - math.log(base)) / (n_levels - 1))
    return np.array([int(math.floor(base * growth ** l + 1e-9)) for l in range(n_levels)],
                    dtype=np.int32)


def _seg_dist(p: np.ndarray, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Distance from points p [..., 3] to segment a-b."""
    ab = b - a
    t = np.clip(((p - a) @ ab) / max(float(ab @ ab), 1e-30), 0.0, 1.0)
    q = a + t[..., None] * ab
    return np.linalg.norm(p - q, axis=-1)


def _bone_segments(parents, joints, dirs, leaf_len):
    """Segments per bone: joint k to each child; leaves extend along their own direction."""
    nb = len(parents)
    children = [[] for _ in range(nb)]
    for k in range(1, nb):
        children[parents[k]].append(k)
    sa, sb, sk = [], [], []
    for k in range(nb):
        if children[k]:
            for c in children[k]:
                sa.append(joints[k]); sb.append(joints[c]); sk.append(k)
        else:
            d = dirs[k] / np.linalg.norm(dirs[k])
            sa.append(joints[k]); sb.append(joints[k] + leaf_len * d); sk.append(k)
    return np.array(sa), np.array(sb), np.array(sk, dtype=np.int32)


def _skin_grid(nb, seg_a, seg_b, seg_bone, cmin, cmax, R, temp=0.05):
    lin = [np.linspace(cmin[d], cmax[d], R) for d in range(3)]
    z, y, x = np.meshgrid(lin[2], lin[1], lin[0], indexing="ij")
    p = np.stack([x, y, z], axis=-1)  # [R, R, R, 3] indexed [z, y, x]
    dist = np.full(p.shape[:3] + (nb,), np.inf)
    for s in range(len(seg_a)):
        k = seg_bone[s]
        dist[..., k] = np.minimum(dist[..., k], _seg_dist(p, seg_a[s], seg_b[s]))
    logits = -dist / temp
    logits -= logits.max(axis=-1, keepdims=True)
    w = np.exp(logits)
    w /= w.sum(axis=-1, keepdims=True)
    return w.astype(np.float32)


def make_scene(config: str = "tiny", seed: int = 0, skin_res: int | None = None) -> Scene:
    """Build the seeded subject for configuration 'tiny' or 'full'."""
    rng = np.random.default_rng(seed)
    if config == "tiny":
        nb = 8
        parents = np.arange(-1, nb - 1, dtype=np.int32)
        lengths = rng.uniform(0.1, 0.3, size=nb)
        joints = np.zeros((nb, 3))
        for k in range(1, nb):
            joints[k] = joints[k - 1] + np.array([0.0, lengths[k - 1], 0.0])
        dirs = np.tile(np.array([0.0, 1.0, 0.0]), (nb, 1))
        seg_a, seg_b, seg_bone = _bone_segments(parents, joints, dirs, lengths[-1])
        seg_r = np.full(len(seg_a), 0.06)
        sres = 32 if skin_res is None else skin_res
        reach = float(lengths.sum())
        kw = dict(occ_res=32, n_levels=8, log2_table=14,
                  level_res=level_resolutions(8, 16, growth=1.5), max_samples=32,
                  pose_angle_max=0.5, root_trans_max=0.0, image_w=64, image_h=64)
    elif config == "full":
        nb = 24
        parents = SMPL_PARENTS.copy()
        lengths = rng.uniform(0.05, 0.4, size=nb)
        joints = np.zeros((nb, 3))
        dirs = _SMPL_DIRS.copy()
        for k in range(1, nb):
            d = dirs[k] / np.linalg.norm(dirs[k])
            joints[k] = joints[parents[k]] + lengths[k] * d
        seg_a, seg_b, seg_bone = _bone_segments(parents, joints, dirs, 0.1)
        seg_r = _SMPL_RADII[seg_bone]
        sres = 64 if skin_res is None else skin_res
        # farthest canonical joint chain from the pelvis bounds any articulated reach
        reach = float(np.max(np.linalg.norm(seg_b - joints[0], axis=-1)))
        kw = dict(occ_res=64, n_levels=16, log2_table=19,
                  level_res=level_resolutions(16, 16, max_res=2048), max_samples=128,
                  pose_angle_max=0.6, root_trans_max=0.2, image_w=540, image_h=540)
    else:
        raise ValueError(config)

    margin = 0.12
    lo = np.minimum(seg_a, seg_b).min(axis=0) - margin
    hi = np.maximum(seg_a, seg_b).max(axis=0) + margin
    canon_min, canon_max = lo.astype(np.float32), hi.astype(np.float32)
    half = reach + 0.15
    norm_min = (joints[0] - half).astype(np.float32)
    norm_max = (joints[0] + half).astype(np.float32)
    skin = _skin_grid(nb, seg_a, seg_b, seg_bone, canon_min.astype(np.float64),
                      canon_max.astype(np.float64), sres)
    focal = 1200.0 if config == "full" else 0.0
    sc = Scene(name=config, n_bones=nb, parents=parents, rest_joints=joints,
               seg_a=seg_a, seg_b=seg_b, seg_bone=seg_bone, seg_radius=seg_r,
               skin_res=sres, skin_grid=skin, canon_min=canon_min, canon_max=canon_max,
               norm_min=norm_min, norm_max=norm_max, n_features=2, mlp_width=64,
               broyden_max_iter=10, broyden_tol=1e-5, occ_tau=0.01, occ_dilate=1,
               focal=focal, **kw)
    if config == "tiny":
        sc.focal = 80.0
    return sc


def capsule_sdf(scene: Scene, p: np.ndarray) -> tuple:
    """Signed distance to the capsule union (negative inside) and the nearest bone."""
    best = np.full(p.shape[:-1], np.inf)
    bone = np.zeros(p.shape[:-1], dtype=np.int32)
    for s in range(len(scene.seg_a)):
        d = _seg_dist(p, scene.seg_a[s], scene.seg_b[s]) - scene.seg_radius[s]
        m = d < best
        best = np.where(m, d, best)
        bone = np.where(m, scene.seg_bone[s], bone)
    return best, bone


def make_field(scene: Scene, seed: int = 0, width: float = 0.05, perturb: float = 0.0):
    """Radiance-field fixture: hash table [entries, F] and MLP weights (fp32).

    Hashed (fine) levels hold U(-1e-4, 1e-4) noise, as a freshly initialised
    hash grid does.  Dense (coarse) levels hold, at each grid vertex, feature 0 =
    tanh(-sdf / width) and feature 1 = a colour code of the nearest bone.  The
    MLP averages those over the dense levels into four hidden units carried
    through both layers; density = exp(6 s - 1), colour = sigmoid of the colour
    code.  All remaining weights are small seeded noise so that every layer does
    its full work.  `perturb` > 0 adds N(0, perturb) to table and weights (a
    seed-perturbed field, used to make training targets).
    """
    rng = np.random.default_rng(10_000 + seed)
    L, F = scene.n_levels, scene.n_features
    sizes, offs = scene.level_sizes(), scene.level_offsets()
    table = rng.uniform(-1e-4, 1e-4, size=(scene.n_table_entries(), F)).astype(np.float64)
    cmin = scene.canon_min.astype(np.float64)
    ext = scene.canon_max.astype(np.float64) - cmin
    dense = scene.dense_levels()
    for l in dense:
        r = int(scene.level_res[l])
        g = np.arange(r + 1, dtype=np.float64) / r
        z, y, x = np.meshgrid(g, g, g, indexing="ij")
        # dense storage format: entry i + (r+1) * (j + (r+1) * k) for vertex (i, j, k)
        p = cmin + np.stack([x, y, z], axis=-1) * ext
        sdf, bone = capsule_sdf(scene, p)
        f0 = np.tanh(-sdf / width)
        f1 = 2.0 * bone / max(scene.n_bones - 1, 1) - 1.0
        table[offs[l]:offs[l] + sizes[l], 0] = f0.reshape(-1)
        table[offs[l]:offs[l] + sizes[l], 1] = f1.reshape(-1)
    W = scene.mlp_width
    nin = scene.mlp_in()
    W1 = rng.normal(0.0, 0.05, size=(W, nin))
    b1 = rng.normal(0.0, 0.02, size=W)
    W2 = rng.normal(0.0, 0.05, size=(W, W))
    b2 = rng.normal(0.0, 0.02, size=W)
    W3 = rng.normal(0.0, 0.02, size=(4, W))
    b3 = rng.normal(0.0, 0.02, size=4)
    nd = float(len(dense))
    W1[:4, :] *= 0.02
    b1[:4] = 0.0
    for l in dense:
        W1[0, l * F + 0] = 1.0 / nd
        W1[1, l * F + 0] = -1.0 / nd
        W1[2, l * F + 1] = 1.0 / nd
        W1[3, l * F + 1] = -1.0 / nd
    W2[:4, :] *= 0.02
    W2[:4, :4] += np.eye(4)
    b2[:4] = 0.0
    W3[0, 0], W3[0, 1], b3[0] = 6.0, -6.0, -1.0
    for c, g in enumerate((2.0, -1.5, 1.0)):
        W3[1 + c, 2] += g
        W3[1 + c, 3] -= g
    mlp = dict(W1=W1, b1=b1, W2=W2, b2=b2, W3=W3, b3=b3)
    if perturb > 0.0:
        prng = np.random.default_rng(20_000 + seed)
        table = table + prng.normal(0.0, perturb, size=table.shape)
        mlp = {k: v + prng.normal(0.0, perturb, size=v.shape) for k, v in mlp.items()}
    return table.astype(np.float32), {k: v.astype(np.float32) for k, v in mlp.items()}


def make_pose(scene: Scene, seed: int) -> tuple:
    """Axis-angle per joint (uniform axis, angle U(0, max)) and root translation (fp64)."""
    rng = np.random.default_rng(1_000 + seed)
    axis = rng.normal(size=(scene.n_bones, 3))
    axis /= np.linalg.norm(axis, axis=-1, keepdims=True)
    ang = rng.uniform(0.0, scene.pose_angle_max, size=(scene.n_bones, 1))
    theta = (axis * ang).astype(np.float64)
    trans = rng.uniform(-scene.root_trans_max, scene.root_trans_max, size=3) \
        if scene.root_trans_max > 0 else np.zeros(3)
    return theta, trans.astype(np.float64)


def make_camera(scene: Scene, width: int | None = None, height: int | None = None) -> dict:
    """Pinhole camera looking at the root joint along -z (OpenCV axes: x right, y down).

    Returns fx, fy, cx, cy, width, height and the 3x4 camera-to-world matrix (fp32).
    """
    W = scene.image_w if width is None else width
    H = scene.image_h if height is None else height
    target = scene.rest_joints[0].copy()
    if scene.name == "full":
        # ~4 m away, pulled back until the canonical box fits the view with 10% slack
        target = 0.5 * (scene.canon_min + scene.canon_max).astype(np.float64)
        half_xy = 0.5 * float(np.max((scene.canon_max - scene.canon_min)[:2]))
        dist = max(4.0, 1.1 * half_xy * scene.focal / (0.5 * scene.image_w))
    else:
        # frame the chain's canonical box with 30% slack (its pose bends it moderately)
        target = 0.5 * (scene.canon_min + scene.canon_max).astype(np.float64)
        half = 0.5 * float(np.max(scene.canon_max - scene.canon_min))
        dist = 1.3 * half * scene.focal / (0.5 * scene.image_w)
    pos = target + np.array([0.0, 0.0, dist])
    R = np.array([[1.0, 0.0, 0.0], [0.0, -1.0, 0.0], [0.0, 0.0, -1.0]]).T  # columns: x, y, z axes
    c2w = np.concatenate([R, pos[:, None]], axis=1).astype(np.float32)
    f = scene.focal * (W / scene.image_w)
    return dict(fx=np.float32(f), fy=np.float32(f), cx=np.float32(0.5 * W),
                cy=np.float32(0.5 * H), width=int(W), height=int(H), c2w=c2w)


def pixel_rays(scene: Scene) -> tuple:
    """World origin and unit direction (fp32 [H*W][3] each) of every pixel centre
    of the default camera, pixel v * W + u, as make_ray_batch draws them."""
    cam = make_camera(scene)
    v, u = np.meshgrid(np.arange(cam["height"]), np.arange(cam["width"]), indexing="ij")
    u, v = u.reshape(-1), v.reshape(-1)
    dc = np.stack([(u + 0.5 - cam["cx"]) / cam["fx"], (v + 0.5 - cam["cy"]) / cam["fy"], np.ones(u.size)], axis=-1)
    d = dc @ cam["c2w"][:, :3].astype(np.float64).T
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    o = np.broadcast_to(cam["c2w"][:, 3].astype(np.float64), d.shape)
    return np.ascontiguousarray(o, dtype=np.float32), d.astype(np.float32)


def init_field(scene: Scene, seed: int = 0):
    """A seeded untrained field (the start of a training run from scratch): table
    U(-1e-4, 1e-4), He-normal MLP weights, zero biases."""
    rng = np.random.default_rng(80_000 + seed)
    table = rng.uniform(-1e-4, 1e-4, size=(scene.n_table_entries(), scene.n_features)).astype(np.float32)
    W, nin = scene.mlp_width, scene.mlp_in()
    mlp = {}
    for name, (o, n) in (("1", (W, nin)), ("2", (W, W)), ("3", (4, W))):
        mlp["W" + name] = rng.normal(0.0, np.sqrt(2.0 / n), size=(o, n)).astype(np.float32)
        mlp["b" + name] = np.zeros(o, np.float32)
    return table, mlp


def perturb_field(table: np.ndarray, mlp: dict, seed: int, table_std: float, weight_std: float):
    """A seeded perturbation of a field (the start of a training run): Gaussian
    noise on every table entry and on the MLP weights."""
    rng = np.random.default_rng(70_000 + seed)
    t = (table + rng.normal(0.0, table_std, table.shape)).astype(np.float32)
    m = {k: (v + rng.normal(0.0, weight_std, v.shape)).astype(np.float32) if k.startswith("W") else v.copy()
         for k, v in mlp.items()}
    return t, m


def make_ray_batch(scene: Scene, n_rays: int, n_poses: int, seed: int = 0) -> dict:
    """Random training rays: pose index, pixel, world origin/direction, target rgb.

    Directions are the pinhole ray of a uniformly drawn pixel centre of the
    default camera (fp32, same convention as make_camera); targets are U(0, 1)
    unless replaced by rendered colours.
    """
    rng = np.random.default_rng(30_000 + seed)
    cam = make_camera(scene)
    pose = rng.integers(0, n_poses, size=n_rays).astype(np.int32)
    u = rng.integers(0, cam["width"], size=n_rays)
    v = rng.integers(0, cam["height"], size=n_rays)
    dc = np.stack([(u + 0.5 - cam["cx"]) / cam["fx"], (v + 0.5 - cam["cy"]) / cam["fy"],
                   np.ones(n_rays)], axis=-1)
    d = dc @ cam["c2w"][:, :3].astype(np.float64).T
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    o = np.broadcast_to(cam["c2w"][:, 3].astype(np.float64), d.shape)
    target = rng.uniform(0.0, 1.0, size=(n_rays, 3))
    return dict(origin=np.ascontiguousarray(o, dtype=np.float32),
                direction=d.astype(np.float32), pose=pose,
                target=target.astype(np.float32), pixel_u=u.astype(np.int32),
                pixel_v=v.astype(np.int32))


def pack_mlp(mlp: dict) -> np.ndarray:
    """Flatten MLP weights in the order W1, b1, W2, b2, W3, b3 (row-major [out, in])."""
    return np.concatenate([mlp[k].reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]
                          ).astype(np.float32)


def occupancy_jitter(scene: Scene, seed: int = 0) -> np.ndarray:
    """Per-cell offsets u in [0, 1)^3 (fp32 [R^3][3]) of the points a training-mode
    occupancy update queries inside each cell (the random draw is an input)."""
    rng = np.random.default_rng(60_000 + seed)
    return rng.uniform(0.0, 1.0, size=(scene.occ_res ** 3, 3)).astype(np.float32)


def random_points(scene: Scene, n: int, seed: int = 0, box: str = "norm") -> np.ndarray:
    """Uniform fp32 points in the normalised (or canonical) box."""
    rng = np.random.default_rng(40_000 + seed)
    lo, hi = (scene.norm_min, scene.norm_max) if box == "norm" else (scene.canon_min, scene.canon_max)
    return rng.uniform(lo, hi, size=(n, 3)).astype(np.float32)


def proposal_config(n_levels: int = 8, log2_table: int = 16, base: int = 8, growth: float = 1.5,
                    top_k: int = 2, offset_weight: float = 100.0) -> dict:
    """Sizes of the correspondence-proposal network (posed-space hash grid over
    the normalised box, 64-wide MLP with three hidden layers)."""
    return dict(n_levels=n_levels, log2_table=log2_table, level_res=level_resolutions(n_levels, base, growth=growth),
                top_k=top_k, offset_weight=offset_weight)


def proposal_init(scene: Scene, cfg: dict, seed: int = 0):
    """Seeded initial proposal parameters: table U(-1e-4, 1e-4), He-normal weights, zero biases.
    Returns the table [entries, 2] and the MLP dict (W1 [64, 2L+3nb], b1, W2, b2, W3, b3, W4 [nb+3, 64], b4)."""
    rng = np.random.default_rng(50_000 + seed)
    T = 1 << cfg["log2_table"]
    entries = sum(min((int(r) + 1) ** 3, T) for r in cfg["level_res"])
    table = rng.uniform(-1e-4, 1e-4, size=(entries, 2))
    nin = 2 * cfg["n_levels"] + 3 * scene.n_bones
    dims = [(64, nin), (64, 64), (64, 64), (scene.n_bones + 3, 64)]
    mlp = {}
    for i, (o, n) in enumerate(dims, start=1):
        mlp[f"W{i}"] = rng.normal(0.0, np.sqrt(2.0 / n), size=(o, n))
        mlp[f"b{i}"] = np.zeros(o)
    return table.astype(np.float32), {k: v.astype(np.float32) for k, v in mlp.items()}


def pack_proposal(mlp: dict) -> np.ndarray:
    return np.concatenate([mlp[k].reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")]
                          ).astype(np.float32)
