"""ctypes wrapper of the oracle's training step (oracle_grad.c).  TEST
INFRASTRUCTURE ONLY: L2 photometric loss over a ray batch and its fp64
reverse-mode gradient (compositing, MLP, hash table, and the implicit-function
gradient through the root to the skinning grid and bone transforms)."""
import ctypes as C

import numpy as np


def declare(L):
    from . import Model, Pose
    P = C.POINTER
    L.or_train.restype = C.c_double
    L.or_train.argtypes = [P(Model), P(Pose), C.c_int, P(C.c_uint32), C.c_int, P(C.c_float), P(C.c_float),
                           P(C.c_int32), P(C.c_double), P(C.c_double), P(C.c_int32), P(C.c_double),
                           P(C.c_double), P(C.c_double), P(C.c_double), C.c_int]
    L.or_train_loss.restype = C.c_double
    L.or_train_loss.argtypes = L.or_train.argtypes + [P(Loss)]
    L.or_train_upstream.restype = None
    L.or_train_upstream.argtypes = [P(Model), P(Pose), C.c_int, P(C.c_uint32), C.c_int, P(C.c_float), P(C.c_float),
                                    P(C.c_int32), P(C.c_double), P(C.c_double), P(C.c_double), P(C.c_double),
                                    P(C.c_int32), P(C.c_double), P(C.c_double), P(C.c_double), P(C.c_double),
                                    C.c_int]
    L.or_density_reg.restype = C.c_double
    L.or_density_reg.argtypes = [P(Model), P(Pose), C.c_int, P(C.c_uint32), C.c_int, P(C.c_float), P(C.c_int32),
                                 C.c_double, P(C.c_int32), P(C.c_double), P(C.c_double), P(C.c_double),
                                 P(C.c_double)]


class Loss(C.Structure):
    _fields_ = [("huber", C.c_int), ("delta", C.c_double), ("w_rgb", C.c_double), ("w_alpha", C.c_double),
                ("w_hard", C.c_double), ("alpha_target", C.POINTER(C.c_double))]


def pose_array(poses):
    from . import Pose
    arr = (Pose * len(poses))()
    for i, p in enumerate(poses):
        C.memmove(C.byref(arr[i]), C.byref(p), C.sizeof(Pose))
    return arr


def mlp_size(sc):
    W = sc.mlp_width
    return W * sc.mlp_in() + W + W * W + W + 4 * W + 4


def train(om, poses, occ_bits, origin, direction, pose_id, target, grad=True, nthreads=0, prop=None,
          theta=None, fallbacks=None, loss=None):
    """Loss, per-ray colour and flags, and (if grad) the gradients as a dict:
    table [entries, F], mlp (packed W1, b1, W2, b2, W3, b3), skin [R, R, R, nb],
    bones [n_poses, nb, 12] (gradient w.r.t. the normalised-space N_k).
    With prop (an oracle.prop.PropModel) and theta ([n_poses, nb, 3] axis-angles)
    the proposal chooses each sample's starts; fallbacks (int32 [n], optional)
    then receives each ray's count of samples that fell back to every bone.
    loss: dict(huber, delta, w_rgb, w_alpha, w_hard, alpha_target) for the loss
    set of Sec. 3.4 (default: L2 over the colour channels)."""
    from . import _p
    sc = om.scene
    n = len(pose_id)
    arr = pose_array(poses) if isinstance(poses, (list, tuple)) else poses
    n_poses = len(arr)
    o = np.ascontiguousarray(origin, dtype=np.float32)
    d = np.ascontiguousarray(direction, dtype=np.float32)
    pid = np.ascontiguousarray(pose_id, dtype=np.int32)
    tgt = np.ascontiguousarray(target, dtype=np.float64)
    occ = np.ascontiguousarray(occ_bits, dtype=np.uint32)
    rgb = np.zeros((n, 3))
    flags = np.zeros(n, dtype=np.int32)
    g = None
    if grad:
        g = dict(table=np.zeros((sc.n_table_entries(), sc.n_features)), mlp=np.zeros(mlp_size(sc)),
                 skin=np.zeros(om.skin.shape), bones=np.zeros((n_poses, sc.n_bones, 12)))
    args = [g[k] if g else None for k in ("table", "mlp", "skin", "bones")]
    common = [C.byref(om.m), arr, n_poses, _p(occ, C.c_uint32), n, _p(o, C.c_float), _p(d, C.c_float),
              _p(pid, C.c_int32), _p(tgt, C.c_double), _p(rgb, C.c_double), _p(flags, C.c_int32),
              *[_p(a, C.c_double) for a in args], nthreads]
    if loss is not None:
        assert prop is None
        lc = Loss()
        lc.huber, lc.delta = int(loss.get("huber", 0)), float(loss.get("delta", 0.1))
        lc.w_rgb, lc.w_alpha, lc.w_hard = (float(loss.get(k, d)) for k, d in
                                           (("w_rgb", 1.0), ("w_alpha", 0.0), ("w_hard", 0.0)))
        at = np.ascontiguousarray(loss.get("alpha_target", np.zeros(n)), dtype=np.float64)
        assert at.shape == (n,)
        lc.alpha_target = _p(at, C.c_double)
        loss = om.L.or_train_loss(*common, C.byref(lc))
    elif prop is None:
        loss = om.L.or_train(*common)
    else:
        th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1)
        assert th.size == n_poses * sc.n_bones * 3
        fb = None
        if fallbacks is not None:
            assert fallbacks.dtype == np.int32 and fallbacks.shape == (n,) and fallbacks.flags.c_contiguous
            fb = _p(fallbacks, C.c_int32)
        loss = om.L.or_train_prop(*common, C.byref(prop.q), _p(th, C.c_double), fb)
    return loss, rgb, flags, g


def train_upstream(om, poses, occ_bits, origin, direction, pose_id, up_rgb=None, up_alpha=None, nthreads=0):
    """Forward colour and alpha of the rays and, with up_rgb ([n, 3] dL/dC) and
    up_alpha ([n] dL/dalpha, optional), the backward of a loss built on them:
    (rgb [n, 3], alpha [n], flags [n], grads dict as train() or None)."""
    from . import _p
    sc = om.scene
    n = len(pose_id)
    arr = pose_array(poses) if isinstance(poses, (list, tuple)) else poses
    o = np.ascontiguousarray(origin, dtype=np.float32)
    d = np.ascontiguousarray(direction, dtype=np.float32)
    pid = np.ascontiguousarray(pose_id, dtype=np.int32)
    occ = np.ascontiguousarray(occ_bits, dtype=np.uint32)
    ur = None if up_rgb is None else np.ascontiguousarray(up_rgb, dtype=np.float64).reshape(n, 3)
    ua = None if up_alpha is None else np.ascontiguousarray(up_alpha, dtype=np.float64).reshape(n)
    rgb, alpha = np.zeros((n, 3)), np.zeros(n)
    flags = np.zeros(n, dtype=np.int32)
    g = None
    if ur is not None:
        g = dict(table=np.zeros((sc.n_table_entries(), sc.n_features)), mlp=np.zeros(mlp_size(sc)),
                 skin=np.zeros(om.skin.shape), bones=np.zeros((len(arr), sc.n_bones, 12)))
    args = [g[k] if g else None for k in ("table", "mlp", "skin", "bones")]
    om.L.or_train_upstream(C.byref(om.m), arr, len(arr), _p(occ, C.c_uint32), n, _p(o, C.c_float), _p(d, C.c_float),
                           _p(pid, C.c_int32), _p(ur, C.c_double), _p(ua, C.c_double), _p(rgb, C.c_double),
                           _p(alpha, C.c_double), _p(flags, C.c_int32), *[_p(a, C.c_double) for a in args], nthreads)
    return rgb, alpha, flags, g


def density_reg(om, poses, occ_bits, x, pose_id, weight, grads=None):
    """Occupancy-based density regulariser (Eq. 12) at normalised-space points:
    (loss, per-point flags).  grads: the dict train() returned, to which the
    regulariser's gradient is added in place (None: loss only)."""
    from . import _p
    arr = pose_array(poses) if isinstance(poses, (list, tuple)) else poses
    xs = np.ascontiguousarray(x, dtype=np.float32)
    pid = np.ascontiguousarray(pose_id, dtype=np.int32)
    occ = np.ascontiguousarray(occ_bits, dtype=np.uint32)
    flags = np.zeros(len(pid), dtype=np.int32)
    args = [None] * 4 if grads is None else [grads[k] for k in ("table", "mlp", "skin", "bones")]
    for a in args:
        assert a is None or (a.dtype == np.float64 and a.flags.c_contiguous)
    loss = om.L.or_density_reg(C.byref(om.m), arr, len(arr), _p(occ, C.c_uint32), len(pid), _p(xs, C.c_float),
                               _p(pid, C.c_int32), float(weight), _p(flags, C.c_int32),
                               *[_p(a, C.c_double) for a in args])
    return loss, flags
