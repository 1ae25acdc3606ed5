"""Thin Python binding of libia.so, the sm_103a articulated radiance-field render path.

Argument marshalling only: every step of the path runs in the CUDA library
(include/ia.h documents each call).  PyTorch provides device memory and streams.
The binding refuses to work without the compiled library: there is no CPU or
PyTorch fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libia.so")

IA_OK, IA_ERR_ARG, IA_ERR_STATE, IA_ERR_CUDA, IA_ERR_OOM, IA_ERR_LIMIT = range(6)
IA_FP32, IA_FP16, IA_BF16 = 0, 1, 2
IA_OCC_POSE, IA_OCC_UNION = 0, 1
IA_SEARCH_ALL_BONES, IA_SEARCH_PROPOSAL = 0, 1
IA_LOSS_L2, IA_LOSS_HUBER = 0, 1
IA_RENDER_FUSED, IA_RENDER_WAVEFRONT = 0, 1
MAX_LEVELS = 16


class IAError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"ia status {status}: {msg}")
        self.status = status


class Config(C.Structure):
    _fields_ = [("n_levels", C.c_int), ("n_features", C.c_int), ("log2_table", C.c_int),
                ("level_res", C.c_int * MAX_LEVELS), ("mlp_width", C.c_int), ("max_samples", C.c_int),
                ("broyden_max_iter", C.c_int), ("broyden_tol", C.c_float), ("occ_res", C.c_int),
                ("occ_tau", C.c_float), ("occ_dilate", C.c_int), ("early_stop_T", C.c_float),
                ("precision", C.c_int)]


class Camera(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int), ("height", C.c_int), ("c2w", C.c_float * 12)]


class RenderStats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("rays", "hit_rays", "marched_slots", "occupied_samples", "starts",
                                         "broyden_iters", "converged", "roots", "early_stopped", "proposed",
                                         "fallbacks", "culled", "grid_gathers",
                                         "rooted_samples", "point_culled")]


    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class ProposalConfig(C.Structure):
    _fields_ = [("n_levels", C.c_int), ("log2_table", C.c_int), ("level_res", C.c_int * MAX_LEVELS),
                ("top_k", C.c_int), ("offset_weight", C.c_float)]


class Batch(C.Structure):
    _fields_ = [("n_rays", C.c_int), ("origin", C.c_void_p), ("direction", C.c_void_p), ("pose", C.c_void_p),
                ("target", C.c_void_p), ("n_reg", C.c_int), ("reg_x", C.c_void_p), ("reg_pose", C.c_void_p),
                ("reg_weight", C.c_float), ("alpha_target", C.c_void_p)]


class Loss(C.Structure):
    _fields_ = [("rgb_loss", C.c_int), ("huber_delta", C.c_float), ("w_rgb", C.c_float), ("w_alpha", C.c_float),
                ("w_hard", C.c_float)]


class KernelTime(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_int64), ("total_ms", C.c_double), ("max_ms", C.c_double)]


class Grads(C.Structure):
    _fields_ = [("table", C.c_void_p), ("mlp", C.c_void_p), ("skin", C.c_void_p), ("bones", C.c_void_p)]


_lib = None


def lib():
    """Load libia.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                              "(nvcc -gencode arch=compute_103a,code=sm_103a)")
        L = C.CDLL(LIB_PATH)
        P, I, V = C.c_void_p, C.c_int, C.c_void_p
        sigs = {
            "ia_create": [C.POINTER(Config), C.POINTER(C.c_void_p)],
            "ia_set_skeleton": [P, I, P, P, P, I, P, P, P, P],
            "ia_param_sizes": [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
            "ia_set_params": [P, P, P, V],
            "ia_get_params": [P, P, P, V],
            "ia_set_pose": [P, I, P, P, V],
            "ia_get_transforms": [P, I, P, P, P, V],
            "ia_update_occupancy": [P, I, I, P, P, C.POINTER(RenderStats), V],
            "ia_occupancy_from_density": [P, P, P, V],
            "ia_set_occupancy": [P, P, V],
            "ia_query_posed": [P, I, I, P, P, P, P, P, V],
            "ia_query_canonical": [P, I, P, P, P, V],
            "ia_render": [P, I, C.POINTER(Camera), P, P, C.POINTER(RenderStats), V],
            "ia_march_mask": [P, I, C.POINTER(Camera), P, V],
            "ia_train_step": [P, C.POINTER(Batch), I, P, P, C.POINTER(Grads), V],
            "ia_train_forward": [P, C.POINTER(Batch), I, P, P, P, P, V],
            "ia_train_backward": [P, P, P, C.POINTER(Grads), V],
            "ia_update_occupancy_static": [P, I, P, V],
            "ia_update_occupancy_ema": [P, I, P, C.c_float, P, P, C.POINTER(RenderStats), V],
            "ia_loss_scale": [P, C.POINTER(C.c_float), C.POINTER(C.c_int32), V],
            "ia_set_wait_limit": [P, C.c_int64],
            "ia_set_fault_injection": [P, I],
            "ia_train_stats": [P, C.POINTER(RenderStats), V],
            "ia_grad_sizes": [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
            "ia_set_loss": [P, C.POINTER(Loss)],
            "ia_gather_probe": [P, C.c_int64, I, I, I, P, V],
            "ia_atomic_probe": [P, C.c_int64, I, I, I, V],
            "ia_adam_step": [P, P, P, P, C.c_float, C.c_float, C.c_float, C.c_float, V],
            "ia_proposal_init": [P, C.POINTER(ProposalConfig)],
            "ia_proposal_param_sizes": [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
            "ia_proposal_set_params": [P, P, P, V],
            "ia_proposal_get_params": [P, P, P, V],
            "ia_proposal_pairs": [P, I, I, P, P, P, V],
            "ia_proposal_grad": [P, I, P, P, P, P, P, P, P, V],
            "ia_proposal_train": [P, I, P, P, P, P, I, I, C.c_float, P, V],
            "ia_set_search": [P, I],
            "ia_set_occupancy_culling": [P, I],
            "ia_set_render_path": [P, I],
            "ia_profile_begin": [],
            "ia_profile_end": [C.POINTER(KernelTime), I, C.POINTER(C.c_int)],
        }
        for name, args in sigs.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.ia_destroy.argtypes = [C.c_void_p]
        L.ia_destroy.restype = None
        L.ia_last_error.argtypes = [C.c_void_p]
        L.ia_last_error.restype = C.c_char_p
        L.ia_version.restype = C.c_char_p
        L.ia_profile_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(st, ctx):
    if st != IA_OK:
        msg = lib().ia_last_error(ctx)
        raise IAError(st, msg.decode() if msg else "")


def _ptr(t):
    """Device or host address of a tensor / ndarray (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data
    assert t.is_contiguous(), "tensors passed to libia must be contiguous"
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def make_config(*, n_levels, log2_table, level_res, max_samples, broyden_max_iter=10, broyden_tol=1e-5,
                occ_res=64, occ_tau=0.01, occ_dilate=1, early_stop_T=1e-4, precision=IA_FP32, n_features=2,
                mlp_width=64):
    cfg = Config()
    cfg.n_levels, cfg.n_features, cfg.log2_table = n_levels, n_features, log2_table
    for i, r in enumerate(level_res):
        cfg.level_res[i] = int(r)
    cfg.mlp_width, cfg.max_samples = mlp_width, max_samples
    cfg.broyden_max_iter, cfg.broyden_tol = broyden_max_iter, broyden_tol
    cfg.occ_res, cfg.occ_tau, cfg.occ_dilate = occ_res, occ_tau, occ_dilate
    cfg.early_stop_T, cfg.precision = early_stop_T, precision
    return cfg


def make_camera(fx, fy, cx, cy, width, height, c2w):
    cam = Camera()
    cam.fx, cam.fy, cam.cx, cam.cy = float(fx), float(fy), float(cx), float(cy)
    cam.width, cam.height = int(width), int(height)
    for i, v in enumerate(np.asarray(c2w, dtype=np.float32).reshape(-1)):
        cam.c2w[i] = float(v)
    return cam


# --------------------------------------------------------------- C ABI names

def ia_create(cfg: Config) -> C.c_void_p:
    ctx = C.c_void_p()
    st = lib().ia_create(C.byref(cfg), C.byref(ctx))
    _check(st, None)
    return ctx


def ia_destroy(ctx):
    lib().ia_destroy(ctx)


def ia_last_error(ctx):
    return lib().ia_last_error(ctx).decode()


def ia_version():
    return lib().ia_version().decode()


def ia_set_skeleton(ctx, parents, rest_joints, skin_grid, canon_min, canon_max, norm_min, norm_max):
    parents = np.ascontiguousarray(parents, dtype=np.int32)
    rest = np.ascontiguousarray(rest_joints, dtype=np.float64)
    skin = skin_grid if not isinstance(skin_grid, np.ndarray) else np.ascontiguousarray(skin_grid, np.float32)
    boxes = [np.ascontiguousarray(b, dtype=np.float32) for b in (canon_min, canon_max, norm_min, norm_max)]
    res = int(skin.shape[0])
    _check(lib().ia_set_skeleton(ctx, len(parents), _ptr(parents), _ptr(rest), _ptr(skin), res,
                                 *[_ptr(b) for b in boxes]), ctx)


def ia_param_sizes(ctx):
    a, b = C.c_int64(), C.c_int64()
    _check(lib().ia_param_sizes(ctx, C.byref(a), C.byref(b)), ctx)
    return a.value, b.value


def ia_set_params(ctx, table, mlp, stream=None):
    _check(lib().ia_set_params(ctx, _ptr(table), _ptr(mlp), _stream(stream)), ctx)


def ia_get_params(ctx, table, mlp, stream=None):
    _check(lib().ia_get_params(ctx, _ptr(table), _ptr(mlp), _stream(stream)), ctx)


def ia_set_pose(ctx, axis_angle, root_trans, stream=None):
    th = np.ascontiguousarray(axis_angle, dtype=np.float64)
    tr = np.ascontiguousarray(root_trans, dtype=np.float64)
    n = th.shape[0] if th.ndim == 3 else 1
    _check(lib().ia_set_pose(ctx, n, _ptr(th), _ptr(tr), _stream(stream)), ctx)


def ia_get_transforms(ctx, pose, N=None, Ninv=None, B0inv=None, stream=None):
    _check(lib().ia_get_transforms(ctx, pose, _ptr(N), _ptr(Ninv), _ptr(B0inv), _stream(stream)), ctx)


def ia_update_occupancy(ctx, pose, mode=IA_OCC_POSE, sigma_out=None, bits_out=None, stats=False, stream=None):
    s = RenderStats() if stats else None
    _check(lib().ia_update_occupancy(ctx, pose, mode, _ptr(sigma_out), _ptr(bits_out),
                                     C.byref(s) if s is not None else None, _stream(stream)), ctx)
    return s.as_dict() if s is not None else None


def ia_occupancy_from_density(ctx, sigma, bits_out=None, stream=None):
    _check(lib().ia_occupancy_from_density(ctx, _ptr(sigma), _ptr(bits_out), _stream(stream)), ctx)


def ia_set_occupancy(ctx, bits, stream=None):
    _check(lib().ia_set_occupancy(ctx, _ptr(bits), _stream(stream)), ctx)


def ia_query_posed(ctx, pose, x, sigma=None, rgb=None, x_canon=None, start=None, stream=None):
    n = int(x.shape[0])
    _check(lib().ia_query_posed(ctx, pose, n, _ptr(x), _ptr(sigma), _ptr(rgb), _ptr(x_canon), _ptr(start),
                                _stream(stream)), ctx)


def ia_query_canonical(ctx, x, sigma, rgb, stream=None):
    _check(lib().ia_query_canonical(ctx, int(x.shape[0]), _ptr(x), _ptr(sigma), _ptr(rgb), _stream(stream)), ctx)


def ia_render(ctx, pose, cam: Camera, rgb, alpha, stats=False, stream=None):
    s = RenderStats() if stats else None
    _check(lib().ia_render(ctx, pose, C.byref(cam), _ptr(rgb), _ptr(alpha), C.byref(s) if s is not None else None,
                           _stream(stream)), ctx)
    return s.as_dict() if s is not None else None


def ia_set_render_path(ctx, path):
    """IA_RENDER_WAVEFRONT (default: kernels over arrays) or IA_RENDER_FUSED (one persistent kernel)."""
    _check(lib().ia_set_render_path(ctx, int(path)), ctx)


def ia_march_mask(ctx, pose, cam: Camera, slot_mask, stream=None):
    _check(lib().ia_march_mask(ctx, pose, C.byref(cam), _ptr(slot_mask), _stream(stream)), ctx)


def ia_train_step(ctx, origin, direction, pose, target, loss, grads, occ_grid=IA_OCC_UNION, rgb_out=None,
                  stream=None, reg_x=None, reg_pose=None, reg_weight=0.0, alpha_target=None):
    """grads: dict of device tensors table, mlp, skin, bones (overwritten); loss: device scalar (added to).
    reg_x [n][3] / reg_pose [n]: points of the density regulariser (optional)."""
    b = Batch()
    b.n_rays = int(pose.shape[0])
    b.origin, b.direction, b.pose, b.target = _ptr(origin), _ptr(direction), _ptr(pose), _ptr(target)
    b.alpha_target = _ptr(alpha_target)
    if reg_x is not None:
        b.n_reg = int(reg_pose.shape[0])
        b.reg_x, b.reg_pose, b.reg_weight = _ptr(reg_x), _ptr(reg_pose), float(reg_weight)
    g = Grads()
    g.table, g.mlp, g.skin, g.bones = (_ptr(grads[k]) for k in ("table", "mlp", "skin", "bones"))
    _check(lib().ia_train_step(ctx, C.byref(b), occ_grid, _ptr(loss), _ptr(rgb_out), C.byref(g),
                               _stream(stream)), ctx)


def ia_train_forward(ctx, origin, direction, pose, rgb_out, alpha_out=None, table=None, mlp=None,
                     occ_grid=IA_OCC_UNION, stream=None):
    """Forward half of the training step: rgb_out [n][3] (and alpha_out [n]) of the batch's rays.
    table / mlp: the field's parameters to use (device fp32; None = the context's own)."""
    b = Batch()
    b.n_rays = int(pose.shape[0])
    b.origin, b.direction, b.pose = _ptr(origin), _ptr(direction), _ptr(pose)
    _check(lib().ia_train_forward(ctx, C.byref(b), occ_grid, _ptr(table), _ptr(mlp), _ptr(rgb_out), _ptr(alpha_out),
                                  _stream(stream)), ctx)


def ia_train_backward(ctx, grad_rgb, grads, grad_alpha=None, stream=None):
    """Backward half: gradients of the last forward from dL/drgb [n][3] (and dL/dalpha [n]) into grads."""
    g = Grads()
    g.table, g.mlp, g.skin, g.bones = (_ptr(grads[k]) for k in ("table", "mlp", "skin", "bones"))
    _check(lib().ia_train_backward(ctx, _ptr(grad_rgb), _ptr(grad_alpha), C.byref(g), _stream(stream)), ctx)


def ia_gather_probe(table, n_records, iters, blocks, sink, stream=None, record_bytes=48):
    """Random record gathers of record_bytes (48, 16, 8 or 4) bytes (a measurement helper)."""
    _check(lib().ia_gather_probe(_ptr(table), int(n_records), int(record_bytes), int(iters), int(blocks), _ptr(sink),
                                 _stream(stream)), None)


def ia_atomic_probe(table, n_records, iters, blocks, stream=None, record_bytes=8):
    """Random vector atomicAdds of record_bytes (8 or 16) bytes (a measurement helper)."""
    _check(lib().ia_atomic_probe(_ptr(table), int(n_records), int(record_bytes), int(iters), int(blocks),
                                 _stream(stream)), None)


def ia_profile_begin():
    """Open a launch profile on this thread (per-kernel CUDA-event times of every library launch)."""
    st = lib().ia_profile_begin()
    if st != IA_OK:
        raise IAError(st, lib().ia_profile_error().decode())


def ia_profile_end(max_kernels=64):
    """Close the profile: {kernel name: (launches, total ms, max ms)} in order of first launch."""
    out = (KernelTime * max_kernels)()
    n = C.c_int()
    st = lib().ia_profile_end(out, max_kernels, C.byref(n))
    if st != IA_OK:
        raise IAError(st, lib().ia_profile_error().decode())
    return {out[i].name.decode(): (int(out[i].launches), float(out[i].total_ms), float(out[i].max_ms))
            for i in range(min(n.value, max_kernels))}


def ia_set_loss(ctx, rgb_loss=IA_LOSS_L2, huber_delta=0.0, w_rgb=1.0, w_alpha=0.0, w_hard=0.0):
    """Loss of the training step (Sec. 3.4, Eq. 9-11)."""
    l = Loss()
    l.rgb_loss, l.huber_delta, l.w_rgb, l.w_alpha, l.w_hard = rgb_loss, huber_delta, w_rgb, w_alpha, w_hard
    _check(lib().ia_set_loss(ctx, C.byref(l)), ctx)


def ia_adam_step(ctx, g_table, g_mlp, lr, beta1=0.9, beta2=0.99, eps=1e-15, g_skin=None, stream=None):
    """Adam on the context's hash table and MLP (and the skinning grid with g_skin)."""
    _check(lib().ia_adam_step(ctx, _ptr(g_table), _ptr(g_mlp), _ptr(g_skin), float(lr), float(beta1), float(beta2),
                              float(eps), _stream(stream)), ctx)


def ia_grad_sizes(ctx):
    """(skinning-grid floats, bone-transform floats) of the training step's gradients."""
    a, b = C.c_int64(), C.c_int64()
    _check(lib().ia_grad_sizes(ctx, C.byref(a), C.byref(b)), ctx)
    return a.value, b.value


def ia_train_stats(ctx, stream=None):
    """Counters of the last training step (dict, same keys as the render counters)."""
    st = RenderStats()
    _check(lib().ia_train_stats(ctx, C.byref(st), _stream(stream)), ctx)
    return st.as_dict()


def ia_set_wait_limit(ctx, limit_ns):
    """Bound (ns) on each wait of the tensor-core weight-gradient pipeline; 0 = default (200 ms)."""
    _check(lib().ia_set_wait_limit(ctx, int(limit_ns)), ctx)


IA_INJECT_WITHHOLD_COPY = 1


def ia_set_fault_injection(ctx, flags):
    """Test-only failure injection (IA_INJECT_WITHHOLD_COPY: the weight-gradient pipeline withholds a copy)."""
    _check(lib().ia_set_fault_injection(ctx, int(flags)), ctx)


def ia_loss_scale(ctx, stream=None):
    """(loss scale S after the last training step, whether that step was skipped: overflow or
    a weight-gradient pipeline that gave up, the latter also raising IAError(IA_ERR_CUDA))."""
    sc, sk = C.c_float(), C.c_int32()
    _check(lib().ia_loss_scale(ctx, C.byref(sc), C.byref(sk), _stream(stream)), ctx)
    return sc.value, bool(sk.value)


def ia_update_occupancy_ema(ctx, pose, jitter=None, decay=0.95, density_out=None, bits_out=None, stats=False,
                            stream=None):
    """Training-mode occupancy update (running density max(decay d, sigma), training grid replaced)."""
    st = RenderStats() if stats else None
    _check(lib().ia_update_occupancy_ema(ctx, pose, _ptr(jitter), float(decay), _ptr(density_out), _ptr(bits_out),
                                         C.byref(st) if st is not None else None, _stream(stream)), ctx)
    return st.as_dict() if st is not None else None


def ia_update_occupancy_static(ctx, pose, bits_out=None, stream=None):
    """Occupancy refresh that allocates nothing (fixed 64^3-cell scratch in the library)."""
    _check(lib().ia_update_occupancy_static(ctx, pose, _ptr(bits_out), _stream(stream)), ctx)


def make_proposal_config(n_levels, log2_table, level_res, top_k=2, offset_weight=100.0):
    q = ProposalConfig()
    q.n_levels, q.log2_table, q.top_k, q.offset_weight = n_levels, log2_table, top_k, offset_weight
    for i, r in enumerate(level_res):
        q.level_res[i] = int(r)
    return q


def ia_proposal_init(ctx, cfg: ProposalConfig):
    _check(lib().ia_proposal_init(ctx, C.byref(cfg)), ctx)


def ia_proposal_param_sizes(ctx):
    a, b = C.c_int64(), C.c_int64()
    _check(lib().ia_proposal_param_sizes(ctx, C.byref(a), C.byref(b)), ctx)
    return a.value, b.value


def ia_proposal_set_params(ctx, table, mlp, stream=None):
    _check(lib().ia_proposal_set_params(ctx, _ptr(table), _ptr(mlp), _stream(stream)), ctx)


def ia_proposal_get_params(ctx, table, mlp, stream=None):
    _check(lib().ia_proposal_get_params(ctx, _ptr(table), _ptr(mlp), _stream(stream)), ctx)


def ia_proposal_pairs(ctx, pose, x, label, offset, stream=None):
    _check(lib().ia_proposal_pairs(ctx, pose, int(x.shape[0]), _ptr(x), _ptr(label), _ptr(offset),
                                   _stream(stream)), ctx)


def ia_proposal_grad(ctx, x, pose, label, target, loss, g_table, g_mlp, stream=None):
    _check(lib().ia_proposal_grad(ctx, int(x.shape[0]), _ptr(x), _ptr(pose), _ptr(label), _ptr(target), _ptr(loss),
                                  _ptr(g_table), _ptr(g_mlp), _stream(stream)), ctx)


def ia_proposal_train(ctx, x, pose, label, target, steps, batch, lr, loss_out=None, stream=None):
    _check(lib().ia_proposal_train(ctx, int(x.shape[0]), _ptr(x), _ptr(pose), _ptr(label), _ptr(target), int(steps),
                                   int(batch), float(lr), _ptr(loss_out), _stream(stream)), ctx)


def ia_set_search(ctx, mode):
    _check(lib().ia_set_search(ctx, mode), ctx)


def ia_set_occupancy_culling(ctx, on):
    _check(lib().ia_set_occupancy_culling(ctx, 1 if on else 0), ctx)
