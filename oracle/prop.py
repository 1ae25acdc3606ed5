"""ctypes wrapper of the oracle's correspondence-proposal network
(oracle_prop.c).  TEST INFRASTRUCTURE ONLY."""
import ctypes as C

import numpy as np

NAMES = ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")


class Prop(C.Structure):
    _fields_ = [("L", C.c_int), ("log2_T", C.c_int), ("res", C.POINTER(C.c_int32)),
                ("table", C.POINTER(C.c_double)), ("n_in", C.c_int), ("width", C.c_int), ("n_out", C.c_int)] + \
               [(n, C.POINTER(C.c_double)) for n in NAMES] + [("top_k", C.c_int), ("offset_weight", C.c_double)]


def declare(L):
    from . import Camera, Model, Pose, Sample
    P = C.POINTER
    PM, PQ = P(Model), P(Prop)
    sig = {
        "or_prop_forward": (None, [PM, PQ, P(C.c_double), P(C.c_double), P(C.c_double)]),
        "or_prop_label": (C.c_int, [PM, P(Pose), P(C.c_double), P(C.c_double), P(C.c_double)]),
        "or_prop_mlp_count": (C.c_long, [PQ]),
        "or_prop_loss_grad": (C.c_double, [PM, PQ, C.c_int, P(C.c_float), P(C.c_int32), P(C.c_double),
                                           P(C.c_int32), P(C.c_double), P(C.c_double), P(C.c_double)]),
        "or_posed_field_prop": (None, [PM, P(Pose), PQ, P(C.c_double), P(C.c_double), P(Sample), P(C.c_int)]),
        "or_render_pixels_prop": (None, [PM, P(Pose), PQ, P(C.c_double), P(Camera), P(C.c_uint32), C.c_int,
                                         P(C.c_int32), P(C.c_double), P(C.c_double), P(C.c_int32), P(C.c_int32),
                                         P(C.c_int32), C.c_int]),
        "or_train_prop": (C.c_double, [PM, P(Pose), C.c_int, P(C.c_uint32), C.c_int, P(C.c_float), P(C.c_float),
                                       P(C.c_int32), P(C.c_double), P(C.c_double), P(C.c_int32), P(C.c_double),
                                       P(C.c_double), P(C.c_double), P(C.c_double), C.c_int, PQ, P(C.c_double),
                                       P(C.c_int32)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


class PropModel:
    """fp64 copies of the proposal parameters and the oracle entry points."""

    def __init__(self, om, cfg, table, mlp):
        from . import _f64, _p
        self.om = om
        self.cfg = cfg
        self.res = np.ascontiguousarray(cfg["level_res"], dtype=np.int32)
        self.table = _f64(table)
        self.mlp = {k: _f64(mlp[k]) for k in NAMES}
        q = Prop()
        q.L, q.log2_T = cfg["n_levels"], cfg["log2_table"]
        q.res = _p(self.res, C.c_int32)
        q.table = _p(self.table, C.c_double)
        nb = om.scene.n_bones
        q.n_in, q.width, q.n_out = 2 * cfg["n_levels"] + 3 * nb, 64, nb + 3
        for k in NAMES:
            setattr(q, k, _p(self.mlp[k], C.c_double))
        q.top_k, q.offset_weight = cfg["top_k"], cfg["offset_weight"]
        self.q = q

    def forward(self, xn, theta):
        from . import _f64, _p
        xn, th = _f64(xn), _f64(theta).reshape(-1)
        out = np.zeros(self.q.n_out)
        self.om.L.or_prop_forward(C.byref(self.om.m), C.byref(self.q), _p(xn, C.c_double), _p(th, C.c_double),
                                  _p(out, C.c_double))
        return out

    def label(self, pose, xs, xn):
        from . import _f64, _p
        off = np.zeros(3)
        k = self.om.L.or_prop_label(C.byref(self.om.m), C.byref(pose), _p(_f64(xs), C.c_double),
                                    _p(_f64(xn), C.c_double), _p(off, C.c_double))
        return k, off

    def loss_grad(self, x, pose_id, theta_all, label, target, grad=True):
        from . import _f64, _p
        x = np.ascontiguousarray(x, dtype=np.float32)
        pid = np.ascontiguousarray(pose_id, dtype=np.int32)
        lab = np.ascontiguousarray(label, dtype=np.int32)
        th, tg = _f64(theta_all).reshape(-1), _f64(target)
        gt = np.zeros_like(self.table) if grad else None
        gm = np.zeros(self.om.L.or_prop_mlp_count(C.byref(self.q))) if grad else None
        loss = self.om.L.or_prop_loss_grad(C.byref(self.om.m), C.byref(self.q), len(pid), _p(x, C.c_float),
                                           _p(pid, C.c_int32), _p(th, C.c_double), _p(lab, C.c_int32),
                                           _p(tg, C.c_double), _p(gt, C.c_double), _p(gm, C.c_double))
        return loss, gt, gm

    def posed_field(self, pose, theta, xn):
        from . import Sample, _f64, _p
        s = Sample()
        fb = C.c_int(0)
        self.om.L.or_posed_field_prop(C.byref(self.om.m), C.byref(pose), C.byref(self.q),
                                      _p(_f64(theta).reshape(-1), C.c_double), _p(_f64(xn), C.c_double),
                                      C.byref(s), C.byref(fb))
        return dict(sigma=s.sigma, rgb=np.array(s.rgb[:]), xstar=np.array(s.xstar[:]), start=s.start,
                    n_unique=s.n_unique, flags=s.flags, iters=s.iters, fallback=fb.value)

    def render_pixels(self, pose, theta, cam, occ_bits, pix, nthreads=0):
        """Proposal-mode render of the listed pixels: rgb, alpha, flags, samples
        and fallbacks per ray (or_render_pixels_prop)."""
        from . import _f64, _p
        pix = np.ascontiguousarray(pix, dtype=np.int32)
        n = len(pix)
        rgb, alpha = np.zeros((n, 3)), np.zeros(n)
        flags, nsamp, fb = (np.zeros(n, dtype=np.int32) for _ in range(3))
        occ = np.ascontiguousarray(occ_bits, dtype=np.uint32)
        c = self.om.camera(cam)
        self.om.L.or_render_pixels_prop(C.byref(self.om.m), C.byref(pose), C.byref(self.q),
                                        _p(_f64(theta).reshape(-1), C.c_double), C.byref(c), _p(occ, C.c_uint32), n,
                                        _p(pix, C.c_int32), _p(rgb, C.c_double), _p(alpha, C.c_double),
                                        _p(flags, C.c_int32), _p(nsamp, C.c_int32), _p(fb, C.c_int32), nthreads)
        return dict(rgb=rgb, alpha=alpha, flags=flags, nsamp=nsamp, fallbacks=fb)
