"""FP64 CPU oracle for the articulated radiance-field render path (InstantAvatar,
arXiv 2212.10550).  TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg use this
package.  It shares no code with the CUDA library: the arithmetic lives in
``oracle.c`` (plain C, fp64, one sample at a time) and this module only marshals
numpy arrays into it through ctypes.  The shared object is compiled with gcc on
first use (or by the build step) with ``-ffp-contract=off`` so that the fp32
indexing functions are the exact rounded operation sequence they document.

Parity notes (readings the paper leaves open, shared with the library by
contract, not pinned by any value the paper prints — "parity unpinned"):
the multi-root aggregation (max-density root), the hash primes and level
rounding, the density activation exp(clamp(., -15, 15)), the occupancy
threshold tau and the dilation radius.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, f) for f in ("oracle.c", "oracle_grad.c", "oracle_prop.c")]
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
MAX_BONES = 32

FLAG_CONV, FLAG_BOX, FLAG_DUP, FLAG_TIE, FLAG_SING, FLAG_TERM, FLAG_PROP = 1, 2, 4, 8, 16, 32, 64


def build(force: bool = False) -> str:
    """Compile liboracle.so next to the sources if missing or stale."""
    srcs = [s for s in _SRC if os.path.exists(s)]
    newest = max(os.path.getmtime(p) for p in srcs + [_HDR])
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp] + srcs + ["-lm"]
    try:
        subprocess.run(cmd, check=True, capture_output=True, text=True)
        os.replace(tmp, _LIB)
    except subprocess.CalledProcessError as e:
        os.unlink(tmp)
        raise RuntimeError("oracle build failed:\n" + e.stderr) from e
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


PD = C.POINTER(C.c_double)
PF = C.POINTER(C.c_float)
PI32 = C.POINTER(C.c_int32)
PU32 = C.POINTER(C.c_uint32)
PI64 = C.POINTER(C.c_int64)


class Model(C.Structure):
    _fields_ = [
        ("nb", C.c_int), ("parent", PI32), ("rest", PD),
        ("rw", C.c_int), ("skin", PD),
        ("cmin", C.c_double * 3), ("cmax", C.c_double * 3),
        ("nmin", C.c_float * 3), ("nmax", C.c_float * 3),
        ("occ_res", C.c_int), ("L", C.c_int), ("F", C.c_int), ("res", PI32), ("log2_T", C.c_int),
        ("table", PD), ("n_in", C.c_int), ("width", C.c_int),
        ("W1", PD), ("b1", PD), ("W2", PD), ("b2", PD), ("W3", PD), ("b3", PD),
        ("max_iter", C.c_int), ("tol", C.c_double), ("n_slots", C.c_int),
        ("early_T", C.c_double), ("tau", C.c_double), ("dilate", C.c_int),
        ("quantize_fp32", C.c_int), ("h0_analytic", C.c_int),
    ]


class Pose(C.Structure):
    _fields_ = [("B", (C.c_double * 12) * MAX_BONES), ("N", (C.c_double * 12) * MAX_BONES),
                ("Ninv", (C.c_double * 12) * MAX_BONES), ("B0inv", C.c_float * 12)]


class Camera(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int), ("height", C.c_int), ("c2w", C.c_float * 12)]


class Sample(C.Structure):
    _fields_ = [("sigma", C.c_double), ("rgb", C.c_double * 3), ("xstar", C.c_double * 3),
                ("start", C.c_int), ("n_conv", C.c_int), ("n_unique", C.c_int),
                ("flags", C.c_int), ("iters", C.c_int)]


def _declare(L):
    PM, PP, PC = C.POINTER(Model), C.POINTER(Pose), C.POINTER(Camera)
    sig = {
        "or_pose_chain": (None, [PM, PD, PD, PP]),
        "or_cos_sin": (None, [C.c_double, PD, PD]),
        "or_skin": (None, [PM, PD, PD, PD]),
        "or_lbs": (None, [PM, PP, PD, PD, PD]),
        "or_broyden": (C.c_int, [PM, PP, PD, PD, PD, PI32, PD, PI32]),
        "or_polish": (C.c_double, [PM, PP, PD, PD]),
        "or_roots": (C.c_int, [PM, PP, PD, PD, PI32, PI32]),
        "or_encode": (None, [PM, PD, PD]),
        "or_mlp": (None, [PM, PD, PD]),
        "or_field": (None, [PM, PD, PD, PD]),
        "or_posed_field": (None, [PM, PP, PD, C.POINTER(Sample)]),
        "or_ray": (C.c_int, [PM, PP, PC, C.c_int, C.c_int, PF, PF, PF, PF]),
        "or_cell": (C.c_int, [PM, PF]),
        "or_cell_center": (None, [PM, C.c_int, PF]),
        "or_render": (None, [PM, PP, PC, PU32, PD, PD, PI32, PI32, PI64, C.c_int]),
        "or_render_pixels": (None, [PM, PP, PC, PU32, C.c_int, PI32, PD, PD, PI32, PI32, C.c_int]),
        "or_occupancy": (None, [PM, PP, PD, PU32, C.c_int]),
        "or_occupancy_ema": (None, [PM, PP, PF, C.c_double, PD, PU32, C.c_int]),
        "or_march_mask": (None, [PM, PP, PC, PU32, PU32]),
        "or_occupancy_cells": (None, [PM, PP, C.c_int, PI32, PD, C.c_int]),
        "or_occ_bits": (None, [C.c_int, C.c_int, C.c_double, PD, PU32]),
        "or_occ_bits_f32": (None, [C.c_int, C.c_int, C.c_float, PF, PU32]),
        "or_bruteforce_roots": (C.c_int, [PM, PP, PD, C.c_int, C.c_double, PD, C.c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    if hasattr(L, "or_train"):
        _declare_grad(L)
    if hasattr(L, "or_prop_forward"):
        from . import prop as _pp
        _pp.declare(L)


def _declare_grad(L):
    from . import grad as _g  # noqa: F401  (signatures live with the wrapper)
    _g.declare(L)


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleModel:
    """Keeps the fp64 arrays alive and exposes the oracle entry points."""

    def __init__(self, scene, table, mlp, *, early_T: float = 0.0, quantize_fp32: bool = True,
                 skin=None, n_slots=None, tol=None, max_iter=None, h0_analytic=False):
        L_ = lib()
        self.scene = scene
        self.parent = np.ascontiguousarray(scene.parents, dtype=np.int32)
        self.rest = _f64(scene.rest_joints)
        self.skin = _f64(scene.skin_grid if skin is None else skin)
        self.res = np.ascontiguousarray(scene.level_res, dtype=np.int32)
        self.table = _f64(table)
        self.mlp = {k: _f64(v) for k, v in mlp.items()}
        m = Model()
        m.nb = scene.n_bones
        m.parent = _p(self.parent, C.c_int32)
        m.rest = _p(self.rest, C.c_double)
        m.rw = int(self.skin.shape[0])
        m.skin = _p(self.skin, C.c_double)
        for a in range(3):
            m.cmin[a] = float(scene.canon_min[a])
            m.cmax[a] = float(scene.canon_max[a])
            m.nmin[a] = float(scene.norm_min[a])
            m.nmax[a] = float(scene.norm_max[a])
        m.occ_res = scene.occ_res
        m.L, m.F = scene.n_levels, scene.n_features
        m.res = _p(self.res, C.c_int32)
        m.log2_T = scene.log2_table
        m.table = _p(self.table, C.c_double)
        m.n_in = scene.mlp_in()
        m.width = scene.mlp_width
        for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
            setattr(m, k, _p(self.mlp[k], C.c_double))
        m.max_iter = scene.broyden_max_iter if max_iter is None else max_iter
        m.tol = scene.broyden_tol if tol is None else tol
        m.n_slots = scene.max_samples if n_slots is None else n_slots
        m.early_T = early_T
        m.tau = scene.occ_tau
        m.dilate = scene.occ_dilate
        m.quantize_fp32 = 1 if quantize_fp32 else 0
        m.h0_analytic = 1 if h0_analytic else 0
        self.m = m
        self.L = L_

    # ---- pose ----
    def pose(self, theta, trans):
        p = Pose()
        th, tr = _f64(theta), _f64(trans)
        self.L.or_pose_chain(C.byref(self.m), _p(th, C.c_double), _p(tr, C.c_double), C.byref(p))
        return p

    def transforms(self, p):
        nb = self.scene.n_bones
        N = np.array([[p.N[k][i] for i in range(12)] for k in range(nb)])
        B = np.array([[p.B[k][i] for i in range(12)] for k in range(nb)])
        Ninv = np.array([[p.Ninv[k][i] for i in range(12)] for k in range(nb)])
        B0inv = np.array([p.B0inv[i] for i in range(12)], dtype=np.float32)
        return dict(B=B.reshape(nb, 3, 4), N=N.reshape(nb, 3, 4), Ninv=Ninv.reshape(nb, 3, 4),
                    B0inv=B0inv.reshape(3, 4))

    # ---- skinning / root finding ----
    def skin_weights(self, x, grad=False):
        x = _f64(x)
        w = np.zeros(self.scene.n_bones)
        dw = np.zeros((self.scene.n_bones, 3)) if grad else None
        self.L.or_skin(C.byref(self.m), _p(x, C.c_double), _p(w, C.c_double), _p(dw, C.c_double))
        return (w, dw) if grad else w

    def lbs(self, p, x, jac=False):
        x = _f64(x)
        y = np.zeros(3)
        J = np.zeros(9) if jac else None
        self.L.or_lbs(C.byref(self.m), C.byref(p), _p(x, C.c_double), _p(y, C.c_double),
                      _p(J, C.c_double))
        return (y, J.reshape(3, 3)) if jac else y

    def broyden(self, p, xn, x0):
        xn, x0 = _f64(xn), _f64(x0)
        x = np.zeros(3)
        it = np.zeros(1, dtype=np.int32)
        rn = np.zeros(1)
        fl = np.zeros(1, dtype=np.int32)
        ok = self.L.or_broyden(C.byref(self.m), C.byref(p), _p(xn, C.c_double), _p(x0, C.c_double),
                               _p(x, C.c_double), _p(it, C.c_int32), _p(rn, C.c_double),
                               _p(fl, C.c_int32))
        return bool(ok), x, int(it[0]), float(rn[0])

    def polish(self, p, xn, x):
        xn, x = _f64(xn), _f64(x).copy()
        r = self.L.or_polish(C.byref(self.m), C.byref(p), _p(xn, C.c_double), _p(x, C.c_double))
        return x, r

    def roots(self, p, xn):
        xn = _f64(xn)
        roots = np.zeros((MAX_BONES, 3))
        starts = np.zeros(MAX_BONES, dtype=np.int32)
        fl = np.zeros(1, dtype=np.int32)
        n = self.L.or_roots(C.byref(self.m), C.byref(p), _p(xn, C.c_double), _p(roots, C.c_double),
                            _p(starts, C.c_int32), _p(fl, C.c_int32))
        return roots[:n].copy(), starts[:n].copy(), int(fl[0])

    def bruteforce_roots(self, p, xn, n=64, seed_thresh=0.05, max_roots=64):
        xn = _f64(xn)
        roots = np.zeros((max_roots, 3))
        k = self.L.or_bruteforce_roots(C.byref(self.m), C.byref(p), _p(xn, C.c_double), n,
                                       seed_thresh, _p(roots, C.c_double), max_roots)
        return roots[:k].copy()

    # ---- canonical field ----
    def encode(self, x):
        x = _f64(x)
        f = np.zeros(self.scene.mlp_in())
        self.L.or_encode(C.byref(self.m), _p(x, C.c_double), _p(f, C.c_double))
        return f

    def mlp_out(self, feat):
        feat = _f64(feat)
        o = np.zeros(4)
        self.L.or_mlp(C.byref(self.m), _p(feat, C.c_double), _p(o, C.c_double))
        return o

    def field(self, x):
        x = _f64(x)
        s = np.zeros(1)
        rgb = np.zeros(3)
        self.L.or_field(C.byref(self.m), _p(x, C.c_double), _p(s, C.c_double), _p(rgb, C.c_double))
        return float(s[0]), rgb

    def posed_field(self, p, xn):
        xn = _f64(xn)
        s = Sample()
        self.L.or_posed_field(C.byref(self.m), C.byref(p), _p(xn, C.c_double), C.byref(s))
        return dict(sigma=s.sigma, rgb=np.array(s.rgb[:]), xstar=np.array(s.xstar[:]),
                    start=s.start, n_conv=s.n_conv, n_unique=s.n_unique, flags=s.flags,
                    iters=s.iters)

    def posed_field_many(self, p, pts):
        out = [self.posed_field(p, x) for x in np.asarray(pts, dtype=np.float64)]
        return dict(sigma=np.array([o["sigma"] for o in out]),
                    rgb=np.array([o["rgb"] for o in out]),
                    xstar=np.array([o["xstar"] for o in out]),
                    start=np.array([o["start"] for o in out]),
                    n_unique=np.array([o["n_unique"] for o in out]),
                    flags=np.array([o["flags"] for o in out]))

    # ---- indexing / rendering ----
    @staticmethod
    def camera(cam):
        c = Camera()
        c.fx, c.fy, c.cx, c.cy = float(cam["fx"]), float(cam["fy"]), float(cam["cx"]), float(cam["cy"])
        c.width, c.height = int(cam["width"]), int(cam["height"])
        for i, v in enumerate(np.asarray(cam["c2w"], dtype=np.float32).reshape(-1)):
            c.c2w[i] = float(v)
        return c

    def ray(self, p, cam, u, v):
        o = np.zeros(3, dtype=np.float32)
        d = np.zeros(3, dtype=np.float32)
        tn = np.zeros(1, dtype=np.float32)
        tf = np.zeros(1, dtype=np.float32)
        c = self.camera(cam)
        hit = self.L.or_ray(C.byref(self.m), C.byref(p), C.byref(c), u, v, _p(o, C.c_float),
                            _p(d, C.c_float), _p(tn, C.c_float), _p(tf, C.c_float))
        return bool(hit), o, d, float(tn[0]), float(tf[0])

    def cell(self, x):
        x = np.ascontiguousarray(x, dtype=np.float32)
        return int(self.L.or_cell(C.byref(self.m), _p(x, C.c_float)))

    def cell_center(self, cell):
        x = np.zeros(3, dtype=np.float32)
        self.L.or_cell_center(C.byref(self.m), int(cell), _p(x, C.c_float))
        return x

    def render(self, p, cam, occ_bits, nthreads=0):
        W, H = int(cam["width"]), int(cam["height"])
        rgb = np.zeros((H * W, 3))
        alpha = np.zeros(H * W)
        flags = np.zeros(H * W, dtype=np.int32)
        nsamp = np.zeros(H * W, dtype=np.int32)
        iters = np.zeros(H * W, dtype=np.int64)
        occ = np.ascontiguousarray(occ_bits, dtype=np.uint32)
        c = self.camera(cam)
        self.L.or_render(C.byref(self.m), C.byref(p), C.byref(c), _p(occ, C.c_uint32),
                         _p(rgb, C.c_double), _p(alpha, C.c_double), _p(flags, C.c_int32),
                         _p(nsamp, C.c_int32), _p(iters, C.c_int64), nthreads)
        return dict(rgb=rgb, alpha=alpha, flags=flags, nsamp=nsamp, iters=iters)

    def render_pixels(self, p, cam, occ_bits, pix, nthreads=0):
        pix = np.ascontiguousarray(pix, dtype=np.int32)
        n = len(pix)
        rgb = np.zeros((n, 3))
        alpha = np.zeros(n)
        flags = np.zeros(n, dtype=np.int32)
        nsamp = np.zeros(n, dtype=np.int32)
        occ = np.ascontiguousarray(occ_bits, dtype=np.uint32)
        c = self.camera(cam)
        self.L.or_render_pixels(C.byref(self.m), C.byref(p), C.byref(c), _p(occ, C.c_uint32), n,
                                _p(pix, C.c_int32), _p(rgb, C.c_double), _p(alpha, C.c_double),
                                _p(flags, C.c_int32), _p(nsamp, C.c_int32), nthreads)
        return dict(rgb=rgb, alpha=alpha, flags=flags, nsamp=nsamp)

    def march_mask(self, p, cam, occ_bits):
        W, H = int(cam["width"]), int(cam["height"])
        words = (self.m.n_slots + 31) // 32
        mask = np.zeros((H * W, words), dtype=np.uint32)
        occ = np.ascontiguousarray(occ_bits, dtype=np.uint32)
        c = self.camera(cam)
        self.L.or_march_mask(C.byref(self.m), C.byref(p), C.byref(c), _p(occ, C.c_uint32),
                             _p(mask, C.c_uint32))
        return mask

    def occupancy_cells(self, p, cells, nthreads=0):
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        sigma = np.zeros(len(cells))
        self.L.or_occupancy_cells(C.byref(self.m), C.byref(p), len(cells), _p(cells, C.c_int32),
                                  _p(sigma, C.c_double), nthreads)
        return sigma

    def occupancy_ema(self, p, d, jitter=None, decay=0.95, nthreads=0):
        """Training-mode update: d <- max(decay d, sigma at the (jittered) cell
        points of pose p), in place; returns the bits of the updated d."""
        R = self.scene.occ_res
        assert d.dtype == np.float64 and d.shape == (R ** 3,) and d.flags.c_contiguous
        bits = np.zeros((R ** 3 + 31) // 32, dtype=np.uint32)
        jit = None if jitter is None else np.ascontiguousarray(jitter, dtype=np.float32).reshape(-1)
        self.L.or_occupancy_ema(C.byref(self.m), C.byref(p), _p(jit, C.c_float), float(decay), _p(d, C.c_double),
                                _p(bits, C.c_uint32), nthreads)
        return bits

    def occupancy(self, p, nthreads=0):
        R = self.scene.occ_res
        sigma = np.zeros(R ** 3)
        bits = np.zeros((R ** 3 + 31) // 32, dtype=np.uint32)
        self.L.or_occupancy(C.byref(self.m), C.byref(p), _p(sigma, C.c_double),
                            _p(bits, C.c_uint32), nthreads)
        return sigma, bits


def cos_sin(a):
    """(cos a, sin a) as the pose chain evaluates them (fixed-order power series)."""
    c, s = C.c_double(), C.c_double()
    lib().or_cos_sin(float(a), C.byref(c), C.byref(s))
    return c.value, s.value


def occ_bits(R, dilate, tau, sigma):
    """Threshold + dilation + packing of a density array (fp64 comparison)."""
    sigma = _f64(sigma).reshape(-1)
    bits = np.zeros((R ** 3 + 31) // 32, dtype=np.uint32)
    lib().or_occ_bits(R, dilate, float(tau), _p(sigma, C.c_double), _p(bits, C.c_uint32))
    return bits


def occ_bits_f32(R, dilate, tau, sigma):
    """Same, comparing fp32 densities against an fp32 threshold."""
    sigma = np.ascontiguousarray(sigma, dtype=np.float32).reshape(-1)
    bits = np.zeros((R ** 3 + 31) // 32, dtype=np.uint32)
    lib().or_occ_bits_f32(R, dilate, np.float32(tau), _p(sigma, C.c_float), _p(bits, C.c_uint32))
    return bits
