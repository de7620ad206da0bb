"""FP64 CPU oracle for MFA-DVR: ctypes wrapper over ``mfa_oracle.c``.

TEST INFRASTRUCTURE ONLY.  The tests, the package smoke check and the
benchmark's CPU-baseline / reference leg are the only callers.  The CUDA
library and its Python binding never import this package, and this package
imports nothing from them.

The C file holds the arithmetic (B-spline model of Sec. 2.3, value and
gradient queries, the ray caster of Algorithm 1); this module only compiles it
with gcc and marshals arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mfa_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
# A prebuilt library to load instead (the mutation tests point this at copies
# of the oracle with planted mistakes, to show that the pins catch them).
_LIB_OVERRIDE = os.environ.get("MFADVR_ORACLE_LIB")
_lock = threading.Lock()
_lib = None


GCC_FLAGS = ["-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off"]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to its source (gcc, -O2, pthreads)."""
    if _LIB_OVERRIDE:
        return _LIB_OVERRIDE
    with _lock:
        stale = (not os.path.exists(_LIB_PATH)
                 or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
        if force or stale:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", *GCC_FLAGS, "-o", tmp, _SRC, "-lm", "-lpthread"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Model(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int32 * 3), ("n", ctypes.c_int32 * 3),
                ("ctrl", ctypes.c_void_p),
                ("box_min", ctypes.c_double * 3), ("box_max", ctypes.c_double * 3),
                ("knots", ctypes.c_void_p * 3), ("weights", ctypes.c_void_p)]


class Camera(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("eye", ctypes.c_double * 3),
                ("center", ctypes.c_double * 3), ("up", ctypes.c_double * 3),
                ("fovy_deg", ctypes.c_double), ("ortho_height", ctypes.c_double)]


class RenderParams(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("step", ctypes.c_double), ("max_opacity", ctypes.c_double),
                ("ref_step", ctypes.c_double), ("tf_rgba", ctypes.c_void_p),
                ("tf_size", ctypes.c_int32), ("tf_lo", ctypes.c_double),
                ("tf_hi", ctypes.c_double), ("shading", ctypes.c_int32),
                ("ka", ctypes.c_double), ("kd", ctypes.c_double),
                ("ks", ctypes.c_double), ("shininess", ctypes.c_double)]


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.POINTER
        L.orc_make_knots.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_double)]
        L.orc_find_span.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_double), ctypes.c_double]
        L.orc_basis_ders.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, P(ctypes.c_double),
                                     P(ctypes.c_double), P(ctypes.c_double)]
        L.orc_basis_ders.restype = None
        L.orc_basis_brute.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, P(ctypes.c_double), ctypes.c_int]
        L.orc_basis_brute.restype = ctypes.c_double
        L.orc_basis_brute_der.argtypes = L.orc_basis_brute.argtypes
        L.orc_basis_brute_der.restype = ctypes.c_double
        L.orc_basis_brute_dk.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         P(ctypes.c_double), ctypes.c_int]
        L.orc_basis_brute_dk.restype = ctypes.c_double
        L.orc_eval_points.argtypes = [P(Model), ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
        L.orc_eval_hessian.argtypes = [P(Model), ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
        L.orc_render.argtypes = [P(Model), P(Camera), P(RenderParams), ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        _lib = L
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def knots(n: int, p: int) -> np.ndarray:
    t = np.zeros(n + p + 1, dtype=np.float64)
    if lib().orc_make_knots(n, p, _dptr(t)) != 0:
        raise ValueError("bad knot sizes")
    return t


def _knot_vector(n, p, t):
    if t is None:
        return knots(n, p)
    t = np.ascontiguousarray(t, dtype=np.float64)
    if t.shape != (n + p + 1,):
        raise ValueError("a knot vector has n + p + 1 entries")
    return t


def find_span(n: int, p: int, u: float, t=None) -> int:
    t = _knot_vector(n, p, t)
    return lib().orc_find_span(n, p, _dptr(t), float(u))


def basis_ders(n: int, p: int, u: float, t=None):
    """(span, N[0..p], dN[0..p]) at u for the knot vector t (default: the
    clamped uniform knots)."""
    t = _knot_vector(n, p, t)
    s = lib().orc_find_span(n, p, _dptr(t), float(u))
    N = np.zeros(p + 1)
    dN = np.zeros(p + 1)
    lib().orc_basis_ders(s, float(u), p, _dptr(t), _dptr(N), _dptr(dN))
    return s, N, dN


def basis_brute(n: int, p: int, u: float, t=None):
    """All n basis functions and derivatives at u by the raw recursion."""
    t = _knot_vector(n, p, t)
    N = np.array([lib().orc_basis_brute(i, p, float(u), _dptr(t), n) for i in range(n)])
    dN = np.array([lib().orc_basis_brute_der(i, p, float(u), _dptr(t), n) for i in range(n)])
    return N, dN


def _model(ctrl: np.ndarray, degree, box_min=(0.0, 0.0, 0.0), box_max=(1.0, 1.0, 1.0), knot_vectors=None,
           weights=None):
    """ctrl: array of shape (n2, n1, n0) (u fastest in memory); FP32
    lattices convert to FP64 exactly.  knot_vectors: None or three entries,
    each None (uniform) or the axis' n + p + 1 knots.  weights: None
    (non-rational) or positive weights shaped like ctrl (NURBS).  Returns the
    ctypes model and the arrays it points into (keep them alive)."""
    ctrl = np.ascontiguousarray(ctrl, dtype=np.float64)
    if ctrl.ndim != 3:
        raise ValueError("ctrl must be 3-D (n_w, n_v, n_u)")
    n = (ctrl.shape[2], ctrl.shape[1], ctrl.shape[0])
    deg = (degree,) * 3 if np.isscalar(degree) else tuple(degree)
    m = Model()
    m.p[:] = [int(x) for x in deg]
    m.n[:] = [int(x) for x in n]
    m.ctrl = ctrl.ctypes.data
    m.box_min[:] = [float(x) for x in box_min]
    m.box_max[:] = [float(x) for x in box_max]
    keep = [ctrl]
    for a, t in enumerate(knot_vectors or (None, None, None)):
        if t is not None:
            t = _knot_vector(m.n[a], m.p[a], t)
            keep.append(t)
            m.knots[a] = t.ctypes.data
    if weights is not None:
        w = np.ascontiguousarray(weights, dtype=np.float64)
        if w.shape != ctrl.shape:
            raise ValueError("weights must have the shape of ctrl")
        keep.append(w)
        m.weights = w.ctypes.data
    return m, keep


def eval_hessian(ctrl, degree, uvw, *, knot_vectors=None, weights=None):
    """(f, f_u, f_v, f_w, f_uu, f_vv, f_ww, f_uv, f_uw, f_vw) in FP64 at FP32
    points (small cases: the derivatives come from the raw recursion)."""
    m, keep = _model(ctrl, degree, knot_vectors=knot_vectors, weights=weights)
    uvw = np.ascontiguousarray(uvw, dtype=np.float32).reshape(-1, 3)
    out = np.zeros((uvw.shape[0], 10), dtype=np.float64)
    if lib().orc_eval_hessian(ctypes.byref(m), uvw.shape[0], uvw.ctypes.data, out.ctypes.data) != 0:
        raise ValueError("oracle: invalid model")
    del keep
    return out


def basis_dk(n: int, p: int, k: int, u: float, t=None):
    """k-th derivatives of all n basis functions at u (raw recursion)."""
    t = _knot_vector(n, p, t)
    return np.array([lib().orc_basis_brute_dk(i, p, k, float(u), _dptr(t), n) for i in range(n)])


def eval_points(ctrl, degree, uvw, *, brute=False, threads=None, with_spans=True, knot_vectors=None, weights=None):
    """Value and gradient (f, df/du, df/dv, df/dw) in FP64 at FP32 points."""
    m, keep = _model(ctrl, degree, knot_vectors=knot_vectors, weights=weights)
    uvw = np.ascontiguousarray(uvw, dtype=np.float32).reshape(-1, 3)
    npts = uvw.shape[0]
    out = np.zeros((npts, 4), dtype=np.float64)
    spans = np.zeros((npts, 3), dtype=np.int32) if (with_spans and not brute) else None
    threads = threads or (os.cpu_count() or 1)
    rc = lib().orc_eval_points(ctypes.byref(m), npts, uvw.ctypes.data, out.ctypes.data,
                               spans.ctypes.data if spans is not None else None,
                               int(threads), int(bool(brute)))
    if rc != 0:
        raise ValueError("oracle: invalid model")
    del keep
    return (out, spans) if spans is not None else out


def render(ctrl, degree, camera: dict, params: dict, *, box_min=(0, 0, 0), box_max=(1, 1, 1),
           row_step=1, threads=None, brute=False, knot_vectors=None, weights=None):
    """Algorithm 1 in FP64.  Returns dict with rgba (H, W, 4), nsamples,
    nambig, rgba_alt, ns_lo and ns_hi (see orc_render in mfa_oracle.c)."""
    m, keep = _model(ctrl, degree, box_min, box_max, knot_vectors, weights)
    cam = Camera()
    cam.kind = int(camera.get("kind", 1))
    cam.eye[:] = [float(x) for x in camera["eye"]]
    cam.center[:] = [float(x) for x in camera.get("center", (0.5, 0.5, 0.5))]
    cam.up[:] = [float(x) for x in camera.get("up", (0.0, 0.0, 1.0))]
    cam.fovy_deg = float(camera.get("fovy_deg", 60.0))
    cam.ortho_height = float(camera.get("ortho_height", 1.0))
    tf = np.ascontiguousarray(params["tf"], dtype=np.float32).reshape(-1, 4)
    rp = RenderParams()
    W, H = int(params["width"]), int(params["height"])
    rp.width, rp.height = W, H
    rp.step = float(params["step"])
    rp.max_opacity = float(params.get("max_opacity", 0.99))
    rp.ref_step = float(params.get("ref_step", 0.0))
    rp.tf_rgba = tf.ctypes.data
    rp.tf_size = tf.shape[0]
    rp.tf_lo = float(params.get("tf_lo", float("nan")))
    rp.tf_hi = float(params.get("tf_hi", float("nan")))
    rp.shading = int(params.get("shading", 1))
    rp.ka = float(params.get("ka", 0.1))
    rp.kd = float(params.get("kd", 0.7))
    rp.ks = float(params.get("ks", 0.2))
    rp.shininess = float(params.get("shininess", 10.0))
    rgba = np.zeros((H, W, 4), dtype=np.float64)
    alt = np.zeros((H, W, 4), dtype=np.float64)
    ns = np.zeros((H, W), dtype=np.int32)
    lo = np.zeros((H, W), dtype=np.int32)
    hi = np.zeros((H, W), dtype=np.int32)
    amb = np.zeros((H, W), dtype=np.int32)
    threads = threads or (os.cpu_count() or 1)
    rc = lib().orc_render(ctypes.byref(m), ctypes.byref(cam), ctypes.byref(rp), int(row_step),
                          int(threads), int(bool(brute)), rgba.ctypes.data, ns.ctypes.data,
                          amb.ctypes.data, alt.ctypes.data, lo.ctypes.data, hi.ctypes.data)
    if rc != 0:
        raise ValueError("oracle: invalid render arguments")
    del keep, tf
    return {"rgba": rgba, "nsamples": ns, "nambig": amb, "rgba_alt": alt, "ns_lo": lo, "ns_hi": hi}
