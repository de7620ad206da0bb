"""Python binding of libmfadvr.so (the C ABI declared in include/mfadvr.h).

Argument marshalling only: every step of the query and rendering path runs in
the library's CUDA kernels.  Device buffers are passed as anything with a
``data_ptr()`` (torch CUDA tensors) or as raw integer addresses; streams as a
``torch.cuda.Stream``, a raw handle or None (the current torch stream when
torch is imported and CUDA is available, else the legacy default stream).

There is no fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

F32, F16, BF16 = 0, 1, 2
QUERY_VALUE, QUERY_GRADIENT, QUERY_BOTH, QUERY_HESSIAN = 1, 2, 3, 4
# mfadvr_render_form
FORM_AUTO, FORM_BSPLINE, FORM_POWER = 0, 1, 2
_DTYPES = {"f32": F32, "float32": F32, "f16": F16, "float16": F16, "bf16": BF16, "bfloat16": BF16}

OK, EINVAL, ENOMEM, ECUDA, ENOTFOUND, ETIMEOUT, EBUSY, EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
MAX_DEGREE = 5
MAX_TF_SIZE = 4096

# Every symbol include/mfadvr.h declares.
EXPORTS = ("mfadvr_create", "mfadvr_destroy", "mfadvr_load_model", "mfadvr_unload_model", "mfadvr_model_info",
           "mfadvr_eval_points", "mfadvr_eval_points_host", "mfadvr_render", "mfadvr_render_host",
           "mfadvr_status_string", "mfadvr_last_error", "mfadvr_render_lattice_noalloc", "mfadvr_render_batch",
           "mfadvr_autotune", "mfadvr_tuning_save", "mfadvr_tuning_load", "mfadvr_serve_start", "mfadvr_serve_stop",
           "mfadvr_submit", "mfadvr_wait", "mfadvr_serve_stats", "mfadvr_serve_trace", "mfadvr_query_points",
           "mfadvr_query_points_host", "mfadvr_query_points_host_async", "mfadvr_probe_fma",
           "mfadvr_render_trace")
MAX_BATCH = 256
NOALLOC_MAX_POINTS = 1 << 19


class MfadvrError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"[{status}] {message}")
        self.status = status


class ModelDesc(ctypes.Structure):
    _fields_ = [("degree", ctypes.c_int32 * 3), ("ncp", ctypes.c_int32 * 3),
                ("box_min", ctypes.c_float * 3), ("box_max", ctypes.c_float * 3),
                ("ctrl", ctypes.c_void_p), ("knots", ctypes.c_void_p * 3), ("storage", ctypes.c_int32),
                ("weights", ctypes.c_void_p), ("render_form", ctypes.c_int32)]


class Camera(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("eye", ctypes.c_float * 3), ("center", ctypes.c_float * 3),
                ("up", ctypes.c_float * 3), ("fovy_deg", ctypes.c_float), ("ortho_height", ctypes.c_float)]


class RenderParams(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("step", ctypes.c_float),
                ("max_opacity", ctypes.c_float), ("ref_step", ctypes.c_float), ("tf_rgba", ctypes.c_void_p),
                ("tf_size", ctypes.c_int32), ("tf_lo", ctypes.c_float), ("tf_hi", ctypes.c_float),
                ("shading", ctypes.c_int32), ("ka", ctypes.c_float), ("kd", ctypes.c_float),
                ("ks", ctypes.c_float), ("shininess", ctypes.c_float)]


class RenderJob(ctypes.Structure):
    _fields_ = [("model_id", ctypes.c_int32), ("camera", Camera), ("params", RenderParams),
                ("rgba_dev", ctypes.c_void_p), ("nsamples_dev", ctypes.c_void_p)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("frame_budget_bytes", ctypes.c_uint64), ("max_batch", ctypes.c_int32),
                ("max_in_flight", ctypes.c_int32)]


class ServeTraceRecord(ctypes.Structure):
    _fields_ = [("oldest_submit_us", ctypes.c_int64), ("t_admit_us", ctypes.c_int64),
                ("t_launched_us", ctypes.c_int64), ("t_done_us", ctypes.c_int64), ("jobs", ctypes.c_int32),
                ("groups", ctypes.c_int32), ("stream", ctypes.c_int32), ("queued_after", ctypes.c_int32)]


class Tuning(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("ms", ctypes.c_float)]


_lib = None


def load_library(build_if_missing: bool = True):
    """Load (building first if needed) libmfadvr.so; raises if impossible."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise ImportError(f"libmfadvr.so not found at {path}; build it with paper_2204_11762_gb300.build")
    L = ctypes.CDLL(path)
    vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    P = ctypes.POINTER
    sig = {
        "mfadvr_create": [P(vp), ctypes.c_int, u64],
        "mfadvr_destroy": [vp],
        "mfadvr_load_model": [vp, P(ModelDesc), P(i32)],
        "mfadvr_unload_model": [vp, i32],
        "mfadvr_model_info": [vp, i32, P(ctypes.c_float), P(ctypes.c_float), P(ctypes.c_float), P(u64)],
        "mfadvr_eval_points": [vp, i32, vp, i64, vp, vp, vp],
        "mfadvr_eval_points_host": [vp, i32, vp, i64, vp, vp, vp],
        "mfadvr_query_points": [vp, i32, vp, i64, i32, vp, vp, vp],
        "mfadvr_query_points_host": [vp, i32, vp, i64, i32, vp, vp, vp],
        "mfadvr_query_points_host_async": [vp, i32, vp, i64, i32, vp, vp, i32, vp],
        "mfadvr_render": [vp, i32, P(Camera), P(RenderParams), vp, vp, vp],
        "mfadvr_render_host": [vp, i32, P(Camera), P(RenderParams), vp, vp, vp],
        "mfadvr_render_trace": [vp, i32, P(Camera), P(RenderParams), vp, vp, i32, vp, vp, vp],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = i32
    L.mfadvr_render_batch.argtypes = [vp, i32, P(RenderJob), vp]
    L.mfadvr_render_batch.restype = i32
    L.mfadvr_autotune.argtypes = [vp, i32, P(Camera), P(RenderParams), vp, vp, vp, P(Tuning)]
    L.mfadvr_autotune.restype = i32
    L.mfadvr_tuning_save.argtypes = [vp, ctypes.c_char_p]
    L.mfadvr_tuning_save.restype = i32
    L.mfadvr_tuning_load.argtypes = [vp, ctypes.c_char_p]
    L.mfadvr_tuning_load.restype = i32
    L.mfadvr_serve_start.argtypes = [vp, P(ServeConfig)]
    L.mfadvr_serve_stop.argtypes = [vp]
    L.mfadvr_submit.argtypes = [vp, P(RenderJob), P(u64)]
    L.mfadvr_wait.argtypes = [vp, u64, i64, P(i64)]
    L.mfadvr_serve_stats.argtypes = [vp, P(u64), P(u64), P(u64)]
    L.mfadvr_serve_trace.argtypes = [vp, P(ServeTraceRecord), i32, P(i32)]
    for name in ("mfadvr_serve_start", "mfadvr_serve_stop", "mfadvr_submit", "mfadvr_wait", "mfadvr_serve_stats",
                 "mfadvr_serve_trace"):
        getattr(L, name).restype = i32
    f3, i3 = ctypes.c_float * 3, ctypes.c_int32 * 3
    L.mfadvr_render_lattice_noalloc.argtypes = [vp, P(i3), P(i3), P(f3), P(f3), P(Camera), P(RenderParams),
                                                vp, vp, vp]
    L.mfadvr_render_lattice_noalloc.restype = i32
    L.mfadvr_probe_fma.argtypes = [i32, i32, vp, vp, P(ctypes.c_double)]
    L.mfadvr_probe_fma.restype = i32
    L.mfadvr_status_string.argtypes = [i32]
    L.mfadvr_status_string.restype = ctypes.c_char_p
    L.mfadvr_last_error.argtypes = [vp]
    L.mfadvr_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        return int(x.ctypes.data)
    raise TypeError(f"cannot take the address of {type(x)!r}")


def _stream(s) -> int | None:
    if s is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return int(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return None
    if isinstance(s, int):
        return s
    if hasattr(s, "cuda_stream"):
        return int(s.cuda_stream)
    raise TypeError(f"not a stream: {type(s)!r}")


def make_camera(cam: dict) -> Camera:
    c = Camera()
    c.kind = int(cam.get("kind", 1))
    c.eye[:] = [float(v) for v in cam["eye"]]
    c.center[:] = [float(v) for v in cam.get("center", (0.5, 0.5, 0.5))]
    c.up[:] = [float(v) for v in cam.get("up", (0.0, 0.0, 1.0))]
    c.fovy_deg = float(cam.get("fovy_deg", 60.0))
    c.ortho_height = float(cam.get("ortho_height", 1.0))
    return c


def make_params(prm: dict, tf_ptr: int, tf_size: int) -> RenderParams:
    r = RenderParams()
    r.width, r.height = int(prm["width"]), int(prm["height"])
    r.step = float(prm["step"])
    r.max_opacity = float(prm.get("max_opacity", 0.99))
    r.ref_step = float(prm.get("ref_step", 0.0))
    r.tf_rgba = tf_ptr
    r.tf_size = int(tf_size)
    r.tf_lo = float(prm.get("tf_lo", math.nan))
    r.tf_hi = float(prm.get("tf_hi", math.nan))
    r.shading = int(prm.get("shading", 1))
    r.ka = float(prm.get("ka", 0.1))
    r.kd = float(prm.get("kd", 0.7))
    r.ks = float(prm.get("ks", 0.2))
    r.shininess = float(prm.get("shininess", 10.0))
    return r


def render_lattice_noalloc(ctrl_dev, degree: int, ncp, camera: dict, params: dict, tf_dev, tf_size, rgba_dev,
                           nsamples_dev=None, box_min=(0.0, 0.0, 0.0), box_max=(1.0, 1.0, 1.0), stream=None):
    """mfadvr_render_lattice_noalloc: render from a caller-owned FP32 device
    lattice (u fastest, ncp = (n_u, n_v, n_w)) without any allocation."""
    L = load_library()
    i3, f3 = ctypes.c_int32 * 3, ctypes.c_float * 3
    cam = make_camera(camera)
    prm = make_params(params, _ptr(tf_dev), tf_size)
    st = L.mfadvr_render_lattice_noalloc(_ptr(ctrl_dev), ctypes.byref(i3(*([int(degree)] * 3))),
                                         ctypes.byref(i3(*[int(v) for v in ncp])),
                                         ctypes.byref(f3(*[float(v) for v in box_min])),
                                         ctypes.byref(f3(*[float(v) for v in box_max])), ctypes.byref(cam),
                                         ctypes.byref(prm), _ptr(rgba_dev), _ptr(nsamples_dev), _stream(stream))
    if st != OK:
        raise MfadvrError(st, L.mfadvr_last_error(None).decode())


def probe_fma(sink_dev, iters: int, packed: bool = True, stream=None) -> float:
    """mfadvr_probe_fma: enqueue the FP32 multiply-add throughput probe on
    `stream` (current device); returns the multiply-adds the launch runs."""
    L = load_library()
    n = ctypes.c_double(0.0)
    st = L.mfadvr_probe_fma(int(bool(packed)), int(iters), _ptr(sink_dev), _stream(stream), ctypes.byref(n))
    if st != OK:
        raise MfadvrError(st, L.mfadvr_last_error(None).decode())
    return n.value


class Context:
    """One library context on one CUDA device (mfadvr_create)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self._L = load_library()
        h = ctypes.c_void_p()
        st = self._L.mfadvr_create(ctypes.byref(h), int(device), int(hbm_budget_bytes))
        if st != OK:
            raise MfadvrError(st, self._L.mfadvr_last_error(None).decode())
        self._h = h

    # -- plumbing ---------------------------------------------------------
    def _check(self, st):
        if st != OK:
            raise MfadvrError(st, self._L.mfadvr_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.mfadvr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> int:
        return self._h.value

    # -- model store ------------------------------------------------------
    def load_model(self, ctrl, degree, storage="f32", box_min=(0.0, 0.0, 0.0), box_max=(1.0, 1.0, 1.0),
                   knots=None, weights=None, render_form=FORM_AUTO) -> int:
        """ctrl: float32 array (n_w, n_v, n_u), u fastest in memory.  knots:
        None (uniform) or three entries, each None or n_d + p + 1 clamped knots
        (u, v, w order).  weights: None or positive weights shaped like ctrl
        (a rational model).  render_form: FORM_AUTO, FORM_BSPLINE or FORM_POWER
        (span polynomials for the render kernels)."""
        ctrl = np.ascontiguousarray(ctrl, dtype=np.float32)
        if ctrl.ndim != 3:
            raise ValueError("ctrl must be a 3-D array (n_w, n_v, n_u)")
        deg = (int(degree),) * 3 if np.isscalar(degree) else tuple(int(d) for d in degree)
        d = ModelDesc()
        d.degree[:] = list(deg)
        d.ncp[:] = [ctrl.shape[2], ctrl.shape[1], ctrl.shape[0]]
        d.box_min[:] = [float(v) for v in box_min]
        d.box_max[:] = [float(v) for v in box_max]
        d.ctrl = ctrl.ctypes.data
        d.storage = _DTYPES[storage] if isinstance(storage, str) else int(storage)
        keep = []
        for a, t in enumerate(knots or (None, None, None)):
            if t is not None:
                t = np.ascontiguousarray(t, dtype=np.float32).ravel()
                keep.append(t)
                d.knots[a] = t.ctypes.data
        if weights is not None:
            w = np.ascontiguousarray(weights, dtype=np.float32)
            if w.shape != ctrl.shape:
                raise ValueError("weights must have the shape of ctrl")
            keep.append(w)
            d.weights = w.ctypes.data
        d.render_form = int(render_form)
        mid = ctypes.c_int32(-1)
        self._check(self._L.mfadvr_load_model(self._h, ctypes.byref(d), ctypes.byref(mid)))
        return mid.value

    def unload_model(self, model_id: int):
        self._check(self._L.mfadvr_unload_model(self._h, int(model_id)))

    def model_info(self, model_id: int) -> dict:
        lo, hi, sc = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
        b = ctypes.c_uint64()
        self._check(self._L.mfadvr_model_info(self._h, int(model_id), ctypes.byref(lo), ctypes.byref(hi),
                                              ctypes.byref(sc), ctypes.byref(b)))
        return {"pmin": lo.value, "pmax": hi.value, "scale": sc.value, "bytes": b.value}

    # -- queries ----------------------------------------------------------
    def eval_points(self, model_id, params_dev, n, out_dev, spans_dev=None, stream=None):
        self._check(self._L.mfadvr_eval_points(self._h, int(model_id), _ptr(params_dev), int(n), _ptr(out_dev),
                                               _ptr(spans_dev), _stream(stream)))

    def eval_points_host(self, model_id, params, out=None, spans=None, stream=None):
        params = np.ascontiguousarray(params, dtype=np.float32).reshape(-1, 3)
        n = params.shape[0]
        if out is None:
            out = np.empty((n, 4), dtype=np.float32)
        self._check(self._L.mfadvr_eval_points_host(self._h, int(model_id), _ptr(params), n, _ptr(out),
                                                    _ptr(spans), _stream(stream)))
        return out

    def query_points(self, model_id, params_dev, n, out_dev, query=QUERY_BOTH, spans_dev=None, stream=None):
        """eval_points for one query: out_dev holds n values (QUERY_VALUE), n x 3
        gradients (QUERY_GRADIENT), n x 4 (QUERY_BOTH) or n x 10 (QUERY_HESSIAN:
        f, f_u, f_v, f_w, f_uu, f_vv, f_ww, f_uv, f_uw, f_vw)."""
        self._check(self._L.mfadvr_query_points(self._h, int(model_id), _ptr(params_dev), int(n), int(query),
                                                _ptr(out_dev), _ptr(spans_dev), _stream(stream)))

    def query_points_host(self, model_id, params, query=QUERY_BOTH, out=None, spans=None, stream=None):
        params = np.ascontiguousarray(params, dtype=np.float32).reshape(-1, 3)
        n = params.shape[0]
        if out is None:
            shape = {QUERY_VALUE: (n,), QUERY_GRADIENT: (n, 3), QUERY_HESSIAN: (n, 10)}.get(int(query), (n, 4))
            out = np.empty(shape, dtype=np.float32)
        self._check(self._L.mfadvr_query_points_host(self._h, int(model_id), _ptr(params), n, int(query),
                                                     _ptr(out), _ptr(spans), _stream(stream)))
        return out

    def query_points_host_async(self, model_id, params_pinned, n, out_pinned, query=QUERY_BOTH, spans_pinned=None,
                                max_ctas=0, stream=None):
        """query_points on page-locked host buffers (pinned tensors or arrays in
        page-locked memory), queued on `stream` without waiting: the results are
        in out_pinned once the stream has reached this call.  max_ctas caps the
        256-thread blocks that serve it (0: the whole GPU)."""
        self._check(self._L.mfadvr_query_points_host_async(self._h, int(model_id), _ptr(params_pinned), int(n),
                                                           int(query), _ptr(out_pinned), _ptr(spans_pinned),
                                                           int(max_ctas), _stream(stream)))

    def render(self, model_id, camera: dict, params: dict, tf_dev, tf_size, rgba_dev, nsamples_dev=None,
               stream=None):
        cam = make_camera(camera)
        prm = make_params(params, _ptr(tf_dev), tf_size)
        self._check(self._L.mfadvr_render(self._h, int(model_id), ctypes.byref(cam), ctypes.byref(prm),
                                          _ptr(rgba_dev), _ptr(nsamples_dev), _stream(stream)))

    def render_trace(self, model_id, camera: dict, params: dict, tf_dev, tf_size, rgba_dev, nsamples_dev,
                     max_samples: int, pos_dev, span_dev, stream=None):
        """mfadvr_render_trace: render and record each ray's first max_samples
        sample positions (H x W x max_samples x 3 float32) and knot spans
        (same shape, int32) in the caller's device buffers."""
        cam = make_camera(camera)
        prm = make_params(params, _ptr(tf_dev), tf_size)
        self._check(self._L.mfadvr_render_trace(self._h, int(model_id), ctypes.byref(cam), ctypes.byref(prm),
                                                _ptr(rgba_dev), _ptr(nsamples_dev), int(max_samples),
                                                _ptr(pos_dev), _ptr(span_dev), _stream(stream)))

    def render_host(self, model_id, camera: dict, params: dict, tf, rgba=None, nsamples=None, stream=None):
        tf = np.ascontiguousarray(tf, dtype=np.float32).reshape(-1, 4)
        W, H = int(params["width"]), int(params["height"])
        if rgba is None:
            rgba = np.empty((H, W, 4), dtype=np.float32)
        cam = make_camera(camera)
        prm = make_params(params, _ptr(tf), tf.shape[0])
        self._check(self._L.mfadvr_render_host(self._h, int(model_id), ctypes.byref(cam), ctypes.byref(prm),
                                               _ptr(rgba), _ptr(nsamples), _stream(stream)))
        return rgba

    # -- serving ----------------------------------------------------------
    def serve_start(self, frame_budget_bytes=0, max_batch=0, max_in_flight=0):
        cfg = ServeConfig(int(frame_budget_bytes), int(max_batch), int(max_in_flight))
        self._check(self._L.mfadvr_serve_start(self._h, ctypes.byref(cfg)))

    def serve_stop(self):
        self._check(self._L.mfadvr_serve_stop(self._h))

    def submit(self, job: dict) -> int:
        """Queue one render request (same dict as render_batch jobs)."""
        j = RenderJob()
        j.model_id = int(job["model_id"])
        j.camera = make_camera(job["camera"])
        j.params = make_params(job["params"], _ptr(job["tf_dev"]), job["tf_size"])
        j.rgba_dev = _ptr(job["rgba_dev"])
        j.nsamples_dev = _ptr(job.get("nsamples_dev"))
        t = ctypes.c_uint64()
        self._check(self._L.mfadvr_submit(self._h, ctypes.byref(j), ctypes.byref(t)))
        return t.value

    def wait(self, ticket: int, timeout_us: int = -1):
        """Latency in microseconds once done; None on timeout."""
        lat = ctypes.c_int64()
        st = self._L.mfadvr_wait(self._h, int(ticket), int(timeout_us), ctypes.byref(lat))
        if st == ETIMEOUT:
            return None
        self._check(st)
        return lat.value

    def serve_stats(self) -> dict:
        a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        self._check(self._L.mfadvr_serve_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"launches": a.value, "graph_updates": b.value, "graph_instantiations": c.value}

    def serve_trace(self, capacity: int = 4096) -> list:
        """The most recent completed batches of the serving loop, oldest first."""
        buf = (ServeTraceRecord * capacity)()
        n = ctypes.c_int32()
        self._check(self._L.mfadvr_serve_trace(self._h, buf, capacity, ctypes.byref(n)))
        return [{f: getattr(buf[i], f) for f, _ in ServeTraceRecord._fields_} for i in range(n.value)]

    # -- batches and tuning -----------------------------------------------
    def render_batch(self, jobs, stream=None):
        """jobs: dicts with model_id, camera, params, tf_dev, tf_size,
        rgba_dev and optionally nsamples_dev (mfadvr_render_batch)."""
        arr = (RenderJob * len(jobs))()
        for k, j in enumerate(jobs):
            arr[k].model_id = int(j["model_id"])
            arr[k].camera = make_camera(j["camera"])
            arr[k].params = make_params(j["params"], _ptr(j["tf_dev"]), j["tf_size"])
            arr[k].rgba_dev = _ptr(j["rgba_dev"])
            arr[k].nsamples_dev = _ptr(j.get("nsamples_dev"))
        self._check(self._L.mfadvr_render_batch(self._h, len(jobs), arr, _stream(stream)))

    def autotune(self, model_id, camera: dict, params: dict, tf_dev, tf_size, rgba_dev, nsamples_dev=None,
                 stream=None) -> dict:
        cam = make_camera(camera)
        prm = make_params(params, _ptr(tf_dev), tf_size)
        t = Tuning()
        self._check(self._L.mfadvr_autotune(self._h, int(model_id), ctypes.byref(cam), ctypes.byref(prm),
                                            _ptr(rgba_dev), _ptr(nsamples_dev), _stream(stream), ctypes.byref(t)))
        return {"tile_w": t.tile_w, "ctas_per_sm": t.ctas_per_sm, "ms": t.ms}

    def tuning_save(self, path: str):
        self._check(self._L.mfadvr_tuning_save(self._h, os.fsencode(path)))

    def tuning_load(self, path: str):
        self._check(self._L.mfadvr_tuning_load(self._h, os.fsencode(path)))
