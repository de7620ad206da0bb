"""Seeded synthetic inputs for MFA-DVR workloads.

This module only makes inputs: control-point lattices, transfer-function
tables, cameras and query points.  It holds none of the rendering or
B-spline evaluation arithmetic, so the CUDA path and the FP64 oracle can both
take their inputs from it.

Fields used as stand-ins for the paper's data (Sec. 4.1.1):
  * Marschner-Lobb (Eq. 2) with f_M = 6, alpha = 0.25 on [-1, 1]^3;
  * Gaussian Beam (Eq. 1) with V in [0, 255], mu = 0, sigma = 1/3, R = sqrt(3);
  * a sum of anisotropic 3-D Gaussians (centres, widths, amplitudes seeded);
  * multi-octave hashed value noise.
The paper fits its MFA models with an encoder (Sec. 2.3, Fig. 1) that is not
part of the rendering path; here control points are set directly by sampling
a field at the Greville abscissae of the clamped uniform knots.

Lattices are float32 arrays of shape (n_w, n_v, n_u): u varies fastest in
memory, i.e. element (i, j, k) sits at i + n_u * (j + n_v * k).
"""
from __future__ import annotations

import math

import numpy as np


def seed_for(config_index: int) -> int:
    """Seed of workload ``config_index`` (1-based)."""
    return 1000 + int(config_index)


# --------------------------------------------------------------------------
# Lattice placement
# --------------------------------------------------------------------------

def graded_knots(rng, n: int, p: int, spread=0.8) -> np.ndarray:
    """A clamped knot vector of n + p + 1 FP32 values with non-uniform interior
    knots (the kind an adaptive MFA fit places, Sec. 2.3): span widths drawn
    from U[1 - spread, 1 + spread] and normalised to [0, 1], so neighbouring
    spans differ by up to a factor (1 + spread) / (1 - spread).  float32."""
    m = n - p
    for _ in range(100):
        w = rng.uniform(1.0 - spread, 1.0 + spread, size=m)
        inner = np.cumsum(w)[:-1] / w.sum()
        t = np.concatenate([np.zeros(p + 1), inner, np.ones(p + 1)]).astype(np.float32)
        if m == 1 or np.all(np.diff(t[p:n + 1]) > 0):
            return t
    raise ValueError("could not draw strictly increasing FP32 knots")


def greville(n: int, p: int) -> np.ndarray:
    """Greville abscissae of the clamped uniform knot vector of n control
    points and degree p (mean of p consecutive interior knots)."""
    m = n - p
    t = np.concatenate([np.zeros(p + 1), np.arange(1, m) / m, np.ones(p + 1)])
    return np.array([t[i + 1:i + p + 1].mean() for i in range(n)])


def _grid(n, p, lo=0.0, hi=1.0):
    """Greville abscissae on each axis, mapped onto [lo, hi]."""
    axes = [lo + (hi - lo) * greville(int(n[d]), int(p)) for d in range(3)]
    return axes


# --------------------------------------------------------------------------
# Fields
# --------------------------------------------------------------------------

def marschner_lobb(x, y, z, f_m=6.0, alpha=0.25):
    """Eq. 2 on [-1, 1]^3."""
    r = np.sqrt(x * x + y * y)
    rho = np.cos(2.0 * np.pi * f_m * np.cos(np.pi * r / 2.0))
    return (1.0 - np.sin(np.pi * z / 2.0) + alpha * (1.0 + rho)) / (2.0 * (1.0 + alpha))


def gaussian_beam(x, y, z, vmin=0.0, vmax=255.0, mu=0.0, sigma=1.0 / 3.0, radius=math.sqrt(3.0)):
    """Eq. 1 on [-1, 1]^3."""
    ell = np.sqrt(x * x + y * y + z * z) / radius
    return vmin + (vmax - vmin) * np.exp(-((ell - mu) ** 2) / (2.0 * sigma * sigma))


def gaussian_sum_params(rng, count=20, sigma_lo=0.02, sigma_hi=0.15):
    centres = rng.uniform(0.0, 1.0, size=(count, 3))
    sigmas = rng.uniform(sigma_lo, sigma_hi, size=(count, 3))
    amps = rng.uniform(-1.0, 1.0, size=count)
    return centres, sigmas, amps


def gaussian_sum_lattice(n, p, rng, count=20):
    """Sum of ``count`` axis-aligned anisotropic Gaussians on [0,1]^3 sampled
    at the Greville abscissae; float32 (n_w, n_v, n_u).  Separable per
    Gaussian, so it is built from 1-D factors."""
    n = tuple(int(v) for v in n)
    xs = _grid(n, p)
    centres, sigmas, amps = gaussian_sum_params(rng, count)
    # 1-D factors per Gaussian: F_d[g, :] along axis d
    F = [np.exp(-((xs[d][None, :] - centres[:, d:d + 1]) ** 2) / (2 * sigmas[:, d:d + 1] ** 2)) for d in range(3)]
    # out[k, j, i] = sum_g a_g Fz[g, k] Fy[g, j] Fx[g, i]: one matrix product
    kj = (amps[:, None, None] * F[2][:, :, None] * F[1][:, None, :]).reshape(count, -1)
    out = kj.T @ F[0]
    return out.reshape(n[2], n[1], n[0]).astype(np.float32)


def field_lattice(field, n, p, lo=-1.0, hi=1.0):
    """Sample ``field(x, y, z)`` at the Greville abscissae mapped to [lo, hi]^3."""
    n = tuple(int(v) for v in n)
    xs = _grid(n, p, lo, hi)
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return field(X, Y, Z).astype(np.float64)


def gaussian_beam_lattice(n, p):
    """Eq. 1 (the Gaussian beam) on [-1, 1]^3 sampled at the Greville
    abscissae; float32 (n_w, n_v, n_u), built one w-slice at a time so that a
    512^3 lattice needs no 512^3 float64 temporaries."""
    n = tuple(int(v) for v in n)
    xs = _grid(n, p, -1.0, 1.0)
    Y, X = np.meshgrid(xs[1], xs[0], indexing="ij")
    out = np.empty((n[2], n[1], n[0]), dtype=np.float32)
    for k, z in enumerate(xs[2]):
        out[k] = gaussian_beam(X, Y, np.full_like(X, z))
    return out


def value_noise_lattice(n, p, rng, octaves=5, persistence=0.5, lacunarity=2.0, base_cells=4):
    """Multi-octave value noise on [0,1]^3 at the Greville abscissae:
    octave o has base_cells * lacunarity^o cells per axis, hashed lattice
    values U[-1, 1], trilinear interpolation with smoothstep weights,
    amplitude persistence^o.  The interpolation is separable, so each octave
    is three small matrix products (one interpolation matrix per axis)."""
    n = tuple(int(v) for v in n)
    xs = _grid(n, p)
    out = np.zeros((n[2], n[1], n[0]), dtype=np.float32)
    amp = 1.0
    for o in range(octaves):
        cells = int(round(base_cells * lacunarity ** o))
        vals = rng.uniform(-1.0, 1.0, size=(cells + 1, cells + 1, cells + 1)).astype(np.float32)
        W = []
        for d in range(3):
            s = xs[d] * cells
            i0 = np.minimum(np.floor(s).astype(np.int64), cells - 1)
            f = s - i0
            w = f * f * (3.0 - 2.0 * f)
            M = np.zeros((n[d], cells + 1), dtype=np.float32)
            M[np.arange(n[d]), i0] = 1.0 - w
            M[np.arange(n[d]), i0 + 1] = w
            W.append(M)
        # vals[c, b, a] (z, y, x) -> out[k, j, i]
        t = vals @ W[0].T                                   # (c, b, i)
        t = np.einsum("jb,cbi->cji", W[1], t, optimize=True)  # (c, j, i)
        t = np.tensordot(W[2], t, axes=([1], [0]))           # (k, j, i)
        out += np.float32(amp) * t.astype(np.float32)
        amp *= persistence
    return out


# --------------------------------------------------------------------------
# Transfer function, camera, points
# --------------------------------------------------------------------------

def transfer_function(rng, size=256, nodes=4, alpha_max=0.5):
    """Piecewise-linear RGBA table from ``nodes`` seeded control nodes:
    x_0 = 0, x_last = 1, inner nodes sorted U(0,1); RGB ~ U(0,1),
    alpha ~ U(0, alpha_max).  float32 (size, 4)."""
    inner = np.sort(rng.uniform(0.0, 1.0, size=nodes - 2))
    xn = np.concatenate([[0.0], inner, [1.0]])
    rgb = rng.uniform(0.0, 1.0, size=(nodes, 3))
    a = rng.uniform(0.0, alpha_max, size=(nodes, 1))
    vals = np.concatenate([rgb, a], axis=1)
    xs = np.linspace(0.0, 1.0, size)
    table = np.stack([np.interp(xs, xn, vals[:, c]) for c in range(4)], axis=1)
    return table.astype(np.float32)


def sphere_camera(rng, radius=2.0, centre=(0.5, 0.5, 0.5), fovy_deg=60.0):
    """Perspective camera on a seeded sphere about ``centre``, looking at it.
    Coordinates are rounded to FP32, the precision of the camera inputs, so
    every consumer sees the same camera."""
    v = rng.normal(size=3)
    v /= np.linalg.norm(v)
    eye = np.asarray(centre) + radius * v
    up = (0.0, 0.0, 1.0) if abs(v[2]) < 0.99 else (0.0, 1.0, 0.0)
    f32 = lambda xs: tuple(float(np.float32(x)) for x in xs)
    return {"kind": 1, "eye": f32(eye), "center": f32(centre), "up": up, "fovy_deg": float(np.float32(fovy_deg)),
            "ortho_height": 1.0}


def axis_ortho_camera():
    """Orthographic view along +z covering the unit box: pixel (x, y) looks
    from ((x+.5)/W, 1-(y+.5)/H, -1) in direction (0, 0, 1)."""
    return {"kind": 0, "eye": (0.5, 0.5, -1.0), "center": (0.5, 0.5, 0.5), "up": (0.0, 1.0, 0.0),
            "fovy_deg": 60.0, "ortho_height": 1.0}


def uniform_points(rng, count):
    """``count`` float32 parameter points U[0,1]^3, shape (count, 3)."""
    return rng.uniform(0.0, 1.0, size=(count, 3)).astype(np.float32)


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------

# The transfer-function opacity of every named workload is the opacity of a
# slab 1/16 of the box thick; samples take alpha_s = 1 - (1 - alpha)^(step /
# REF_STEP).  Applied per sample without the correction, alpha ~ U(0, 0.5)
# at step 1/1024 saturates every ray within a few dozen samples.
REF_STEP = 1.0 / 16.0

def small_ml_workload():
    """Degree 3, 32^3 lattice of Marschner-Lobb (Eq. 2) at the Greville
    abscissae plus N(0, 0.01) noise; 128^2 orthographic view along +z, step
    1/256, 256-entry TF from 4 seeded nodes, shading on, O_max 0.99,
    TF opacity per REF_STEP."""
    rng = np.random.default_rng(seed_for(1))
    p, n = 3, (32, 32, 32)
    ctrl = field_lattice(marschner_lobb, n, p) + rng.normal(0.0, 0.01, size=(n[2], n[1], n[0]))
    tf = transfer_function(rng, 256)
    return {"name": "ml32_p3_ortho128", "degree": p, "ctrl": ctrl.astype(np.float32), "tf": tf,
            "camera": axis_ortho_camera(),
            "params": {"width": 128, "height": 128, "step": 1.0 / 256, "max_opacity": 0.99,
                       "ref_step": REF_STEP, "shading": 1}}


def gaussian_sum_workload(n_eval_points=1 << 24, with_points=True):
    """Degree 3, 128^3 lattice of 20 anisotropic Gaussians; 1024^2
    perspective view (60 deg) from a seeded radius-2 sphere, step 1/1024,
    O_max 0.99, 256-entry TF; plus 2^24 uniform parameter points."""
    rng = np.random.default_rng(seed_for(2))
    p, n = 3, (128, 128, 128)
    ctrl = gaussian_sum_lattice(n, p, rng)
    tf = transfer_function(rng, 256)
    cam = sphere_camera(rng)
    pts = uniform_points(rng, n_eval_points) if with_points else None
    return {"name": "gauss20_128_p3_persp1024", "degree": p, "ctrl": ctrl, "tf": tf, "camera": cam,
            "params": {"width": 1024, "height": 1024, "step": 1.0 / 1024, "max_opacity": 0.99,
                       "ref_step": REF_STEP, "shading": 1},
            "points": pts}


def value_noise_workload(n=512):
    """Degree 4, n^3 lattice of 5-octave value noise; 3840x2160 perspective
    view, step 1/2048, 1024-entry TF."""
    rng = np.random.default_rng(seed_for(5))
    p = 4
    ctrl = value_noise_lattice((n, n, n), p, rng)
    tf = transfer_function(rng, 1024)
    cam = sphere_camera(rng)
    return {"name": f"noise{n}_p4_persp3840x2160", "degree": p, "ctrl": ctrl, "tf": tf, "camera": cam,
            "params": {"width": 3840, "height": 2160, "step": 1.0 / 2048, "max_opacity": 0.99,
                       "ref_step": REF_STEP, "shading": 1}}


def multi_model_workload(count=16, seed_index=3, step=1.0 / 1024):
    """``count`` render jobs for one batched launch: degrees drawn from
    {2, 3, 4, 5}, lattices drawn per axis from 64..256 (anisotropic), each a
    sum of 20 Gaussians as in gaussian_sum_workload; square images of side
    512, 1024 or 2048; seeded cameras and 256-entry TFs."""
    rng = np.random.default_rng(seed_for(seed_index))
    jobs = []
    for _ in range(count):
        p = int(rng.choice([2, 3, 4, 5]))
        n = tuple(int(v) for v in rng.integers(64, 257, size=3))
        side = int(rng.choice([512, 1024, 2048]))
        ctrl = gaussian_sum_lattice(n, p, rng)
        tf = transfer_function(rng, 256)
        cam = sphere_camera(rng)
        jobs.append({"degree": p, "ncp": n, "ctrl": ctrl, "tf": tf, "camera": cam,
                     "params": {"width": side, "height": side, "step": step, "max_opacity": 0.99,
                                "ref_step": REF_STEP, "shading": 1}})
    return jobs


def serving_workload(models=48, requests=2000, rate=200.0, sizes=(256, 512, 1024, 2048), step=1.0 / 512,
                     seed_index=4):
    """Resident models and a request stream for the serving loop: ``models``
    models of degree 3 or 4 with cubic lattices drawn from 96..384 per side
    (Gaussian sums), each with its own 256-entry TF; ``requests`` requests
    arriving as a Poisson process of ``rate`` per second, each drawing its
    model uniformly, its square image side from ``sizes`` and a camera on the
    radius-2 sphere.  Returns (models, requests); a request is a dict with
    arrival time (s), model index, side and camera."""
    rng = np.random.default_rng(seed_for(seed_index))
    mods = []
    for _ in range(models):
        p = int(rng.choice([3, 4]))
        n = int(rng.integers(96, 385))
        mods.append({"degree": p, "ncp": (n, n, n), "ctrl": gaussian_sum_lattice((n, n, n), p, rng),
                     "tf": transfer_function(rng, 256)})
    t = np.cumsum(rng.exponential(1.0 / rate, size=requests))
    reqs = [{"arrival": float(t[i]), "model": int(rng.integers(0, models)), "side": int(rng.choice(sizes)),
             "camera": sphere_camera(rng)} for i in range(requests)]
    params = {"step": step, "max_opacity": 0.99, "ref_step": REF_STEP, "shading": 1}
    return mods, reqs, params
