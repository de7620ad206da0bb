"""Pins for the FP64 oracle: each test checks it against something other than
itself -- closed forms, library routines, exact integer arithmetic, invariants
and brute force -- so that a dropped term, a wrong index or sign, or a
transposed operand in the oracle fails at least one of them."""
import math
import os
from fractions import Fraction
from itertools import product

import numpy as np
import pytest
from scipy.interpolate import BSpline, NdBSpline, RegularGridInterpolator

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

CASES_1D = [(2, 1), (5, 1), (3, 2), (9, 2), (4, 3), (5, 3), (12, 3), (5, 4), (14, 4), (6, 5), (17, 5)]


def _f32(x):
    return float(np.float32(x))


# --------------------------------------------------------------------------
# 1-D basis
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,p", CASES_1D)
def test_partition_of_unity_and_nonnegativity(orc, n, p):
    rng = np.random.default_rng(7)
    m = n - p
    us = list(rng.uniform(0, 1, 2000)) + [j / m for j in range(m + 1)]
    for u in us:
        s, N, dN = orc.basis_ders(n, p, u)
        assert p <= s <= n - 1
        assert abs(N.sum() - 1.0) < 1e-14
        assert abs(dN.sum()) < 1e-11 * m
        assert (N >= -1e-16).all()


@pytest.mark.parametrize("n,p", CASES_1D)
def test_span_mode_equals_brute_mode_1d(orc, n, p):
    rng = np.random.default_rng(11)
    m = n - p
    for u in list(rng.uniform(0, 1, 200)) + [0.0, 1.0] + [j / m for j in range(1, m)]:
        s, N, dN = orc.basis_ders(n, p, u)
        Nb, dNb = orc.basis_brute(n, p, u)
        full = np.zeros(n)
        dfull = np.zeros(n)
        full[s - p:s + 1] = N
        dfull[s - p:s + 1] = dN
        np.testing.assert_allclose(full, Nb, atol=1e-14)
        np.testing.assert_allclose(dfull, dNb, atol=1e-12 * m)


@pytest.mark.parametrize("n,p", CASES_1D)
def test_basis_matches_scipy_bspline(orc, n, p):
    """scipy's de Boor evaluation of the same clamped knot vector."""
    rng = np.random.default_rng(3)
    t = orc.knots(n, p)
    us = rng.uniform(0, 1, 300)
    D = BSpline.design_matrix(us, t, p).toarray()
    for row, u in zip(D, us):
        s, N, dN = orc.basis_ders(n, p, u)
        full = np.zeros(n)
        full[s - p:s + 1] = N
        np.testing.assert_allclose(full, row, atol=1e-13)
    for i in range(n):
        c = np.zeros(n)
        c[i] = 1.0
        dspl = BSpline(t, c, p).derivative()
        for u in us[:40]:
            s, N, dN = orc.basis_ders(n, p, u)
            got = dN[i - (s - p)] if s - p <= i <= s else 0.0
            assert abs(got - float(dspl(u))) < 1e-10 * (n - p)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_single_span_is_bernstein(orc, p):
    """n = p + 1: the clamped basis is the Bernstein basis of degree p."""
    for u in np.linspace(0, 1, 37):
        s, N, dN = orc.basis_ders(p + 1, p, u)
        bern = [math.comb(p, r) * u ** r * (1 - u) ** (p - r) for r in range(p + 1)]
        dbern = [p * ((math.comb(p - 1, r - 1) * u ** (r - 1) * (1 - u) ** (p - r) if r >= 1 else 0.0)
                      - (math.comb(p - 1, r) * u ** r * (1 - u) ** (p - 1 - r) if r <= p - 1 else 0.0))
                 for r in range(p + 1)]
        np.testing.assert_allclose(N, bern, atol=1e-14)
        np.testing.assert_allclose(dN, dbern, atol=1e-12)


def _golden_uniform():
    rows = {}
    with open(os.path.join(GOLDEN, "uniform_bspline_basis.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            p, vals, ders = line.split("|")
            rows[int(p)] = ([float(Fraction(x)) for x in vals.split()],
                            [float(Fraction(x)) for x in ders.split()])
    return rows


@pytest.mark.parametrize("p", [1, 2, 3])
def test_interior_span_matches_textbook_uniform_pieces(orc, p):
    vals, ders = _golden_uniform()[p]
    m = 4 * p + 4
    n = m + p
    j = 2 * p + 1  # interior span index (local), knots t_{s-p+1}..t_{s+p} uniform
    u = (j + 0.5) / m
    s, N, dN = orc.basis_ders(n, p, u)
    assert s == p + j
    np.testing.assert_allclose(N, vals, atol=1e-14)
    np.testing.assert_allclose(dN / m, ders, atol=1e-13)


# --------------------------------------------------------------------------
# Knot spans: exact integer work
# --------------------------------------------------------------------------

def _span_exact(u32, n, p):
    """p + floor(u*m) in exact rational arithmetic, clamped to [p, n-1]."""
    m = n - p
    k = math.floor(Fraction(u32) * m)
    return p + min(max(k, 0), m - 1)


@pytest.mark.parametrize("n,p", [(128, 3), (131, 3), (512, 4), (69, 2), (261, 5), (4, 3), (2, 1), (300, 4)])
def test_span_is_exact_floor(orc, n, p):
    rng = np.random.default_rng(5)
    m = n - p
    us = [_f32(x) for x in rng.uniform(0, 1, 500)]
    # values at and next to every knot, in FP32
    for j in range(0, m + 1, max(1, m // 40)):
        k32 = np.float32(j / m)
        us += [float(k32), float(np.nextafter(k32, np.float32(2))), float(np.nextafter(k32, np.float32(-1)))]
    us += [0.0, 1.0]
    for u in us:
        u = min(max(u, 0.0), 1.0)
        assert orc.find_span(n, p, u) == _span_exact(u, n, p), (u, n, p)


def test_point_query_spans_are_exact_floor(orc):
    """The spans a point query reports, per axis, equal p + floor(u m) in
    exact arithmetic on the clamped FP32 coordinate; points outside [0, 1]
    take the end spans.  Several threads share the points."""
    rng = np.random.default_rng(6)
    p, n = 3, (9, 8, 13)
    ctrl = rng.normal(size=(n[2], n[1], n[0]))
    cols = []
    for d in range(3):
        m = n[d] - p
        us = list(rng.uniform(-0.1, 1.1, 300))
        for j in range(m + 1):
            k32 = np.float32(j / m)
            us += [float(k32), float(np.nextafter(k32, np.float32(2))), float(np.nextafter(k32, np.float32(-1)))]
        cols.append(us)
    npts = max(len(c) for c in cols)  # shorter axes padded with more random points
    uvw = np.stack([np.asarray(c + list(rng.uniform(0, 1, npts - len(c))), dtype=np.float32) for c in cols], axis=1)
    _, spans = orc.eval_points(ctrl, p, uvw, threads=3)
    for d in range(3):
        want = [_span_exact(min(max(float(u), 0.0), 1.0), n[d], p) for u in uvw[:, d]]
        np.testing.assert_array_equal(spans[:, d], want)


# --------------------------------------------------------------------------
# Tensor-product queries
# --------------------------------------------------------------------------

def _lattice(rng, n):
    return rng.normal(size=(n[2], n[1], n[0]))


@pytest.mark.parametrize("p,n", [(1, (4, 5, 3)), (2, (6, 5, 7)), (3, (9, 8, 10)), (4, (7, 9, 6)), (5, (8, 6, 7)),
                                 ((3, 2, 1), (7, 5, 4))])
def test_tensor_eval_matches_scipy_ndbspline(orc, p, n):
    rng = np.random.default_rng(17)
    deg = (p,) * 3 if np.isscalar(p) else p
    ctrl = _lattice(rng, n)
    pts = rng.uniform(0, 1, size=(200, 3)).astype(np.float32)
    pts[:4] = [[0, 0, 0], [1, 1, 1], [0, 1, 0.5], [1, 0, 0.25]]
    out, spans = orc.eval_points(ctrl, deg, pts)
    t = tuple(orc.knots(n[d], deg[d]) for d in range(3))
    c = ctrl.transpose(2, 1, 0)  # (n_u, n_v, n_w)
    spl = NdBSpline(t, c, deg)
    x = pts.astype(np.float64)
    np.testing.assert_allclose(out[:, 0], spl(x), atol=1e-12)
    for d in range(3):
        nu = [0, 0, 0]
        nu[d] = 1
        np.testing.assert_allclose(out[:, 1 + d], spl(x, nu=nu), atol=1e-10 * max(n))


def _marsden_coeffs(t, p, n, r):
    """Control points of u^r (r <= p): the symmetric mean of order r of the
    p interior knots of each basis function (Marsden's identity)."""
    from itertools import combinations
    out = np.zeros(n)
    for i in range(n):
        ks = t[i + 1:i + p + 1]
        out[i] = sum(np.prod(c) for c in combinations(ks, r)) / math.comb(p, r) if r else 1.0
    return out


@pytest.mark.parametrize("p,n", [(1, 6), (2, 7), (3, 11), (4, 9), (5, 12)])
def test_polynomial_reproduction_marsden(orc, p, n):
    """Every monomial u^a v^b w^c with a, b, c <= p is reproduced exactly,
    value and analytic partial derivatives."""
    rng = np.random.default_rng(23)
    t = orc.knots(n, p)
    pts = rng.uniform(0, 1, size=(60, 3)).astype(np.float32)
    x = pts.astype(np.float64)
    for (a, b, c) in [(p, 0, 0), (0, p, 0), (0, 0, p), (1, 1, 1), (p, p - 1, 1), (p, p, p), (0, 0, 0)]:
        ca, cb, cc = (_marsden_coeffs(t, p, n, r) for r in (a, b, c))
        ctrl = cc[:, None, None] * cb[None, :, None] * ca[None, None, :]
        out, _ = orc.eval_points(ctrl, p, pts)
        u, v, w = x[:, 0], x[:, 1], x[:, 2]
        f = u ** a * v ** b * w ** c
        fu = a * u ** max(a - 1, 0) * v ** b * w ** c
        fv = b * u ** a * v ** max(b - 1, 0) * w ** c
        fw = c * u ** a * v ** b * w ** max(c - 1, 0)
        np.testing.assert_allclose(out[:, 0], f, atol=1e-12)
        np.testing.assert_allclose(out[:, 1], fu, atol=1e-11)
        np.testing.assert_allclose(out[:, 2], fv, atol=1e-11)
        np.testing.assert_allclose(out[:, 3], fw, atol=1e-11)


def test_greville_sampling_reproduces_linear_fields(orc):
    """Control points f(Greville) reproduce degree <= 1 fields exactly."""
    from paper_2204_11762_gb300.workloads import field_lattice
    p, n = 3, (9, 10, 11)
    lin = lambda X, Y, Z: 0.3 + 1.5 * X - 2.0 * Y + 0.25 * Z
    ctrl = field_lattice(lin, n, p, lo=0.0, hi=1.0)
    pts = np.random.default_rng(2).uniform(0, 1, size=(100, 3)).astype(np.float32)
    out, _ = orc.eval_points(ctrl, p, pts)
    x = pts.astype(np.float64)
    np.testing.assert_allclose(out[:, 0], lin(x[:, 0], x[:, 1], x[:, 2]), atol=1e-12)
    np.testing.assert_allclose(out[:, 1:], np.tile([1.5, -2.0, 0.25], (100, 1)), atol=1e-11)


def test_gradient_central_differences(orc):
    rng = np.random.default_rng(29)
    p, n = 3, (10, 9, 11)
    ctrl = _lattice(rng, n)
    h = 2.0 ** -17
    base = (np.round(rng.uniform(0.1, 0.9, size=(40, 3)) * 2 ** 20) / 2 ** 20).astype(np.float32)
    out, _ = orc.eval_points(ctrl, p, base)
    scale = np.abs(ctrl).max() * max(n)
    for d in range(3):
        e = np.zeros(3, dtype=np.float32)
        e[d] = h
        fp, _ = orc.eval_points(ctrl, p, base + e)
        fm, _ = orc.eval_points(ctrl, p, base - e)
        fd = (fp[:, 0] - fm[:, 0]) / (2 * h)
        assert np.max(np.abs(fd - out[:, 1 + d])) < 1e-6 * scale


@pytest.mark.parametrize("p,n", [(1, (3, 4, 3)), (2, (5, 4, 6)), (3, (6, 5, 4))])
def test_tensor_span_mode_equals_brute_mode(orc, p, n):
    rng = np.random.default_rng(31)
    ctrl = _lattice(rng, n)
    pts = rng.uniform(0, 1, size=(50, 3)).astype(np.float32)
    pts[0] = [1, 1, 1]
    a, _ = orc.eval_points(ctrl, p, pts)
    b = orc.eval_points(ctrl, p, pts, brute=True)
    np.testing.assert_allclose(a, b, atol=1e-12)


def test_degree1_is_trilinear_interpolation(orc):
    """p = 1 with knots i/(n-1): the model is trilinear interpolation of the
    lattice (scipy RegularGridInterpolator)."""
    rng = np.random.default_rng(37)
    n = (5, 7, 4)
    ctrl = _lattice(rng, n)
    grid = tuple(np.linspace(0, 1, n[d]) for d in range(3))
    rgi = RegularGridInterpolator(grid, ctrl.transpose(2, 1, 0), method="linear")
    pts = rng.uniform(0, 1, size=(300, 3)).astype(np.float32)
    out, _ = orc.eval_points(ctrl, 1, pts)
    np.testing.assert_allclose(out[:, 0], rgi(pts.astype(np.float64)), atol=1e-12)


def test_out_of_box_points_clamp(orc):
    rng = np.random.default_rng(41)
    ctrl = _lattice(rng, (6, 6, 6))
    pts = np.array([[-0.5, 0.5, 0.5], [1.5, 0.2, 2.0], [np.nan, 0.3, 0.3]], dtype=np.float32)
    ref = np.array([[0.0, 0.5, 0.5], [1.0, 0.2, 1.0], [0.0, 0.3, 0.3]], dtype=np.float32)
    a, sa = orc.eval_points(ctrl, 3, pts)
    b, sb = orc.eval_points(ctrl, 3, ref)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(sa, sb)


def test_marschner_lobb_error_shrinks_with_lattice(orc):
    """Loose sanity check: the MFA of Eq. 2 sampled at the Greville abscissae
    approaches the analytic field as the lattice is refined."""
    from paper_2204_11762_gb300.workloads import field_lattice, marschner_lobb
    rng = np.random.default_rng(43)
    pts = rng.uniform(0.05, 0.95, size=(400, 3)).astype(np.float32)
    x = 2 * pts.astype(np.float64) - 1
    truth = marschner_lobb(x[:, 0], x[:, 1], x[:, 2])
    errs = []
    for n in (16, 32, 64, 128):
        ctrl = field_lattice(marschner_lobb, (n, n, n), 3)
        out, _ = orc.eval_points(ctrl, 3, pts)
        errs.append(np.sqrt(np.mean((out[:, 0] - truth) ** 2)))
    assert errs[0] > errs[1] > errs[2] > errs[3]
    # second-order once the f_M = 6 ripples are resolved (64 -> 128)
    assert errs[3] < 0.35 * errs[2]


# --------------------------------------------------------------------------
# Ray caster (Algorithm 1)
# --------------------------------------------------------------------------

def _const_tf(rgba, size=8):
    return np.tile(np.asarray(rgba, dtype=np.float32), (size, 1))


def _ortho(W=8, H=8):
    return {"kind": 0, "eye": (0.5, 0.5, -1.0), "center": (0.5, 0.5, 0.5), "up": (0.0, 1.0, 0.0),
            "ortho_height": 1.0}


@pytest.mark.parametrize("alpha,step,ert", [(0.01, 1 / 64, 1.0), (0.05, 1 / 128, 0.99), (0.2, 1 / 32, 0.99),
                                            (0.003, 1 / 256, 1.0)])
def test_beer_lambert_constant_field(orc, alpha, step, ert):
    """Constant field, shading off: each ray through the unit cube composites
    N = 1/step identical samples, A = 1 - (1 - alpha)^N, rgb = c A, and ERT
    stops at the first N with A > O_max."""
    ctrl = np.full((5, 5, 5), 0.7)
    col = (0.9, 0.4, 0.1)
    tf = _const_tf(col + (alpha,))
    res = orc.render(ctrl, 2, _ortho(), {"width": 6, "height": 5, "step": step, "max_opacity": ert,
                                         "tf": tf, "shading": 0})
    Nfull = round(1 / step)
    Ns = Nfull
    if ert < 1.0:
        k = math.floor(math.log(1 - ert) / math.log(1 - float(np.float32(alpha)))) + 1
        Ns = min(Nfull, k)
    a = float(np.float32(alpha))
    A = 1 - (1 - a) ** Ns
    exp = np.array([float(np.float32(c)) * A for c in col] + [A])
    # (t_exit - t_enter)/step is an exact integer here: every pixel carries the tie
    assert (res["nambig"] >= 1).all()
    np.testing.assert_allclose(res["rgba"], np.broadcast_to(exp, res["rgba"].shape), atol=1e-12)
    assert (res["nsamples"] == Ns).all()
    # tied early termination: an FP32 march may stop anywhere from the first
    # sample with A > O_max - 2e-4 to the first with A > O_max + 2e-4; the
    # tied sample count widens that by the other N
    Ak = 1 - (1 - a) ** np.arange(1, Nfull + 2)
    def first_above(th, N):
        idx = np.nonzero(Ak[:N] > th)[0]
        return int(idx[0]) + 1 if idx.size else N
    lo = min(first_above(ert - 2e-4, n) for n in (Nfull - 1, Nfull, Nfull + 1))
    hi = max(first_above(ert + 2e-4, n) for n in (Nfull - 1, Nfull, Nfull + 1))
    assert (res["ns_lo"] >= lo).all() and (res["ns_lo"] <= Ns).all()
    assert (res["ns_hi"] <= hi).all() and (res["ns_hi"] >= Ns).all()
    if ert < 1.0 and Ns < Nfull:
        assert (res["ns_lo"] == first_above(ert - 2e-4, Nfull)).all()
        assert (res["ns_hi"] == first_above(ert + 2e-4, Nfull)).all()


def test_opacity_correction_closed_form(orc):
    """alpha_s = 1 - (1 - alpha)^(step/ref): with ref = step/2 each sample
    counts twice, so A = 1 - (1 - alpha)^(2N)."""
    ctrl = np.full((4, 4, 4), 1.0)
    a = float(np.float32(0.02))
    tf = _const_tf((1.0, 1.0, 1.0, a))
    step = 1 / 64
    res = orc.render(ctrl, 3, _ortho(), {"width": 3, "height": 3, "step": step, "max_opacity": 1.0,
                                         "ref_step": step / 2, "tf": tf, "shading": 0})
    A = 1 - (1 - a) ** (2 * 64)
    np.testing.assert_allclose(res["rgba"][..., 3], A, atol=1e-12)


@pytest.mark.parametrize("grad", [(0.0, 0.0, 2.0), (1.0, -2.0, 0.5), (0.3, 0.0, -0.2)])
def test_shading_closed_form_linear_field(orc, grad):
    """Linear field (exact for p >= 1), constant TF colour and opacity, view
    along +z: every sample has the same shaded colour
    c (ka + kd |n.L|) + ks |n.L|^s, n = g/|g|, L = -z."""
    from paper_2204_11762_gb300.workloads import field_lattice
    g = np.array(grad)
    lin = lambda X, Y, Z: g[0] * X + g[1] * Y + g[2] * Z
    ctrl = field_lattice(lin, (5, 5, 5), 2, lo=0.0, hi=1.0)
    col = np.array([float(np.float32(c)) for c in (0.8, 0.5, 0.3)])
    a = float(np.float32(0.03))
    tf = _const_tf(tuple(col) + (a,))
    ka, kd, ks, sh = 0.1, 0.7, 0.2, 10.0
    res = orc.render(ctrl, 2, _ortho(), {"width": 4, "height": 4, "step": 1 / 32, "max_opacity": 1.0,
                                         "tf": tf, "shading": 1, "ka": ka, "kd": kd, "ks": ks,
                                         "shininess": sh})
    ndl = abs(g[2]) / np.linalg.norm(g)
    rgb = np.clip(col * (ka + kd * ndl) + ks * ndl ** sh, 0, 1)
    A = 1 - (1 - a) ** 32
    np.testing.assert_allclose(res["rgba"][..., :3], np.broadcast_to(rgb * A, (4, 4, 3)), atol=1e-12)
    np.testing.assert_allclose(res["rgba"][..., 3], A, atol=1e-12)


@pytest.mark.parametrize("grad", [(1.0, -2.0, 0.5), (0.3, 0.4, -0.2)])
def test_shading_closed_form_world_box(orc, grad):
    """The same linear field on a world box of extents (2, 0.5, 1): the world
    gradient is the parameter gradient divided by the extents per axis, so
    n = (g0/2, g1/0.5, g2/1) normalised, and with the view along +z every
    sample has c (ka + kd |n_z|) + ks |n_z|^s."""
    from paper_2204_11762_gb300.workloads import field_lattice
    g = np.array(grad)
    lin = lambda X, Y, Z: g[0] * X + g[1] * Y + g[2] * Z
    ctrl = field_lattice(lin, (5, 5, 5), 2, lo=0.0, hi=1.0)
    col = np.array([float(np.float32(c)) for c in (0.8, 0.5, 0.3)])
    a = float(np.float32(0.03))
    tf = _const_tf(tuple(col) + (a,))
    ka, kd, ks, sh = 0.1, 0.7, 0.2, 10.0
    box = ((0.0, 0.0, 0.0), (2.0, 0.5, 1.0))
    cam = {"kind": 0, "eye": (1.0, 0.25, -1.0), "center": (1.0, 0.25, 0.5), "up": (0.0, 1.0, 0.0),
           "ortho_height": 0.4}
    res = orc.render(ctrl, 2, cam, {"width": 4, "height": 4, "step": 1 / 32, "max_opacity": 1.0, "tf": tf,
                                    "shading": 1, "ka": ka, "kd": kd, "ks": ks, "shininess": sh},
                     box_min=box[0], box_max=box[1])
    gw = g / np.array([2.0, 0.5, 1.0])
    ndl = abs(gw[2]) / np.linalg.norm(gw)
    rgb = np.clip(col * (ka + kd * ndl) + ks * ndl ** sh, 0, 1)
    A = 1 - (1 - a) ** 32
    np.testing.assert_allclose(res["rgba"][..., :3], np.broadcast_to(rgb * A, (4, 4, 3)), atol=1e-12)


def test_perspective_rows_and_fov_closed_form(orc):
    """One image column from an eye at (1.5, 0.5, 0.7) looking along -x (up
    +z, vertical FOV 40 deg): row y's ray is (-1, 0, s_y) normalised with
    s_y = (1 - 2 (y + 1/2)/H) tan(20 deg), row 0 at the top.  It enters the
    box through the face x = 1 and leaves through the top face z = 1 after
    x-travel 0.3/s_y - 0.5 when that is below 1 (upward rays), else through
    the face x = 0; the chord is that x-travel times sqrt(1 + s_y^2), and the
    ray takes floor(chord/step) samples."""
    ctrl = np.full((4, 4, 4), 0.5)
    tf = _const_tf((1, 1, 1, 0.0))
    H, step = 8, 1 / 200
    cam = {"kind": 1, "eye": (1.5, 0.5, 0.7), "center": (0.5, 0.5, 0.7), "up": (0, 0, 1), "fovy_deg": 40.0}
    res = orc.render(ctrl, 3, cam, {"width": 1, "height": H, "step": step, "max_opacity": 1.0, "tf": tf,
                                    "shading": 0})
    for y in range(H):
        s = (1 - 2 * (y + 0.5) / H) * math.tan(math.radians(20.0))
        h = min(1.0, 0.3 / s - 0.5) if s > 0 else 1.0
        chord = h * math.sqrt(1 + s * s)
        r = chord / step
        assert abs(r - round(r)) > 1e-6  # no tied count in this set-up
        assert res["nsamples"][y, 0] == math.floor(r), (y, res["nsamples"][y, 0], r)
    assert res["nsamples"][0, 0] < res["nsamples"][H - 1, 0]  # the top row leaves through the top


def test_depth_ramp_brute_force_product(orc):
    """Field f = w (exact for p = 1), TF ramp in opacity and red: along +z the
    k-th sample sits at w_k = (k + 1/2) step, so the pixel is the explicit
    front-to-back sum over the N samples."""
    n = 2
    ctrl = np.zeros((n, n, n))
    ctrl[1] = 1.0  # value = w
    size = 65
    xs = np.linspace(0, 1, size)
    tf = np.stack([xs, 0.5 * np.ones(size), 1 - xs, 0.1 * xs], axis=1).astype(np.float32)
    step = 1 / 40
    res = orc.render(ctrl, 1, _ortho(), {"width": 3, "height": 2, "step": step, "max_opacity": 1.0,
                                         "tf": tf, "shading": 0})
    tfd = tf.astype(np.float64)
    C = np.zeros(3)
    A = 0.0
    for k in range(40):
        w = (k + 0.5) * step
        x = w * (size - 1)
        i = min(int(math.floor(x)), size - 2)
        fr = x - i
        rgba = tfd[i] + fr * (tfd[i + 1] - tfd[i])
        wgt = (1 - A) * rgba[3]
        C += wgt * rgba[:3]
        A += wgt
    np.testing.assert_allclose(res["rgba"][0, 0], list(C) + [A], atol=1e-12)
    np.testing.assert_allclose(res["rgba"], np.broadcast_to(res["rgba"][0, 0], res["rgba"].shape), atol=1e-12)


def test_perspective_centre_ray_chord(orc):
    """Eye at distance 2 on the +x axis through the box centre: the centre
    pixel's ray crosses the unit box along a chord of length 1, so it takes
    floor(1/step) samples; a pixel whose ray misses the box stays empty."""
    ctrl = np.full((4, 4, 4), 0.5)
    tf = _const_tf((1, 1, 1, 0.0))
    cam = {"kind": 1, "eye": (2.5, 0.5, 0.5), "center": (0.5, 0.5, 0.5), "up": (0, 0, 1), "fovy_deg": 60.0}
    res = orc.render(ctrl, 3, cam, {"width": 5, "height": 5, "step": 1 / 100, "max_opacity": 1.0, "tf": tf,
                                    "shading": 0})
    assert res["nsamples"][2, 2] in (99, 100)
    # a corner ray at 60 deg vertical FOV from distance 2 passes outside the box
    assert res["nsamples"][0, 0] == 0


def test_orthographic_footprint_closed_form(orc):
    """Orthographic view along +z of the field f = X + 2Y (exact for p = 2),
    image 8 x 4, view height 0.7: pixel (x, y) looks down the line
    X = 1/2 + ((x + 1/2)/8 - 1/2) 0.7 (8/4), Y = 1/2 + (1/2 - (y + 1/2)/4) 0.7,
    row 0 at the top.  A two-entry TF ramps red over [-1, 3] with a constant
    opacity, so a hit pixel is ((f + 1)/4 A, 0, 0, A) with A = 1 - (1 - a)^32;
    the columns x = 0 and x = 7 pass beside the box (X < 0 and X > 1) and stay
    empty."""
    from paper_2204_11762_gb300.workloads import field_lattice
    ctrl = field_lattice(lambda X, Y, Z: X + 2.0 * Y, (5, 5, 5), 2, lo=0.0, hi=1.0)
    a = _f32(0.05)
    tf = np.array([[0, 0, 0, a], [1, 0, 0, a]], dtype=np.float32)
    W, H, h = 8, 4, 0.7
    cam = {"kind": 0, "eye": (0.5, 0.5, -1.0), "center": (0.5, 0.5, 0.5), "up": (0.0, 1.0, 0.0),
           "ortho_height": h}
    res = orc.render(ctrl, 2, cam, {"width": W, "height": H, "step": 1 / 32, "max_opacity": 1.0, "tf": tf,
                                    "tf_lo": -1.0, "tf_hi": 3.0, "shading": 0})
    A = 1 - (1 - a) ** 32
    for y in range(H):
        for x in range(W):
            X = 0.5 + ((x + 0.5) / W - 0.5) * h * (W / H)
            Y = 0.5 + (0.5 - (y + 0.5) / H) * h
            if not 0.0 < X < 1.0:
                assert res["nsamples"][y, x] == 0 and (res["rgba"][y, x] == 0).all(), (x, y)
                continue
            assert res["nsamples"][y, x] == 32
            np.testing.assert_allclose(res["rgba"][y, x], [(X + 2 * Y + 1) / 4 * A, 0, 0, A], atol=1e-12)


@pytest.mark.parametrize("ert,n_exp", [(0.75, 3), (0.7, 2), (0.875, 4)])
def test_termination_is_strictly_above_o_max(orc, ert, n_exp):
    """Sample opacity 1/2: the cumulative opacity after k samples is
    1 - 2^-k exactly (0.5, 0.75, 0.875, ...), and the march stops at the first
    k with A > O_max, so an O_max met exactly takes one sample more."""
    ctrl = np.full((4, 4, 4), 0.5)
    tf = _const_tf((1.0, 1.0, 1.0, 0.5))
    res = orc.render(ctrl, 2, _ortho(), {"width": 3, "height": 3, "step": 1 / 16, "max_opacity": ert,
                                         "tf": tf, "shading": 0})
    A = 1 - 0.5 ** n_exp
    assert (res["nsamples"] == n_exp).all()
    np.testing.assert_array_equal(res["rgba"], np.full(res["rgba"].shape, A))


@pytest.mark.parametrize("ert,ns,lo,hi", [(0.99225, 8, 7, 8), (0.992, 7, 7, 8)])
def test_termination_tie_bracket_closed_form(orc, ert, ns, lo, hi):
    """Sample opacity 1/2, so A_k = 1 - 2^-k exactly (A_6 = 0.984375,
    A_7 = 0.9921875, A_8 = 0.99609375).  The exact march stops at the first
    k with A_k > O_max; the bracket an FP32 march may stop in runs from the
    first k with A_k > O_max - 2e-4 to the first with A_k > O_max + 2e-4.
    O_max = 0.99225 puts A_7 just below the threshold (stop 8, bracket 7-8);
    O_max = 0.992 puts it just above (stop 7, bracket 7-8)."""
    ctrl = np.full((4, 4, 4), 0.5)
    tf = _const_tf((1.0, 1.0, 1.0, 0.5))
    res = orc.render(ctrl, 2, _ortho(), {"width": 2, "height": 2, "step": 1 / 16, "max_opacity": ert,
                                         "tf": tf, "shading": 0})
    assert (res["nsamples"] == ns).all()
    assert (res["ns_lo"] == lo).all() and (res["ns_hi"] == hi).all()
    np.testing.assert_array_equal(res["rgba"], np.full(res["rgba"].shape, 1 - 0.5 ** ns))


def test_flat_field_takes_the_ambient_term_only(orc):
    """Zero field: every gradient is exactly zero, so a shaded sample keeps
    only the ambient part, c ka, and the pixel is c ka A."""
    ctrl = np.zeros((5, 5, 5))
    col = np.array([_f32(c) for c in (0.8, 0.5, 0.3)])
    a = _f32(0.04)
    tf = _const_tf(tuple(col) + (a,))
    ka, kd, ks = 0.25, 0.6, 0.3
    res = orc.render(ctrl, 2, _ortho(), {"width": 3, "height": 3, "step": 1 / 32, "max_opacity": 1.0, "tf": tf,
                                         "shading": 1, "ka": ka, "kd": kd, "ks": ks, "shininess": 8.0})
    A = 1 - (1 - a) ** 32
    np.testing.assert_allclose(res["rgba"][..., :3], np.broadcast_to(col * ka * A, (3, 3, 3)), atol=1e-12)
    np.testing.assert_allclose(res["rgba"][..., 3], A, atol=1e-12)


@pytest.mark.parametrize("p,n,shading", [(1, 4, 0), (2, 5, 1), (3, 6, 1)])
def test_render_span_mode_equals_brute_mode(orc, p, n, shading):
    rng = np.random.default_rng(53 + p)
    ctrl = rng.uniform(0, 1, size=(n, n, n))
    from paper_2204_11762_gb300.workloads import transfer_function
    tf = transfer_function(rng, 32)
    cam = {"kind": 1, "eye": (1.9, 1.4, 1.7), "center": (0.5, 0.5, 0.5), "up": (0, 0, 1), "fovy_deg": 50.0}
    prm = {"width": 8, "height": 8, "step": 1 / 48, "max_opacity": 0.99, "tf": tf, "shading": shading}
    a = orc.render(ctrl, p, cam, prm)
    b = orc.render(ctrl, p, cam, prm, brute=True)
    np.testing.assert_allclose(a["rgba"], b["rgba"], atol=1e-12)
    np.testing.assert_array_equal(a["nsamples"], b["nsamples"])


def test_render_row_subset_and_threads(orc):
    from paper_2204_11762_gb300.workloads import transfer_function
    rng = np.random.default_rng(59)
    ctrl = rng.uniform(0, 1, size=(6, 6, 6))
    tf = transfer_function(rng, 16)
    cam = {"kind": 1, "eye": (2.0, 1.0, 1.5), "center": (0.5, 0.5, 0.5), "up": (0, 0, 1), "fovy_deg": 60.0}
    prm = {"width": 9, "height": 7, "step": 1 / 32, "tf": tf, "shading": 1}
    full = orc.render(ctrl, 3, cam, prm, threads=1)
    sub = orc.render(ctrl, 3, cam, prm, threads=3, row_step=3)
    np.testing.assert_array_equal(full["rgba"][::3], sub["rgba"][::3])
    assert (sub["rgba"][1::3] == 0).all()
