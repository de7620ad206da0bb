"""Pins for the oracle on general (non-uniform) clamped knots, the adaptive
knots of an MFA fit (Sec. 2.3).  Each test checks the span-mode oracle
against something other than itself: scipy's de Boor evaluation, the raw
recursive definition over the whole knot vector, Marsden's identity, central
differences, and the uniform special case."""
import math
from itertools import combinations

import numpy as np
import pytest
from scipy.interpolate import BSpline

from paper_2204_11762_gb300.workloads import graded_knots, transfer_function

CASES = [(2, 1), (7, 1), (5, 2), (11, 2), (4, 3), (9, 3), (20, 3), (8, 4), (15, 4), (9, 5), (18, 5)]


def _knots(seed, n, p):
    return graded_knots(np.random.default_rng(seed), n, p).astype(np.float64)


@pytest.mark.parametrize("n,p", CASES)
def test_general_knots_match_scipy_bspline(orc, n, p):
    t = _knots(100 + n + p, n, p)
    rng = np.random.default_rng(5)
    us = np.concatenate([rng.uniform(0, 1, 300), t[p:n + 1]])
    D = BSpline.design_matrix(us, t, p).toarray()
    for row, u in zip(D, us):
        s, N, dN = orc.basis_ders(n, p, u, t)
        assert t[s] <= u and (u < t[s + 1] or (u == 1.0 and s == n - 1))
        full = np.zeros(n)
        full[s - p:s + 1] = N
        np.testing.assert_allclose(full, row, atol=1e-13)
    hmin = np.diff(t[p:n + 1]).min()
    for i in range(n):
        c = np.zeros(n)
        c[i] = 1.0
        dspl = BSpline(t, c, p).derivative()
        for u in us[:40]:
            s, N, dN = orc.basis_ders(n, p, u, t)
            got = dN[i - (s - p)] if s - p <= i <= s else 0.0
            assert abs(got - float(dspl(u))) < 1e-10 / hmin


@pytest.mark.parametrize("n,p", CASES)
def test_general_knots_span_mode_equals_brute_mode_1d(orc, n, p):
    t = _knots(200 + n + p, n, p)
    rng = np.random.default_rng(9)
    for u in list(rng.uniform(0, 1, 100)) + list(t[p:n + 1]):
        s, N, dN = orc.basis_ders(n, p, u, t)
        Nb, dNb = orc.basis_brute(n, p, u, t)
        full = np.zeros(n)
        dfull = np.zeros(n)
        full[s - p:s + 1] = N
        dfull[s - p:s + 1] = dN
        np.testing.assert_allclose(full, Nb, atol=1e-14)
        np.testing.assert_allclose(dfull, dNb, atol=1e-11 * n)


def _knot_set(seed, n, p):
    return [_knots(seed + d, n[d], p) for d in range(3)]


@pytest.mark.parametrize("p,n", [(1, (3, 5, 4)), (2, (5, 4, 6)), (3, (6, 7, 5)), (4, (7, 6, 8)), (5, (8, 7, 6))])
def test_general_knots_tensor_span_mode_equals_brute_mode(orc, p, n):
    rng = np.random.default_rng(300 + p)
    ctrl = rng.normal(size=(n[2], n[1], n[0]))
    kv = _knot_set(310 + p, n, p)
    pts = rng.uniform(0, 1, size=(60, 3)).astype(np.float32)
    pts[0] = [1, 1, 1]
    pts[1] = [0, 0, 0]
    pts[2] = [np.float32(kv[0][p + 1]), np.float32(kv[1][p + 1]), np.float32(kv[2][p + 1])]
    a, spans = orc.eval_points(ctrl, p, pts, knot_vectors=kv)
    b = orc.eval_points(ctrl, p, pts, brute=True, knot_vectors=kv)
    np.testing.assert_allclose(a, b, atol=1e-11)
    for d in range(3):  # spans satisfy t_s <= u < t_{s+1} (u = 1: last span)
        u = pts[:, d].astype(np.float64)
        s = spans[:, d]
        assert np.all(kv[d][s] <= u)
        assert np.all((u < kv[d][s + 1]) | ((u == 1.0) & (s == n[d] - 1)))


def _marsden(t, p, n, r):
    out = np.zeros(n)
    for i in range(n):
        ks = t[i + 1:i + p + 1]
        out[i] = sum(np.prod(c) for c in combinations(ks, r)) / math.comb(p, r) if r else 1.0
    return out


@pytest.mark.parametrize("p,n", [(1, 6), (2, 7), (3, 10), (4, 9), (5, 11)])
def test_general_knots_polynomial_reproduction_marsden(orc, p, n):
    """Marsden's identity holds for any knot vector: monomials of degree <= p
    per axis come out exactly, value and partial derivatives."""
    kv = _knot_set(400 + p, (n, n, n), p)
    rng = np.random.default_rng(41)
    pts = rng.uniform(0, 1, size=(50, 3)).astype(np.float32)
    x = pts.astype(np.float64)
    for (a, b, c) in [(p, 0, 0), (0, p, 0), (0, 0, p), (1, 1, 1), (p, p - 1, 1), (p, p, p)]:
        ca, cb, cc = _marsden(kv[0], p, n, a), _marsden(kv[1], p, n, b), _marsden(kv[2], p, n, c)
        ctrl = cc[:, None, None] * cb[None, :, None] * ca[None, None, :]
        out, _ = orc.eval_points(ctrl, p, pts, knot_vectors=kv)
        u, v, w = x[:, 0], x[:, 1], x[:, 2]
        np.testing.assert_allclose(out[:, 0], u ** a * v ** b * w ** c, atol=1e-12)
        np.testing.assert_allclose(out[:, 1], a * u ** max(a - 1, 0) * v ** b * w ** c, atol=1e-10)
        np.testing.assert_allclose(out[:, 2], b * u ** a * v ** max(b - 1, 0) * w ** c, atol=1e-10)
        np.testing.assert_allclose(out[:, 3], c * u ** a * v ** b * w ** max(c - 1, 0), atol=1e-10)


def test_general_knots_gradient_central_differences(orc):
    rng = np.random.default_rng(47)
    p, n = 3, (11, 9, 12)
    ctrl = rng.normal(size=(n[2], n[1], n[0]))
    kv = _knot_set(470, n, p)
    h = 2.0 ** -18
    base = (np.round(rng.uniform(0.1, 0.9, size=(40, 3)) * 2 ** 20) / 2 ** 20).astype(np.float32)
    out, _ = orc.eval_points(ctrl, p, base, knot_vectors=kv)
    for d in range(3):
        e = np.zeros(3, dtype=np.float32)
        e[d] = h
        fp, _ = orc.eval_points(ctrl, p, base + e, knot_vectors=kv)
        fm, _ = orc.eval_points(ctrl, p, base - e, knot_vectors=kv)
        fd = (fp[:, 0] - fm[:, 0]) / (2 * h)
        scale = np.abs(ctrl).max() / np.diff(kv[d][p:n[d] + 1]).min()
        assert np.max(np.abs(fd - out[:, 1 + d])) < 1e-5 * scale


def test_explicit_uniform_knots_equal_the_default(orc):
    p, n = 3, (9, 8, 10)
    rng = np.random.default_rng(53)
    ctrl = rng.normal(size=(n[2], n[1], n[0]))
    kv = [np.concatenate([np.zeros(p), np.arange(n[d] - p + 1) / (n[d] - p), np.ones(p)]) for d in range(3)]
    pts = rng.uniform(0, 1, size=(200, 3)).astype(np.float32)
    a, sa = orc.eval_points(ctrl, p, pts)
    b, sb = orc.eval_points(ctrl, p, pts, knot_vectors=kv)
    np.testing.assert_allclose(a, b, atol=1e-13)
    np.testing.assert_array_equal(sa, sb)


def test_invalid_knot_vectors_are_refused(orc):
    p, n = 2, (6, 6, 6)
    ctrl = np.zeros((6, 6, 6))
    pts = np.zeros((1, 3), dtype=np.float32)
    good = np.array([0, 0, 0, 0.3, 0.5, 0.7, 1, 1, 1], dtype=np.float64)
    for bad in (good * 0.5, good[::-1].copy(), np.where(good == 0.5, 0.2, good)):
        with pytest.raises(ValueError):
            orc.eval_points(ctrl, p, pts, knot_vectors=[bad, None, None])


@pytest.mark.parametrize("p,n,shading", [(1, 5, 0), (2, 6, 1), (3, 7, 1)])
def test_general_knots_render_span_mode_equals_brute_mode(orc, p, n, shading):
    rng = np.random.default_rng(61 + p)
    ctrl = rng.uniform(0, 1, size=(n, n, n))
    kv = _knot_set(610 + p, (n, n, n), p)
    tf = transfer_function(rng, 32)
    cam = {"kind": 1, "eye": (1.9, 1.4, 1.7), "center": (0.5, 0.5, 0.5), "up": (0, 0, 1), "fovy_deg": 50.0}
    prm = {"width": 8, "height": 8, "step": 1 / 48, "max_opacity": 0.99, "tf": tf, "shading": shading}
    a = orc.render(ctrl, p, cam, prm, knot_vectors=kv)
    b = orc.render(ctrl, p, cam, prm, brute=True, knot_vectors=kv)
    np.testing.assert_allclose(a["rgba"], b["rgba"], atol=1e-12)
    np.testing.assert_array_equal(a["nsamples"], b["nsamples"])
