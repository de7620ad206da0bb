"""Pins for the oracle's second derivatives (the higher-order query of
Sec. 3.1; Sec. 2: analytic derivatives up to the degree): scipy's BSpline
derivatives, the first-derivative routines, Marsden's identity for
polynomials, and central differences of the gradient (plain and rational)."""
import math
from itertools import combinations

import numpy as np
import pytest
from scipy.interpolate import BSpline

from paper_2204_11762_gb300.workloads import graded_knots


@pytest.mark.parametrize("n,p,general", [(5, 2, False), (9, 3, False), (8, 3, True), (10, 4, True), (11, 5, False)])
def test_second_derivative_of_the_basis_matches_scipy(orc, n, p, general):
    t = graded_knots(np.random.default_rng(n), n, p).astype(np.float64) if general else orc.knots(n, p)
    us = np.random.default_rng(3).uniform(0, 1, 40)
    for i in range(n):
        c = np.zeros(n)
        c[i] = 1.0
        d1, d2 = BSpline(t, c, p).derivative(1), BSpline(t, c, p).derivative(2)
        for u in us:
            assert abs(orc.basis_dk(n, p, 1, u, t)[i] - float(d1(u))) < 1e-9 * n
            assert abs(orc.basis_dk(n, p, 2, u, t)[i] - float(d2(u))) < 1e-7 * n * n
    # order 0 and 1 agree with the existing routines
    for u in us[:10]:
        N, dN = orc.basis_brute(n, p, u, t)
        np.testing.assert_allclose(orc.basis_dk(n, p, 0, u, t), N, atol=1e-15)
        np.testing.assert_allclose(orc.basis_dk(n, p, 1, u, t), dN, atol=1e-12 * n)


def _marsden(t, p, n, r):
    out = np.zeros(n)
    for i in range(n):
        ks = t[i + 1:i + p + 1]
        out[i] = sum(np.prod(c) for c in combinations(ks, r)) / math.comb(p, r) if r else 1.0
    return out


@pytest.mark.parametrize("p,n", [(2, 6), (3, 8), (4, 9), (5, 10)])
def test_hessian_of_monomials_is_exact(orc, p, n):
    t = orc.knots(n, p)
    rng = np.random.default_rng(17)
    pts = rng.uniform(0, 1, size=(30, 3)).astype(np.float32)
    x = pts.astype(np.float64)
    a, b, c = p, p - 1, 2
    ctrl = _marsden(t, p, n, c)[:, None, None] * _marsden(t, p, n, b)[None, :, None] * _marsden(t, p, n, a)[None, None, :]
    out = orc.eval_hessian(ctrl, p, pts)
    u, v, w = x[:, 0], x[:, 1], x[:, 2]
    D = lambda k, e, z: (math.perm(e, k) * z ** (e - k)) if e >= k else 0.0 * z
    want = [D(0, a, u) * D(0, b, v) * D(0, c, w), D(1, a, u) * D(0, b, v) * D(0, c, w),
            D(0, a, u) * D(1, b, v) * D(0, c, w), D(0, a, u) * D(0, b, v) * D(1, c, w),
            D(2, a, u) * D(0, b, v) * D(0, c, w), D(0, a, u) * D(2, b, v) * D(0, c, w),
            D(0, a, u) * D(0, b, v) * D(2, c, w), D(1, a, u) * D(1, b, v) * D(0, c, w),
            D(1, a, u) * D(0, b, v) * D(1, c, w), D(0, a, u) * D(1, b, v) * D(1, c, w)]
    for o in range(10):
        np.testing.assert_allclose(out[:, o], want[o], atol=1e-9)


@pytest.mark.parametrize("rational,general", [(False, False), (True, False), (False, True), (True, True)])
def test_hessian_central_differences_of_the_gradient(orc, rational, general):
    rng = np.random.default_rng(31 + rational + 2 * general)
    p, n = 3, (10, 9, 11)
    ctrl = rng.normal(size=(n[2], n[1], n[0]))
    w = rng.uniform(0.3, 3.0, size=ctrl.shape) if rational else None
    kv = [graded_knots(rng, n[d], p).astype(np.float64) for d in range(3)] if general else None
    base = (np.round(rng.uniform(0.15, 0.85, size=(25, 3)) * 2 ** 20) / 2 ** 20).astype(np.float32)
    H = orc.eval_hessian(ctrl, p, base, weights=w, knot_vectors=kv)
    g0, _ = orc.eval_points(ctrl, p, base, weights=w, knot_vectors=kv)
    np.testing.assert_allclose(H[:, :4], g0, atol=1e-11)  # value and gradient agree with the span-mode query
    h = 2.0 ** -16
    pair = {(0, 0): 4, (1, 1): 5, (2, 2): 6, (0, 1): 7, (0, 2): 8, (1, 2): 9}
    scale = np.abs(H[:, 4:]).max()
    for d in range(3):
        e = np.zeros(3, dtype=np.float32)
        e[d] = h
        gp, _ = orc.eval_points(ctrl, p, base + e, weights=w, knot_vectors=kv)
        gm, _ = orc.eval_points(ctrl, p, base - e, weights=w, knot_vectors=kv)
        fd = (gp[:, 1:] - gm[:, 1:]) / (2 * h)  # d/dx_d of (f_u, f_v, f_w)
        for j in range(3):
            col = pair[tuple(sorted((d, j)))]
            assert np.max(np.abs(fd[:, j] - H[:, col])) < 1e-5 * scale
