"""Pins for the oracle on rational models (NURBS: positive weights per
control point, Sec. 2.3), each against something other than the span-mode
code: the non-rational model (equal weights), projective invariance, a conic
that a rational quadratic reproduces exactly (the quarter circle), the raw
recursive definition over the whole lattice, and central differences."""
import math

import numpy as np
import pytest

from paper_2204_11762_gb300.workloads import graded_knots, transfer_function


def _weights(rng, shape, lo=0.3, hi=3.0):
    return rng.uniform(lo, hi, size=shape)


@pytest.mark.parametrize("p,n", [(1, (4, 5, 3)), (2, (6, 5, 7)), (3, (8, 9, 7)), (4, (7, 8, 6)), (5, (9, 8, 7))])
def test_equal_weights_give_the_plain_model(orc, p, n):
    rng = np.random.default_rng(500 + p)
    ctrl = rng.normal(size=(n[2], n[1], n[0]))
    pts = rng.uniform(0, 1, size=(300, 3)).astype(np.float32)
    plain, sp = orc.eval_points(ctrl, p, pts)
    rat, sr = orc.eval_points(ctrl, p, pts, weights=np.full(ctrl.shape, 2.5))
    np.testing.assert_allclose(rat, plain, atol=1e-12)
    np.testing.assert_array_equal(sp, sr)


def test_scaling_all_weights_changes_nothing(orc):
    rng = np.random.default_rng(51)
    p, n = 3, (9, 8, 10)
    ctrl = rng.normal(size=(n[2], n[1], n[0]))
    w = _weights(rng, ctrl.shape)
    pts = rng.uniform(0, 1, size=(300, 3)).astype(np.float32)
    a, _ = orc.eval_points(ctrl, p, pts, weights=w)
    b, _ = orc.eval_points(ctrl, p, pts, weights=3.7 * w)
    np.testing.assert_allclose(a, b, atol=1e-12)


def test_quarter_circle_is_exact(orc):
    """Degree 2, one span, control points (1,0), (1,1), (0,1) with weights
    1, cos(45 deg), 1: the rational quadratic traces the unit quarter circle,
    so x^2 + y^2 = 1 and the tangent is orthogonal to the radius."""
    p = 2
    wi = np.array([1.0, math.sqrt(0.5), 1.0])
    w = np.broadcast_to(wi[None, None, :], (3, 3, 3)).copy()
    X = np.broadcast_to(np.array([1.0, 1.0, 0.0])[None, None, :], (3, 3, 3)).copy()
    Y = np.broadcast_to(np.array([0.0, 1.0, 1.0])[None, None, :], (3, 3, 3)).copy()
    rng = np.random.default_rng(57)
    pts = rng.uniform(0, 1, size=(400, 3)).astype(np.float32)
    pts[:2] = [[0, 0.3, 0.6], [1, 0.2, 0.9]]
    x, _ = orc.eval_points(X, p, pts, weights=w)
    y, _ = orc.eval_points(Y, p, pts, weights=w)
    np.testing.assert_allclose(x[:, 0] ** 2 + y[:, 0] ** 2, 1.0, atol=1e-13)
    np.testing.assert_allclose(x[:, 0] * x[:, 1] + y[:, 0] * y[:, 1], 0.0, atol=1e-12)
    np.testing.assert_allclose(x[:, 2:], 0.0, atol=1e-13)  # constant along v and w
    np.testing.assert_allclose(x[:2, 0], [1.0, 0.0], atol=1e-15)  # end points


@pytest.mark.parametrize("p,n,general", [(1, (3, 4, 3), False), (2, (5, 4, 6), True), (3, (6, 5, 4), False),
                                         (3, (5, 6, 7), True), (4, (6, 7, 5), False)])
def test_rational_span_mode_equals_brute_mode(orc, p, n, general):
    rng = np.random.default_rng(600 + p)
    ctrl = rng.normal(size=(n[2], n[1], n[0]))
    w = _weights(rng, ctrl.shape)
    kv = [graded_knots(rng, n[d], p).astype(np.float64) for d in range(3)] if general else None
    pts = rng.uniform(0, 1, size=(60, 3)).astype(np.float32)
    pts[0] = [1, 1, 1]
    a, _ = orc.eval_points(ctrl, p, pts, weights=w, knot_vectors=kv)
    b = orc.eval_points(ctrl, p, pts, brute=True, weights=w, knot_vectors=kv)
    np.testing.assert_allclose(a, b, atol=1e-11)


def test_rational_gradient_central_differences(orc):
    rng = np.random.default_rng(67)
    p, n = 3, (10, 9, 11)
    ctrl = rng.normal(size=(n[2], n[1], n[0]))
    w = _weights(rng, ctrl.shape)
    h = 2.0 ** -18
    base = (np.round(rng.uniform(0.1, 0.9, size=(40, 3)) * 2 ** 20) / 2 ** 20).astype(np.float32)
    out, _ = orc.eval_points(ctrl, p, base, weights=w)
    for d in range(3):
        e = np.zeros(3, dtype=np.float32)
        e[d] = h
        fp, _ = orc.eval_points(ctrl, p, base + e, weights=w)
        fm, _ = orc.eval_points(ctrl, p, base - e, weights=w)
        fd = (fp[:, 0] - fm[:, 0]) / (2 * h)
        assert np.max(np.abs(fd - out[:, 1 + d])) < 1e-5 * np.abs(ctrl).max() * max(n) * 10


def test_invalid_weights_are_refused(orc):
    ctrl = np.zeros((4, 4, 4))
    pts = np.zeros((1, 3), dtype=np.float32)
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        w = np.ones(ctrl.shape)
        w[1, 2, 3] = bad
        with pytest.raises(ValueError):
            orc.eval_points(ctrl, 2, pts, weights=w)


@pytest.mark.parametrize("p,n,shading", [(2, 5, 1), (3, 6, 0)])
def test_rational_render_span_mode_equals_brute_mode(orc, p, n, shading):
    rng = np.random.default_rng(71 + p)
    ctrl = rng.uniform(0, 1, size=(n, n, n))
    w = _weights(rng, ctrl.shape)
    tf = transfer_function(rng, 32)
    cam = {"kind": 1, "eye": (1.9, 1.4, 1.7), "center": (0.5, 0.5, 0.5), "up": (0, 0, 1), "fovy_deg": 50.0}
    prm = {"width": 8, "height": 8, "step": 1 / 48, "max_opacity": 0.99, "tf": tf, "shading": shading}
    a = orc.render(ctrl, p, cam, prm, weights=w)
    b = orc.render(ctrl, p, cam, prm, brute=True, weights=w)
    np.testing.assert_allclose(a["rgba"], b["rgba"], atol=1e-12)
    np.testing.assert_array_equal(a["nsamples"], b["nsamples"])
