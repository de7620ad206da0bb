"""GPU parity for rational models (NURBS weights, Sec. 2.3) through the C ABI:
f = A / W with A = sum w P N N N and W = sum w N N N, gradient by the
quotient rule.  The library stores w P and w (16-bit: each with its own
own scale); the oracle evaluates the same stored lattices, i.e. weights
W' and control points Q' / W'."""
import numpy as np
import pytest

from _parity import assert_eval_parity, assert_render_parity, dequantize

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def ctx(torch_cuda):
    from paper_2204_11762_gb300 import mfadvr
    c = mfadvr.Context(0)
    yield c
    c.close()


def _stored(ctrl, w, storage):
    """(control points, weights) of the rational model the library holds."""
    q = (w.astype(np.float64) * ctrl.astype(np.float64)).astype(np.float32)
    qd, wd = dequantize(q, storage), dequantize(w, storage)
    return qd / wd, wd


def _eval(ctx, torch, mid, pts):
    dev = torch.device("cuda:0")
    k = pts.shape[0]
    d_pts = torch.from_numpy(pts).to(dev)
    d_out = torch.full((k, 4), float("nan"), device=dev)
    d_sp = torch.full((k, 3), -1, dtype=torch.int32, device=dev)
    ctx.eval_points(mid, d_pts, k, d_out, d_sp)
    torch.cuda.synchronize()
    return d_out.cpu().numpy(), d_sp.cpu().numpy()


@pytest.mark.parametrize("p,n,storage,general", [(1, (7, 9, 8), "f32", False), (2, (11, 9, 13), "f32", False),
                                                 (3, (17, 14, 19), "f32", False), (3, (13, 15, 12), "f16", False),
                                                 (3, (12, 14, 16), "f32", True), (4, (12, 11, 13), "bf16", False),
                                                 (5, (11, 12, 10), "f32", True)])
def test_eval_rational(ctx, torch_cuda, orc, p, n, storage, general):
    from paper_2204_11762_gb300 import mfadvr, workloads
    rng = np.random.default_rng(5000 + p * 10 + general)
    ctrl = rng.normal(size=(n[2], n[1], n[0])).astype(np.float32)
    w = rng.uniform(0.3, 3.0, size=ctrl.shape).astype(np.float32)
    kv = [workloads.graded_knots(rng, n[d], p) for d in range(3)] if general else None
    pts = rng.uniform(0, 1, size=(3000, 3)).astype(np.float32)
    pts[:4] = [[0, 0, 0], [1, 1, 1], [0.5, 1, 0], [1, 0, 0.25]]
    mid = ctx.load_model(ctrl, p, storage=storage, knots=kv, weights=w)
    got, sp = _eval(ctx, torch_cuda, mid, pts)
    c_eff, w_eff = _stored(ctrl, w, storage)
    ref, ref_sp = orc.eval_points(c_eff, p, pts, weights=w_eff,
                                  knot_vectors=[t.astype(np.float64) for t in kv] if kv else None)
    # gradients of a rational model are normalised by max|P| / (smallest span width)
    hmin = min(float(np.diff(kv[d][p:n[d] + 1]).min()) for d in range(3)) if kv else 1.0 / max(x - p for x in n)
    mm = int(round(1.0 / hmin))
    assert_eval_parity(got, ref, c_eff, (mm + p,) * 3, p, sp, ref_sp)
    np.testing.assert_array_equal(ctx.query_points_host(mid, pts, mfadvr.QUERY_VALUE), got[:, 0])
    np.testing.assert_array_equal(ctx.query_points_host(mid, pts, mfadvr.QUERY_GRADIENT), got[:, 1:])
    ctx.unload_model(mid)


def test_equal_weights_match_the_plain_model(ctx, torch_cuda):
    rng = np.random.default_rng(51)
    ctrl = rng.normal(size=(14, 12, 13)).astype(np.float32)
    pts = rng.uniform(0, 1, size=(2000, 3)).astype(np.float32)
    a = ctx.load_model(ctrl, 3)
    b = ctx.load_model(ctrl, 3, weights=np.full(ctrl.shape, 2.0, np.float32))
    ga, _ = _eval(ctx, torch_cuda, a, pts)
    gb, _ = _eval(ctx, torch_cuda, b, pts)
    np.testing.assert_allclose(gb, ga, atol=1e-5 * np.abs(ctrl).max() * 10)
    ctx.unload_model(a)
    ctx.unload_model(b)


def test_bad_weights_rejected(ctx, torch_cuda):
    from paper_2204_11762_gb300 import mfadvr
    ctrl = np.ones((5, 5, 5), np.float32)
    for bad in (0.0, -2.0, float("nan"), float("inf")):
        w = np.ones_like(ctrl)
        w[2, 1, 3] = bad
        with pytest.raises(mfadvr.MfadvrError) as e:
            ctx.load_model(ctrl, 2, weights=w)
        assert e.value.status == mfadvr.EINVAL


@pytest.mark.parametrize("form", [0, 1])  # AUTO (span polynomials for FP32 up to degree 3), B-spline
@pytest.mark.parametrize("p,storage,shading,general", [(2, "f32", 1, False), (3, "f32", 1, False),
                                                       (3, "f32", 0, True), (3, "bf16", 1, False),
                                                       (4, "f32", 1, True), (5, "f16", 0, False),
                                                       (3, "f32", 1, True), (1, "f32", 1, False)])
def test_render_rational(ctx, torch_cuda, orc, p, storage, shading, general, form):
    from paper_2204_11762_gb300 import workloads
    torch = torch_cuda
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(6000 + p * 7 + shading + 2 * general)
    n = (p + 12, p + 10, p + 13)
    ctrl = workloads.gaussian_sum_lattice(n, p, rng)
    w = rng.uniform(0.5, 2.0, size=ctrl.shape).astype(np.float32)
    kv = [workloads.graded_knots(rng, n[d], p) for d in range(3)] if general else None
    tf = workloads.transfer_function(rng, 128)
    cam = {"kind": 1, "eye": (1.8, -1.3, 1.5), "center": (0.5, 0.5, 0.5), "up": (0, 0, 1), "fovy_deg": 50.0}
    prm = {"width": 48, "height": 40, "step": 1 / 256, "max_opacity": 0.99, "ref_step": 1 / 16, "shading": shading}
    mid = ctx.load_model(ctrl, p, storage=storage, knots=kv, weights=w, render_form=form)
    img = torch.full((40, 48, 4), float("nan"), device=dev)
    ns = torch.full((40, 48), -1, dtype=torch.int32, device=dev)
    ctx.render(mid, cam, prm, torch.from_numpy(tf).to(dev), tf.shape[0], img, ns)
    torch.cuda.synchronize()
    c_eff, w_eff = _stored(ctrl, w, storage)
    ref = orc.render(c_eff, p, cam, dict(prm, tf=tf, tf_lo=float(ctrl.min()), tf_hi=float(ctrl.max())),
                     weights=w_eff, knot_vectors=[t.astype(np.float64) for t in kv] if kv else None)
    assert_render_parity(img.cpu().numpy(), ns.cpu().numpy(), ref)
    ctx.unload_model(mid)


def test_batch_mixes_rational_and_plain(torch_cuda):
    from paper_2204_11762_gb300 import mfadvr, workloads
    torch = torch_cuda
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(81)
    with mfadvr.Context(0) as ctx:
        jobs = []
        for i, (p, n, st) in enumerate([(3, (18, 20, 16), "f32"), (3, (17, 15, 19), "f32"), (2, (14, 13, 15), "f16"),
                                        (4, (13, 14, 15), "f32")]):
            ctrl = workloads.gaussian_sum_lattice(n, p, rng)
            w = rng.uniform(0.5, 2.0, size=ctrl.shape).astype(np.float32) if i % 2 == 0 else None
            mid = ctx.load_model(ctrl, p, storage=st, weights=w)
            W, H = 40 + 8 * i, 32 + 4 * i
            tf = workloads.transfer_function(rng, 64)
            jobs.append({"model_id": mid, "camera": workloads.sphere_camera(rng),
                         "params": {"width": W, "height": H, "step": 1 / 256, "max_opacity": 0.99, "shading": 1},
                         "tf_dev": torch.from_numpy(tf).to(dev), "tf_size": tf.shape[0],
                         "rgba_dev": torch.full((H, W, 4), float("nan"), device=dev),
                         "nsamples_dev": torch.full((H, W), -1, dtype=torch.int32, device=dev)})
        ctx.render_batch(jobs)
        torch.cuda.synchronize()
        batch = [(j["rgba_dev"].cpu().numpy(), j["nsamples_dev"].cpu().numpy()) for j in jobs]
        for j, (img, ns) in zip(jobs, batch):
            ctx.render(j["model_id"], j["camera"], j["params"], j["tf_dev"], j["tf_size"], j["rgba_dev"],
                       j["nsamples_dev"])
            torch.cuda.synchronize()
            np.testing.assert_array_equal(img, j["rgba_dev"].cpu().numpy())
            np.testing.assert_array_equal(ns, j["nsamples_dev"].cpu().numpy())
