"""GPU parity on general (non-uniform) clamped knots (Sec. 2.3: the knots an
adaptive MFA fit places), through the C ABI: exact spans (binary search over
FP32 breakpoints on both sides), values within 1e-5 of max|P|, gradients
within 1e-4 of max|P| / (smallest span width), pixels within 2e-3."""
import numpy as np
import pytest

from _parity import assert_render_parity, dequantize

pytestmark = pytest.mark.gpu

VALUE_RTOL, GRAD_RTOL = 1e-5, 1e-4


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


def _uniform_f32(n, p):
    """The knots the library uses for an axis given as None: j/m rounded to FP32."""
    m = n - p
    inner = np.array([np.float32(j / m) for j in range(1, m)], dtype=np.float32)
    return np.concatenate([np.zeros(p + 1, np.float32), inner, np.ones(p + 1, np.float32)])


def _knots(seed, n, p, axes=(0, 1, 2)):
    from paper_2204_11762_gb300.workloads import graded_knots
    rng = np.random.default_rng(seed)
    given = [graded_knots(rng, n[d], p) if d in axes else None for d in range(3)]
    used = [g if g is not None else _uniform_f32(n[d], p) for d, g in enumerate(given)]
    return given, [u.astype(np.float64) for u in used]


def _edge_points(kv, p, n):
    pts = []
    for d in range(3):
        for b in np.float32(kv[d][p:n[d] + 1]):
            for u in (b, np.nextafter(b, np.float32(2)), np.nextafter(b, np.float32(-1))):
                q = np.full(3, 0.41, dtype=np.float32)
                q[d] = u
                pts.append(q)
    pts += [np.zeros(3), np.ones(3), [-0.5, 1.5, 0.25]]
    return np.asarray(pts, dtype=np.float32)


def _check(got, sp, ref, ref_sp, ctrl, kv, p, n):
    bad = np.nonzero((sp != ref_sp).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} span mismatches, first {sp[bad[:3]]} vs {ref_sp[bad[:3]]}"
    pabs = float(np.abs(ctrl).max()) or 1.0
    hmin = min(float(np.diff(kv[d][p:n[d] + 1]).min()) for d in range(3))
    verr = np.abs(got[:, 0] - ref[:, 0]) / np.maximum(np.abs(ref[:, 0]), pabs)
    gerr = np.abs(got[:, 1:] - ref[:, 1:]).max(axis=1) / np.maximum(np.linalg.norm(ref[:, 1:], axis=1), pabs / hmin)
    assert verr.max() <= VALUE_RTOL, f"value error {verr.max():.3e}"
    assert gerr.max() <= GRAD_RTOL, f"gradient error {gerr.max():.3e}"


def _eval(ctx, torch, mid, pts, query=3):
    dev = torch.device("cuda:0")
    k = pts.shape[0]
    d_pts = torch.from_numpy(pts).to(dev)
    d_out = torch.full((k, 4), float("nan"), device=dev)
    d_sp = torch.full((k, 3), -1, dtype=torch.int32, device=dev)
    ctx.eval_points(mid, d_pts, k, d_out, d_sp)
    torch.cuda.synchronize()
    return d_out.cpu().numpy(), d_sp.cpu().numpy()


@pytest.mark.parametrize("p,n,storage,axes", [(1, (9, 12, 7), "f32", (0, 1, 2)), (2, (13, 8, 17), "f32", (0, 2)),
                                              (3, (21, 18, 25), "f32", (0, 1, 2)), (3, (15, 19, 11), "f16", (1,)),
                                              (4, (17, 14, 12), "f32", (0, 1, 2)), (4, (9, 10, 11), "bf16", (0, 1, 2)),
                                              (5, (13, 16, 12), "f32", (0, 1, 2)), (3, (4, 4, 4), "f32", (0, 1, 2))])
def test_eval_general_knots(ctx, torch_cuda, orc, p, n, storage, axes):
    from paper_2204_11762_gb300 import mfadvr
    torch = torch_cuda
    rng = np.random.default_rng(1000 + p * 10 + len(axes))
    ctrl = rng.normal(size=(n[2], n[1], n[0])).astype(np.float32)
    given, kv = _knots(2000 + p, n, p, axes)
    pts = np.concatenate([rng.uniform(0, 1, size=(3000, 3)).astype(np.float32), _edge_points(kv, p, n)])
    mid = ctx.load_model(ctrl, p, storage=storage, knots=given)
    got, sp = _eval(ctx, torch, mid, pts)
    deq = dequantize(ctrl, storage)
    ref, ref_sp = orc.eval_points(deq, p, pts, knot_vectors=kv)
    _check(got, sp, ref, ref_sp, deq, kv, p, n)
    # value-only and gradient-only queries equal the combined one bit for bit
    np.testing.assert_array_equal(ctx.query_points_host(mid, pts, mfadvr.QUERY_VALUE), got[:, 0])
    np.testing.assert_array_equal(ctx.query_points_host(mid, pts, mfadvr.QUERY_GRADIENT), got[:, 1:])
    ctx.unload_model(mid)


def test_general_knots_rejected_when_invalid(ctx, torch_cuda):
    from paper_2204_11762_gb300 import mfadvr
    p, n = 2, (6, 6, 6)
    ctrl = np.zeros((6, 6, 6), np.float32)
    good = np.array([0, 0, 0, 0.3, 0.5, 0.7, 1, 1, 1], np.float32)
    bads = [good * 0.5, good[::-1].copy(), np.where(good == 0.5, np.float32(0.2), good),
            np.where(good == 0.5, np.float32(0.3), good), np.where(good == 0.5, np.float32(np.nan), good)]
    for bad in bads:
        with pytest.raises(mfadvr.MfadvrError) as e:
            ctx.load_model(ctrl, p, knots=[bad, None, None])
        assert e.value.status == mfadvr.EINVAL
    ctx.unload_model(ctx.load_model(ctrl, p, knots=[good, None, good]))


def _persp(eye, fovy=50.0):
    return {"kind": 1, "eye": eye, "center": (0.5, 0.5, 0.5), "up": (0, 0, 1), "fovy_deg": fovy}


def _render(ctx, torch, mid, cam, prm, tf):
    dev = torch.device("cuda:0")
    H, W = prm["height"], prm["width"]
    img = torch.full((H, W, 4), float("nan"), device=dev)
    ns = torch.full((H, W), -1, dtype=torch.int32, device=dev)
    ctx.render(mid, cam, prm, torch.from_numpy(tf).to(dev), tf.shape[0], img, ns)
    torch.cuda.synchronize()
    return img.cpu().numpy(), ns.cpu().numpy()


@pytest.mark.parametrize("form", [0, 1])  # AUTO (span polynomials for FP32 up to degree 3), B-spline
@pytest.mark.parametrize("p,storage,shading", [(1, "f32", 1), (2, "f32", 0), (3, "f32", 1), (3, "bf16", 1),
                                               (3, "f32", 0), (4, "f32", 1), (5, "f16", 1), (2, "f32", 1)])
def test_render_general_knots(ctx, torch_cuda, orc, p, storage, shading, form):
    from paper_2204_11762_gb300 import workloads
    torch = torch_cuda
    rng = np.random.default_rng(3000 + p * 7 + shading)
    n = (p + 12, p + 9, p + 14)
    ctrl = workloads.gaussian_sum_lattice(n, p, rng)
    given, kv = _knots(3100 + p, n, p)
    tf = workloads.transfer_function(rng, 128)
    cam = _persp((1.9, -1.2, 1.4))
    prm = {"width": 48, "height": 40, "step": 1 / 256, "max_opacity": 0.99, "ref_step": 1 / 16,
           "shading": shading}
    mid = ctx.load_model(ctrl, p, storage=storage, knots=given, render_form=form)
    img, ns = _render(ctx, torch, mid, cam, prm, tf)
    ref = orc.render(dequantize(ctrl, storage), p, cam,
                     dict(prm, tf=tf, tf_lo=float(ctrl.min()), tf_hi=float(ctrl.max())), knot_vectors=kv)
    assert_render_parity(img, ns, ref)
    ctx.unload_model(mid)


def test_batch_mixes_general_and_uniform_knots(torch_cuda):
    """Jobs on general and on uniform knots run in separate launch groups; every
    image equals its single render bit for bit."""
    from paper_2204_11762_gb300 import mfadvr, workloads
    torch = torch_cuda
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(77)
    with mfadvr.Context(0) as ctx:
        jobs = []
        for i, (p, n, st) in enumerate([(3, (20, 24, 18), "f32"), (3, (19, 17, 22), "f32"), (2, (16, 15, 14), "f16"),
                                        (4, (15, 16, 17), "f32"), (3, (21, 20, 19), "bf16")]):
            ctrl = workloads.gaussian_sum_lattice(n, p, rng)
            given = _knots(4000 + i, n, p)[0] if i % 2 == 0 else None
            mid = ctx.load_model(ctrl, p, storage=st, knots=given)
            W, H = 40 + 8 * i, 32 + 4 * i
            tf = workloads.transfer_function(rng, 64)
            jobs.append({"model_id": mid, "camera": workloads.sphere_camera(rng),
                         "params": {"width": W, "height": H, "step": 1 / 256, "max_opacity": 0.99,
                                    "shading": int(i % 3 != 1)},
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
