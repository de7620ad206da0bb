"""The POWER render form (span polynomials evaluated by Horner's rule; the
renders of tests/test_gpu_knots.py and tests/test_gpu_nurbs.py cover it on
general knots and rational models),
through the C ABI: renders agree with the FP64 oracle as the B-spline form's
do (pixels within 2e-3 per channel, sample counts on a branch of every tied
decision), the polynomials take the bytes the header states, and the form is
refused or dropped where it does not apply."""
import numpy as np
import pytest

from _parity import assert_render_parity

pytestmark = pytest.mark.gpu

CELL_BYTES = {1: 32, 2: 160, 3: 256, 4: 608}


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


def _render(ctx, torch, mid, cam, prm, tf):
    dev = torch.device("cuda:0")
    W, H = prm["width"], prm["height"]
    d_tf = torch.from_numpy(np.ascontiguousarray(tf, dtype=np.float32)).to(dev)
    d_img = torch.full((H, W, 4), float("nan"), dtype=torch.float32, device=dev)
    d_ns = torch.full((H, W), -1, dtype=torch.int32, device=dev)
    ctx.render(mid, cam, prm, d_tf, tf.shape[0], d_img, d_ns)
    torch.cuda.synchronize()
    return d_img.cpu().numpy(), d_ns.cpu().numpy()


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("shading", [1, 0])
def test_power_form_matches_oracle(ctx, torch_cuda, orc, p, shading):
    """Random lattices (every cell's polynomial differs, clamped cells at all
    six faces), both forms against the oracle."""
    from paper_2204_11762_gb300 import mfadvr, workloads
    rng = np.random.default_rng(40 + 2 * p + shading)
    ctrl = rng.normal(size=(13 + p, 11, 12 + 2 * p)).astype(np.float32)
    tf = workloads.transfer_function(rng, 64)
    cam = {"kind": 1, "eye": (1.9, -0.8, 1.4), "center": (0.5, 0.5, 0.5), "up": (0, 0, 1), "fovy_deg": 50.0}
    prm = {"width": 44, "height": 36, "step": 1 / 160, "max_opacity": 0.99, "ref_step": 1 / 40, "shading": shading}
    ref = orc.render(ctrl, p, cam, dict(prm, tf=tf))
    imgs = {}
    for form in (mfadvr.FORM_POWER, mfadvr.FORM_BSPLINE):
        mid = ctx.load_model(ctrl, p, render_form=form)
        img, ns = _render(ctx, torch_cuda, mid, cam, prm, tf)
        assert_render_parity(img, ns, ref)
        imgs[form] = img
        ctx.unload_model(mid)
    assert np.abs(imgs[mfadvr.FORM_POWER] - imgs[mfadvr.FORM_BSPLINE]).max() < 2e-3


@pytest.mark.parametrize("p,n", [(3, (4, 4, 4)), (3, (5, 4, 6)), (2, (3, 5, 3)), (1, (2, 2, 3)), (4, (5, 6, 5))])
def test_power_form_single_span_axes(ctx, torch_cuda, orc, p, n):
    """Lattices with one or two spans per axis: every cell is clamped at both
    ends of some axis (the knot patterns with both ends cut)."""
    from paper_2204_11762_gb300 import mfadvr, workloads
    rng = np.random.default_rng(sum(n) + 10 * p)
    ctrl = rng.uniform(-1, 1, size=n[::-1]).astype(np.float32)
    tf = workloads.transfer_function(rng, 32)
    cam = {"kind": 1, "eye": (2.1, 1.3, 1.6), "center": (0.5, 0.5, 0.5), "up": (0, 0, 1), "fovy_deg": 45.0}
    prm = {"width": 24, "height": 20, "step": 1 / 96, "max_opacity": 0.99, "shading": 1}
    mid = ctx.load_model(ctrl, p, render_form=mfadvr.FORM_POWER)
    img, ns = _render(ctx, torch_cuda, mid, cam, prm, tf)
    assert_render_parity(img, ns, orc.render(ctrl, p, cam, dict(prm, tf=tf)))
    ctx.unload_model(mid)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_power_form_bytes_and_point_queries(ctx, torch_cuda, p):
    """The span polynomials add m0 m1 m2 cells of the stated size; point
    queries keep using the row array, bit for bit."""
    from paper_2204_11762_gb300 import mfadvr
    torch = torch_cuda
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(p)
    n = (9 + p, 7 + p, 8)  # (n_u, n_v, n_w)
    ctrl = rng.normal(size=n[::-1]).astype(np.float32)
    a = ctx.load_model(ctrl, p, render_form=mfadvr.FORM_POWER)
    b = ctx.load_model(ctrl, p, render_form=mfadvr.FORM_BSPLINE)
    c = ctx.load_model(ctrl, p)  # AUTO
    cells = (n[0] - p) * (n[1] - p) * (n[2] - p)
    assert ctx.model_info(a)["bytes"] - ctx.model_info(b)["bytes"] == cells * CELL_BYTES[p]
    assert ctx.model_info(c)["bytes"] == ctx.model_info(a)["bytes"]
    k = 5000
    pts = torch.from_numpy(rng.uniform(0, 1, size=(k, 3)).astype(np.float32)).to(dev)
    outs = []
    for mid in (a, b):
        o = torch.empty((k, 4), device=dev)
        ctx.eval_points(mid, pts, k, o)
        outs.append(o)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1])
    for mid in (a, b, c):
        ctx.unload_model(mid)


def test_power_form_requirements(torch_cuda):
    from paper_2204_11762_gb300 import mfadvr
    rng = np.random.default_rng(3)
    ctrl = rng.normal(size=(10, 10, 10)).astype(np.float32)
    knots = np.concatenate([np.zeros(4), [0.3, 0.35, 0.5, 0.6, 0.8, 0.9], np.ones(4)]).astype(np.float32)
    with mfadvr.Context(0) as ctx:
        for kw in ({"storage": "f16"}, {"storage": "bf16"}):
            with pytest.raises(mfadvr.MfadvrError) as e:
                ctx.load_model(ctrl, 3, render_form=mfadvr.FORM_POWER, **kw)
            assert e.value.status == mfadvr.EUNSUPPORTED
            mid = ctx.load_model(ctrl, 3, **kw)  # AUTO: the B-spline form
            ctx.unload_model(mid)
        w = np.full_like(ctrl, 2.0)
        a = ctx.load_model(ctrl, 3, weights=w, render_form=mfadvr.FORM_POWER)
        b = ctx.load_model(ctrl, 3, weights=w, render_form=mfadvr.FORM_BSPLINE)
        # a rational model's polynomials: of w P and of w
        assert ctx.model_info(a)["bytes"] - ctx.model_info(b)["bytes"] == 2 * 7 ** 3 * CELL_BYTES[3]
        mid = ctx.load_model(ctrl, 3, knots=(knots, None, knots), render_form=mfadvr.FORM_POWER)
        assert ctx.model_info(mid)["bytes"] > ctx.model_info(ctx.load_model(ctrl, 3, knots=(knots, None, knots),
                                                                             render_form=mfadvr.FORM_BSPLINE))["bytes"]
        for deg, kw in ((5, {}), (4, {"weights": w})):  # degree 5; rational degree 4
            with pytest.raises(mfadvr.MfadvrError) as e:
                ctx.load_model(ctrl, deg, render_form=mfadvr.FORM_POWER, **kw)
            assert e.value.status == mfadvr.EUNSUPPORTED
        with pytest.raises(mfadvr.MfadvrError) as e:
            ctx.load_model(ctrl, 3, render_form=3)
        assert e.value.status == mfadvr.EINVAL
    rows = 10 ** 3 * 32
    with mfadvr.Context(0, hbm_budget_bytes=rows + 1000) as ctx:
        with pytest.raises(mfadvr.MfadvrError) as e:
            ctx.load_model(ctrl, 3, render_form=mfadvr.FORM_POWER)
        assert e.value.status == mfadvr.ENOMEM
        mid = ctx.load_model(ctrl, 3)  # AUTO falls back to the B-spline form within the budget
        assert ctx.model_info(mid)["bytes"] == rows
        ctx.unload_model(mid)


def test_batch_mixed_forms_equal_single_renders(torch_cuda):
    """Jobs on the same lattice in both forms, and 16-bit jobs, in one batched
    call: each image equals its single render, and the two forms agree."""
    from paper_2204_11762_gb300 import mfadvr, workloads
    torch = torch_cuda
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(77)
    with mfadvr.Context(0) as ctx:
        jobs = []
        for p, form, storage in [(3, mfadvr.FORM_POWER, "f32"), (3, mfadvr.FORM_BSPLINE, "f32"),
                                 (2, mfadvr.FORM_POWER, "f32"), (3, mfadvr.FORM_AUTO, "f16")]:
            ctrl = workloads.gaussian_sum_lattice((30, 26, 28), p, np.random.default_rng(p))
            tf = workloads.transfer_function(np.random.default_rng(9), 256)
            cam = workloads.sphere_camera(np.random.default_rng(4))
            prm = {"width": 72, "height": 56, "step": 1 / 200, "max_opacity": 0.99, "shading": 1}
            mid = ctx.load_model(ctrl, p, storage=storage, render_form=form)
            jobs.append({"model_id": mid, "camera": cam, "params": prm, "tf_dev": torch.from_numpy(tf).to(dev),
                         "tf_size": 256, "rgba_dev": torch.full((56, 72, 4), float("nan"), device=dev),
                         "nsamples_dev": torch.full((56, 72), -1, dtype=torch.int32, device=dev)})
        ctx.render_batch(jobs)
        torch.cuda.synchronize()
        batch = [j["rgba_dev"].cpu().numpy() for j in jobs]
        for j, img in zip(jobs, batch):
            ctx.render(j["model_id"], j["camera"], j["params"], j["tf_dev"], j["tf_size"], j["rgba_dev"],
                       j["nsamples_dev"])
            torch.cuda.synchronize()
            np.testing.assert_array_equal(img, j["rgba_dev"].cpu().numpy())
        assert np.abs(batch[0] - batch[1]).max() < 2e-3
