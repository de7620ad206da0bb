"""Knot spans on the render path (Algorithm 1, queryValueMFA inside the ray
loop): every sample a ray contracts is evaluated on the span that the oracle's
span search gives for that sample's own FP32 position.  mfadvr_render_trace
records the positions and spans the kernel used; the oracle's find_span
(binary search on the FP64 knot vector) is run on exactly those positions.
Uniform knots in both render forms, general knots in both forms, and rays
and samples that lie exactly on knots."""
import numpy as np
import pytest

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


def _trace(ctx, torch, mid, cam, prm, tf, max_samples):
    dev = torch.device("cuda:0")
    W, H = prm["width"], prm["height"]
    d_tf = torch.from_numpy(np.ascontiguousarray(tf, dtype=np.float32)).to(dev)
    img = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    ns = torch.full((H, W), -1, dtype=torch.int32, device=dev)
    pos = torch.full((H, W, max_samples, 3), float("nan"), dtype=torch.float32, device=dev)
    span = torch.full((H, W, max_samples, 3), -1, dtype=torch.int32, device=dev)
    ctx.render_trace(mid, cam, prm, d_tf, tf.shape[0], img, ns, max_samples, pos, span)
    torch.cuda.synchronize()
    return img.cpu().numpy(), ns.cpu().numpy(), pos.cpu().numpy(), span.cpu().numpy()


def _check_spans(orc, ns, pos, span, n, p, knots=None):
    """Every recorded sample: span == find_span of its position.  Returns the
    number of samples checked."""
    H, W, K, _ = pos.shape
    checked = 0
    for a in range(3):
        m = n[a] - p
        t = None if knots is None else np.asarray(knots[a], dtype=np.float64)
        written = span[..., a] >= 0
        x = pos[..., a][written].astype(np.float64)
        u = x / m if knots is None else x  # lattice units -> parameter (exact ratio, then FP64)
        got = span[..., a][written]
        cache = {}
        want = np.empty_like(got)
        for i, ui in enumerate(u):
            key = float(ui)
            if key not in cache:
                cache[key] = orc.find_span(n[a], p, key, t)
            want[i] = cache[key]
        bad = np.nonzero(got != want)[0]
        assert bad.size == 0, (f"axis {a}: {bad.size} of {got.size} spans differ; first positions "
                               f"{x[bad[:4]]} spans {got[bad[:4]]} vs oracle {want[bad[:4]]}")
        checked += got.size
    # every ray records its contracted samples 0..ns (the last one may lie
    # past the box), nothing beyond
    k = np.arange(K)[None, None, :]
    hit = ns > 0
    expect = (k <= ns[..., None]) & hit[..., None] & (k < K)
    assert np.array_equal(span[..., 0] >= 0, expect), "recorded samples differ from the contracted ones"
    return checked


def _case(seed, n, p, knots=False):
    from paper_2204_11762_gb300 import workloads
    rng = np.random.default_rng(seed)
    ctrl = workloads.gaussian_sum_lattice(n, p, rng)
    kv = [workloads.graded_knots(rng, n[a], p) for a in range(3)] if knots else None
    tf = workloads.transfer_function(rng, 64)
    cam = workloads.sphere_camera(rng, fovy_deg=35.0)  # the box fills most of the image
    return ctrl, kv, tf, cam


@pytest.mark.parametrize("form", ["power", "bspline"])
@pytest.mark.parametrize("knots", [False, True])
@pytest.mark.parametrize("p", [2, 3])
def test_render_spans_match_the_oracle(ctx, torch_cuda, orc, form, knots, p):
    from paper_2204_11762_gb300 import mfadvr
    n = (21, 17, 26)
    ctrl, kv, tf, cam = _case(400 + 10 * p + int(knots), n, p, knots)
    mid = ctx.load_model(ctrl, p, knots=kv,
                         render_form=mfadvr.FORM_POWER if form == "power" else mfadvr.FORM_BSPLINE)
    prm = {"width": 25, "height": 19, "step": 1 / 128, "max_opacity": 0.99, "ref_step": 1 / 16, "shading": 1}
    K = 256  # > sqrt(3) * 128 + 2 samples per ray
    img, ns, pos, span = _trace(ctx, torch_cuda, mid, cam, prm, tf, K)
    checked = _check_spans(orc, ns, pos, span, n, p, kv)
    assert (ns > 0).sum() > 200 and checked > 3 * 10000
    # the traced render is the render
    d_tf = torch_cuda.from_numpy(tf).cuda()
    out = torch_cuda.empty_like(torch_cuda.from_numpy(img)).cuda()
    ns2 = torch_cuda.empty((prm["height"], prm["width"]), dtype=torch_cuda.int32, device="cuda")
    ctx.render(mid, cam, prm, d_tf, tf.shape[0], out, ns2)
    torch_cuda.cuda.synchronize()
    ref = out.cpu().numpy()
    # the same arithmetic in another instantiation: equal up to FP32 rounding
    assert np.abs(img - ref).max() <= 1e-5
    assert (ns == ns2.cpu().numpy()).mean() >= 0.999
    ctx.unload_model(mid)


@pytest.mark.parametrize("form", ["power", "bspline"])
def test_rays_and_samples_on_knots(ctx, torch_cuda, orc, form):
    """Orthographic rays along +w through pixel centres u, v = (2i+1)/16 with
    16 spans per axis: every ray lies on a u knot and a v knot, and with step
    2/16 every sample lies on a w knot (lattice positions 2s + 1).  A position
    on a knot belongs to the span on its right."""
    from paper_2204_11762_gb300 import mfadvr, workloads
    p, n = 3, (19, 19, 19)
    rng = np.random.default_rng(431)
    ctrl = workloads.gaussian_sum_lattice(n, p, rng)
    tf = workloads.transfer_function(rng, 64)
    mid = ctx.load_model(ctrl, p, render_form=mfadvr.FORM_POWER if form == "power" else mfadvr.FORM_BSPLINE)
    cam = {"kind": 0, "eye": (0.5, 0.5, -1.0), "center": (0.5, 0.5, 0.5), "up": (0.0, 1.0, 0.0),
           "ortho_height": 1.0}
    prm = {"width": 8, "height": 8, "step": 2 / 16, "max_opacity": 1.0, "ref_step": 1 / 16, "shading": 1}
    img, ns, pos, span = _trace(ctx, torch_cuda, mid, cam, prm, tf, 16)
    assert (ns == 8).all(), "every ray crosses the box in 8 samples"
    x = pos[:, :, :8, :]
    assert np.array_equal(x, np.round(x)), "positions are not exactly on knots"
    assert (np.round(x[..., 2]) % 2 == 1).all()
    _check_spans(orc, ns, pos, span, n, p)
    # on a knot: the span starting there (clamped to the last span at u = 1)
    k = np.minimum(np.round(pos[:, :, :8, :]).astype(int), n[0] - p - 1) + p
    np.testing.assert_array_equal(span[:, :, :8, :], k)
    ctx.unload_model(mid)


def test_trace_refuses_what_it_does_not_cover(ctx, torch_cuda):
    from paper_2204_11762_gb300 import mfadvr
    torch = torch_cuda
    mid = ctx.load_model(np.ones((6, 6, 6), dtype=np.float32), 2, storage="bf16")
    tf = torch.ones((4, 4), device="cuda")
    img = torch.empty((4, 4, 4), device="cuda")
    pos = torch.empty((4, 4, 4, 3), device="cuda")
    span = torch.empty((4, 4, 4, 3), dtype=torch.int32, device="cuda")
    prm = {"width": 4, "height": 4, "step": 0.1, "shading": 1}
    with pytest.raises(mfadvr.MfadvrError) as e:
        ctx.render_trace(mid, {"kind": 1, "eye": (2, 2, 2)}, prm, tf, 4, img, None, 4, pos, span)
    assert e.value.status == mfadvr.EUNSUPPORTED
    ctx.unload_model(mid)
    mid = ctx.load_model(np.ones((6, 6, 6), dtype=np.float32), 2)
    with pytest.raises(mfadvr.MfadvrError) as e:
        ctx.render_trace(mid, {"kind": 1, "eye": (2, 2, 2)}, dict(prm, width=4096, height=4096), tf, 4, img,
                         None, 4, pos, span)
    assert e.value.status == mfadvr.EINVAL
    ctx.unload_model(mid)
