"""The allocation-free render entry point (mfadvr_render_lattice_noalloc),
for callers that cannot allocate device memory during a render: stream
captures, plug-in hosts whose memory belongs to a pool allocator, real-time
loops.  It must give the same image as the regular entry point
(mfadvr_load_model + mfadvr_render) on the same lattice, call after call.

This file is collected last so that, if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest

from _parity import PIXEL_ATOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _case(seed, p, n, W, H, shading):
    from paper_2204_11762_gb300 import workloads
    rng = np.random.default_rng(seed)
    ctrl = workloads.gaussian_sum_lattice(n, p, rng)
    tf = workloads.transfer_function(rng, 256)
    cam = workloads.sphere_camera(rng)
    prm = {"width": W, "height": H, "step": 1 / 256, "max_opacity": 0.99, "ref_step": 1 / 16,
           "shading": shading, "tf_lo": float(ctrl.min()), "tf_hi": float(ctrl.max())}
    return ctrl, tf, cam, prm


@pytest.mark.parametrize("p,n,W,H,shading", [(3, (40, 36, 44), 96, 80, 1), (2, (17, 23, 19), 61, 47, 0)])
def test_noalloc_matches_regular_render_twice(torch_cuda, p, n, W, H, shading):
    from paper_2204_11762_gb300 import mfadvr
    torch = torch_cuda
    dev = torch.device("cuda:0")
    ctrl, tf, cam, prm = _case(11 + p, p, n, W, H, shading)
    d_tf = torch.from_numpy(tf).to(dev)
    with mfadvr.Context(0) as ctx:
        mid = ctx.load_model(ctrl, p)
        ref = torch.empty((H, W, 4), device=dev)
        ref_ns = torch.empty((H, W), dtype=torch.int32, device=dev)
        ctx.render(mid, cam, prm, d_tf, tf.shape[0], ref, ref_ns)
        torch.cuda.synchronize()
        ref, ref_ns = ref.cpu().numpy(), ref_ns.cpu().numpy()
    d_ctrl = torch.from_numpy(ctrl).to(dev)  # caller-owned lattice
    for call in range(2):
        img = torch.full((H, W, 4), float("nan"), device=dev)
        ns = torch.full((H, W), -1, dtype=torch.int32, device=dev)
        mfadvr.render_lattice_noalloc(d_ctrl, p, (n[0], n[1], n[2]), cam, prm, d_tf, tf.shape[0], img, ns)
        torch.cuda.synchronize()
        img, ns = img.cpu().numpy(), ns.cpu().numpy()
        assert np.isfinite(img).all(), f"call {call}: unwritten pixels"
        assert np.abs(img - ref).max() <= PIXEL_ATOL, f"call {call}: max diff {np.abs(img - ref).max()}"
        assert (ns == ref_ns).mean() > 0.999, f"call {call}: sample counts differ"


def test_noalloc_rejects_oversize_lattice(torch_cuda):
    from paper_2204_11762_gb300 import mfadvr
    torch = torch_cuda
    dev = torch.device("cuda:0")
    n = (100, 100, 53)  # 530,000 > 2^19 control points
    assert n[0] * n[1] * n[2] > mfadvr.NOALLOC_MAX_POINTS
    d_ctrl = torch.zeros(n[0] * n[1] * n[2], device=dev)
    d_tf = torch.ones((4, 4), device=dev)
    img = torch.empty((8, 8, 4), device=dev)
    prm = {"width": 8, "height": 8, "step": 0.05, "tf_lo": 0.0, "tf_hi": 1.0}
    with pytest.raises(mfadvr.MfadvrError) as e:
        mfadvr.render_lattice_noalloc(d_ctrl, 3, n, {"kind": 1, "eye": (2, 2, 2)}, prm, d_tf, 4, img)
    assert e.value.status == mfadvr.ENOMEM
    assert "exceeds the allocation-free scratch" in str(e.value)


def test_noalloc_rejects_sides_whose_product_wraps(torch_cuda):
    """Sides of 2^24 x 2^24 x 2^16 control points multiply to 2^64, which is 0
    in 64-bit arithmetic; the call must refuse them before any launch
    rather than let a wrapped count pass the size limit."""
    from paper_2204_11762_gb300 import mfadvr
    torch = torch_cuda
    dev = torch.device("cuda:0")
    n = (1 << 24, 1 << 24, 1 << 16)
    d_ctrl = torch.zeros(64, device=dev)
    d_tf = torch.ones((4, 4), device=dev)
    img = torch.empty((8, 8, 4), device=dev)
    prm = {"width": 8, "height": 8, "step": 0.05, "tf_lo": 0.0, "tf_hi": 1.0}
    with pytest.raises(mfadvr.MfadvrError) as e:
        mfadvr.render_lattice_noalloc(d_ctrl, 3, n, {"kind": 1, "eye": (2, 2, 2)}, prm, d_tf, 4, img)
    assert e.value.status == mfadvr.ENOMEM
    torch.cuda.synchronize()
