"""GPU parity of mfadvr_eval_points against the FP64 oracle, through the C ABI.

Spans must match exactly; values within 1e-5 and gradients within 1e-4 of
the model scale (see tests/_parity.py)."""
import numpy as np
import pytest

from _parity import assert_eval_parity, dequantize, storage_scale

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


def _edge_points(n, p):
    """Parameters at, just above and just below every knot (FP32), the box
    corners, and points outside the box."""
    pts = []
    for d in range(3):
        m = n[d] - p
        for j in range(m + 1):
            k = np.float32(j / m)
            for u in (k, np.nextafter(k, np.float32(2)), np.nextafter(k, np.float32(-1))):
                q = np.full(3, 0.37, dtype=np.float32)
                q[d] = u
                pts.append(q)
    pts += [np.zeros(3), np.ones(3), [-0.25, 1.5, 0.5], [2.0, -1.0, 1.0], [0.5, 0.5, 1.0]]
    return np.asarray(pts, dtype=np.float32)


def _run(ctx, torch, mid, pts):
    dev = torch.device("cuda:0")
    n = pts.shape[0]
    d_pts = torch.from_numpy(np.ascontiguousarray(pts)).to(dev)
    d_out = torch.full((max(n, 1), 4), float("nan"), dtype=torch.float32, device=dev)
    d_sp = torch.full((max(n, 1), 3), -1, dtype=torch.int32, device=dev)
    ctx.eval_points(mid, d_pts, n, d_out, d_sp)
    torch.cuda.synchronize()
    return d_out.cpu().numpy()[:n], d_sp.cpu().numpy()[:n]


@pytest.mark.parametrize("p,n", [(1, (2, 3, 2)), (1, (17, 9, 33)), (2, (3, 4, 5)), (2, (40, 21, 13)),
                                 (3, (4, 4, 4)), (3, (5, 9, 6)), (3, (32, 33, 34)), (4, (5, 6, 7)),
                                 (4, (29, 18, 25)), (5, (6, 6, 6)), (5, (9, 11, 10)), (5, (31, 24, 27))])
def test_eval_parity_f32(ctx, torch_cuda, orc, p, n):
    rng = np.random.default_rng(100 + p * 7 + n[0])
    ctrl = rng.normal(size=(n[2], n[1], n[0])).astype(np.float32)
    pts = np.concatenate([rng.uniform(0, 1, size=(3001, 3)).astype(np.float32), _edge_points(n, p)])
    mid = ctx.load_model(ctrl, p)
    got, sp = _run(ctx, torch_cuda, mid, pts)
    ref, ref_sp = orc.eval_points(ctrl, p, pts)
    assert_eval_parity(got, ref, ctrl, n, p, sp, ref_sp)
    ctx.unload_model(mid)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_eval_parity_16bit_storage(ctx, torch_cuda, orc, storage, p):
    """16-bit storage with a per-model scale, FP32 accumulation: parity with
    the oracle evaluated on the lattice the model actually stores."""
    rng = np.random.default_rng(300 + p)
    n = (23, 17, 29)
    ctrl = (rng.normal(size=(n[2], n[1], n[0])) * 3.7).astype(np.float32)
    pts = rng.uniform(0, 1, size=(4000, 3)).astype(np.float32)
    mid = ctx.load_model(ctrl, p, storage=storage)
    info = ctx.model_info(mid)
    assert info["scale"] == storage_scale(float(np.abs(ctrl).max()), storage)
    if storage == "f16":  # a power of two putting max|P| in FP16's top binade
        assert 2 ** 14 <= np.abs(ctrl).max() / info["scale"] < 2 ** 15
    assert info["bytes"] == ctrl.size * 32  # row layout: 16 16-bit values per lattice point
    got, sp = _run(ctx, torch_cuda, mid, pts)
    deq = dequantize(ctrl, storage)
    ref, ref_sp = orc.eval_points(deq, p, pts)
    assert_eval_parity(got, ref, deq, n, p, sp, ref_sp)
    ctx.unload_model(mid)


def test_eval_empty_and_tiny(ctx, torch_cuda, orc):
    rng = np.random.default_rng(5)
    ctrl = rng.normal(size=(4, 4, 4)).astype(np.float32)
    mid = ctx.load_model(ctrl, 3)
    got, sp = _run(ctx, torch_cuda, mid, np.zeros((0, 3), dtype=np.float32))
    assert got.shape == (0, 4)
    pts = np.array([[0.5, 0.25, 0.75]], dtype=np.float32)
    got, sp = _run(ctx, torch_cuda, mid, pts)
    ref, ref_sp = orc.eval_points(ctrl, 3, pts)
    assert_eval_parity(got, ref, ctrl, (4, 4, 4), 3, sp, ref_sp)
    ctx.unload_model(mid)


def test_eval_host_buffers_match_device(ctx, torch_cuda, orc):
    rng = np.random.default_rng(9)
    n = (20, 21, 22)
    ctrl = rng.normal(size=(n[2], n[1], n[0])).astype(np.float32)
    pts = rng.uniform(0, 1, size=(10007, 3)).astype(np.float32)
    mid = ctx.load_model(ctrl, 3)
    sp = np.empty((pts.shape[0], 3), dtype=np.int32)
    out = ctx.eval_points_host(mid, pts, spans=sp)
    dev_out, dev_sp = _run(ctx, torch_cuda, mid, pts)
    np.testing.assert_array_equal(out, dev_out)
    np.testing.assert_array_equal(sp, dev_sp)
    ctx.unload_model(mid)


def test_eval_full_size_gaussian_workload(ctx, torch_cuda, orc):
    """The 128^3 degree-3 Gaussian-sum model with 2^24 uniform points, in
    one launch as the benchmark times it; 20000 sampled outputs against the
    oracle, every span checked against the exact floor rule."""
    from paper_2204_11762_gb300 import workloads
    torch = torch_cuda
    wl = workloads.gaussian_sum_workload()
    ctrl, p, pts = wl["ctrl"], wl["degree"], wl["points"]
    n = ctrl.shape[::-1]
    mid = ctx.load_model(ctrl, p)
    got, sp = _run(ctx, torch, mid, pts)
    idx = np.random.default_rng(0).choice(pts.shape[0], 20000, replace=False)
    ref, ref_sp = orc.eval_points(ctrl, p, pts[idx])
    assert_eval_parity(got[idx], ref, ctrl, n, p, sp[idx], ref_sp)
    # every span: exact floor(u*m) (property that holds at any size)
    m = np.array(n) - p
    exact = np.floor(pts.astype(np.float64) * m).astype(np.int64)
    exact = np.clip(exact, 0, m - 1) + p
    assert np.array_equal(sp, exact)
    ctx.unload_model(mid)


def test_invalid_arguments(ctx, torch_cuda):
    from paper_2204_11762_gb300 import mfadvr
    rng = np.random.default_rng(1)
    with pytest.raises(mfadvr.MfadvrError) as e:
        ctx.load_model(rng.normal(size=(3, 3, 3)).astype(np.float32), 3)
    assert e.value.status == mfadvr.EINVAL
    with pytest.raises(mfadvr.MfadvrError) as e:
        ctx.load_model(rng.normal(size=(8, 8, 8)).astype(np.float32), 6)
    assert e.value.status == mfadvr.EUNSUPPORTED
    bad = rng.normal(size=(5, 5, 5)).astype(np.float32)
    bad[2, 2, 2] = np.nan
    with pytest.raises(mfadvr.MfadvrError) as e:
        ctx.load_model(bad, 2)
    assert e.value.status == mfadvr.EINVAL
    with pytest.raises(mfadvr.MfadvrError) as e:
        ctx.eval_points(12345, 0, 1, 0)
    assert e.value.status == mfadvr.ENOTFOUND


def test_hbm_budget(torch_cuda):
    from paper_2204_11762_gb300 import mfadvr
    with mfadvr.Context(0, hbm_budget_bytes=400_000) as c:
        a = c.load_model(np.zeros((20, 20, 20), dtype=np.float32), 3)  # 8000 row entries x 32 B
        with pytest.raises(mfadvr.MfadvrError) as e:
            c.load_model(np.zeros((20, 20, 20), dtype=np.float32), 3)
        assert e.value.status == mfadvr.ENOMEM
        c.unload_model(a)
        c.load_model(np.zeros((20, 20, 20), dtype=np.float32), 3)


@pytest.mark.parametrize("p,storage", [(1, "f32"), (2, "f16"), (3, "f32"), (3, "bf16"), (4, "f32"), (5, "f32"),
                                       (5, "f16")])
def test_query_modes_equal_both_bitwise(ctx, torch_cuda, orc, p, storage):
    """Value-only and gradient-only queries (Sec. 4.3.3) form only the sums
    they need; each output must equal the matching component of the combined
    query bit for bit, and the value and gradient must match the oracle."""
    from paper_2204_11762_gb300 import mfadvr
    torch = torch_cuda
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(900 + p)
    n = (p + 12, p + 7, p + 15)
    ctrl = rng.normal(size=(n[2], n[1], n[0])).astype(np.float32)
    pts = np.concatenate([rng.uniform(0, 1, size=(2049, 3)).astype(np.float32), _edge_points(n, p)])
    mid = ctx.load_model(ctrl, p, storage=storage)
    both, sp = _run(ctx, torch, mid, pts)
    d_pts = torch.from_numpy(pts).to(dev)
    k = pts.shape[0]
    d_val = torch.full((k,), float("nan"), device=dev)
    d_grad = torch.full((k, 3), float("nan"), device=dev)
    d_sp = torch.full((k, 3), -1, dtype=torch.int32, device=dev)
    ctx.query_points(mid, d_pts, k, d_val, mfadvr.QUERY_VALUE, d_sp)
    ctx.query_points(mid, d_pts, k, d_grad, mfadvr.QUERY_GRADIENT)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(d_val.cpu().numpy(), both[:, 0])
    np.testing.assert_array_equal(d_grad.cpu().numpy(), both[:, 1:])
    np.testing.assert_array_equal(d_sp.cpu().numpy(), sp)
    # host-buffer variants give the same bits
    np.testing.assert_array_equal(ctx.query_points_host(mid, pts, mfadvr.QUERY_VALUE), both[:, 0])
    np.testing.assert_array_equal(ctx.query_points_host(mid, pts, mfadvr.QUERY_GRADIENT), both[:, 1:])
    deq = dequantize(ctrl, storage)
    ref, ref_sp = orc.eval_points(deq, p, pts)
    assert_eval_parity(both, ref, deq, n, p, sp, ref_sp)
    ctx.unload_model(mid)


def test_query_rejects_bad_query(ctx, torch_cuda):
    from paper_2204_11762_gb300 import mfadvr
    torch = torch_cuda
    dev = torch.device("cuda:0")
    mid = ctx.load_model(np.ones((6, 6, 6), dtype=np.float32), 2)
    d_pts = torch.zeros((4, 3), device=dev)
    d_out = torch.zeros((4, 4), device=dev)
    for q in (0, 5, -1):
        with pytest.raises(mfadvr.MfadvrError) as e:
            ctx.query_points(mid, d_pts, 4, d_out, q)
        assert e.value.status == mfadvr.EINVAL
    with pytest.raises(mfadvr.MfadvrError) as e:  # QUERY_BOTH needs 16-byte alignment
        ctx.query_points(mid, d_pts, 3, d_out.view(-1)[1:], mfadvr.QUERY_BOTH)
    assert e.value.status == mfadvr.EINVAL
    ctx.query_points(mid, d_pts, 3, d_out.view(-1)[1:], mfadvr.QUERY_VALUE)  # 4-byte aligned is enough
    torch.cuda.synchronize()
    assert np.allclose(d_out.view(-1)[1:4].cpu().numpy(), 1.0)
    ctx.unload_model(mid)


def test_host_query_pipeline_matches_device_path(ctx, torch_cuda):
    """Host-buffer queries of 2^20 points or more run in chunks on the
    context's pipe streams; every chunk, the ragged last one included, must
    give the device-buffer bits, spans too."""
    from paper_2204_11762_gb300 import mfadvr
    torch = torch_cuda
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(1234)
    ctrl = rng.normal(size=(21, 19, 23)).astype(np.float32)
    mid = ctx.load_model(ctrl, 3)
    k = (1 << 20) + 7
    pts = rng.uniform(-0.05, 1.05, size=(k, 3)).astype(np.float32)
    d_out = torch.empty((k, 4), device=dev)
    d_sp = torch.empty((k, 3), dtype=torch.int32, device=dev)
    ctx.eval_points(mid, torch.from_numpy(pts).to(dev), k, d_out, d_sp)
    torch.cuda.synchronize()
    sp = np.empty((k, 3), dtype=np.int32)
    got = ctx.eval_points_host(mid, pts, spans=sp)
    np.testing.assert_array_equal(got, d_out.cpu().numpy())
    np.testing.assert_array_equal(sp, d_sp.cpu().numpy())
    hv = ctx.query_points_host(mid, pts, mfadvr.QUERY_VALUE)
    np.testing.assert_array_equal(hv, d_out.cpu().numpy()[:, 0])
    ctx.unload_model(mid)


def test_host_query_on_pinned_buffers_matches_device_path(ctx, torch_cuda):
    """Pinned host buffers are read and written by the kernel directly (no
    staging); the results must be the device-buffer bits, spans too."""
    from paper_2204_11762_gb300 import mfadvr
    torch = torch_cuda
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(4321)
    ctrl = rng.normal(size=(17, 22, 19)).astype(np.float32)
    mid = ctx.load_model(ctrl, 4, storage="bf16")
    k = 300001
    h_pts = torch.from_numpy(rng.uniform(0, 1, size=(k, 3)).astype(np.float32)).pin_memory()
    h_out = torch.full((k, 4), float("nan")).pin_memory()
    h_sp = torch.full((k, 3), -1, dtype=torch.int32).pin_memory()
    ctx.eval_points_host(mid, h_pts.numpy(), out=h_out.numpy(), spans=h_sp.numpy())
    d_out = torch.empty((k, 4), device=dev)
    d_sp = torch.empty((k, 3), dtype=torch.int32, device=dev)
    ctx.eval_points(mid, h_pts.to(dev), k, d_out, d_sp)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(h_out.numpy(), d_out.cpu().numpy())
    np.testing.assert_array_equal(h_sp.numpy(), d_sp.cpu().numpy())
    h_val = torch.empty(k).pin_memory()
    ctx.query_points_host(mid, h_pts.numpy(), mfadvr.QUERY_VALUE, out=h_val.numpy())
    np.testing.assert_array_equal(h_val.numpy(), d_out.cpu().numpy()[:, 0])
    ctx.unload_model(mid)


@pytest.mark.parametrize("max_ctas", [0, 3])
def test_async_host_query_matches_device_path(ctx, torch_cuda, max_ctas):
    """The stream-ordered host query on pinned buffers, on the whole GPU or
    on a few blocks (each block then strides over many points), must give the
    device-buffer bits for every query kind, spans too."""
    from paper_2204_11762_gb300 import mfadvr
    torch = torch_cuda
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(777)
    ctrl = rng.normal(size=(23, 18, 20)).astype(np.float32)
    mid = ctx.load_model(ctrl, 3)
    k = 100003
    h_pts = torch.from_numpy(rng.uniform(-0.05, 1.05, size=(k, 3)).astype(np.float32)).pin_memory()
    d_pts = h_pts.to(dev)
    s = torch.cuda.Stream(device=dev)
    widths = {mfadvr.QUERY_VALUE: 1, mfadvr.QUERY_GRADIENT: 3, mfadvr.QUERY_BOTH: 4, mfadvr.QUERY_HESSIAN: 10}
    for q, wdt in widths.items():
        h_out = torch.full((k, wdt), float("nan")).pin_memory()
        h_sp = torch.full((k, 3), -1, dtype=torch.int32).pin_memory()
        ctx.query_points_host_async(mid, h_pts, k, h_out, q, h_sp, max_ctas=max_ctas, stream=s.cuda_stream)
        d_out = torch.empty((k, wdt), device=dev)
        d_sp = torch.empty((k, 3), dtype=torch.int32, device=dev)
        ctx.query_points(mid, d_pts, k, d_out, q, d_sp)
        s.synchronize()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(h_out.numpy(), d_out.cpu().numpy())
        np.testing.assert_array_equal(h_sp.numpy(), d_sp.cpu().numpy())
    ctx.unload_model(mid)


def test_async_host_query_rejects_pageable_buffers(ctx, torch_cuda):
    from paper_2204_11762_gb300 import mfadvr
    torch = torch_cuda
    rng = np.random.default_rng(5)
    mid = ctx.load_model(rng.normal(size=(8, 8, 8)).astype(np.float32), 2)
    k = 1000
    pts = rng.uniform(0, 1, size=(k, 3)).astype(np.float32)
    h_pts = torch.from_numpy(pts).pin_memory()
    h_out = torch.empty((k, 4)).pin_memory()
    with pytest.raises(RuntimeError, match="page-locked"):
        ctx.query_points_host_async(mid, pts, k, h_out)
    with pytest.raises(RuntimeError, match="page-locked"):
        ctx.query_points_host_async(mid, h_pts, k, np.empty((k, 4), dtype=np.float32))
    with pytest.raises(RuntimeError, match="max_ctas"):
        ctx.query_points_host_async(mid, h_pts, k, h_out, max_ctas=-1)
    with pytest.raises(RuntimeError):
        ctx.query_points_host_async(mid, h_pts, k, h_out, query=5)
    ctx.query_points_host_async(mid, h_pts, 0, h_out)  # n = 0: no work, no error
    torch.cuda.synchronize()
    ctx.unload_model(mid)


def test_async_host_query_beside_a_render(ctx, torch_cuda):
    """A capped host query queued on one stream with a render on another (the
    end-to-end step): both results equal those of the same calls run alone."""
    from paper_2204_11762_gb300 import mfadvr, workloads
    torch = torch_cuda
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(99)
    ctrl = workloads.gaussian_sum_lattice((48, 40, 44), 3, rng)
    mid = ctx.load_model(ctrl, 3)
    k = 1 << 18
    h_pts = torch.from_numpy(rng.uniform(0, 1, size=(k, 3)).astype(np.float32)).pin_memory()
    h_out = torch.empty((k, 4)).pin_memory()
    tf = workloads.transfer_function(rng, 256)
    prm = {"width": 160, "height": 120, "step": 1 / 512, "max_opacity": 0.99, "shading": 1}
    cam = workloads.sphere_camera(rng)
    ref_img = ctx.render_host(mid, cam, prm, tf)
    d_out = torch.empty((k, 4), device=dev)
    ctx.eval_points(mid, h_pts.to(dev), k, d_out)
    torch.cuda.synchronize()
    ref_out = d_out.cpu().numpy()
    h_img = torch.empty((120, 160, 4)).pin_memory()
    sq, sr = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    for cap in (8, 0):
        h_out.fill_(float("nan"))
        h_img.fill_(float("nan"))
        ctx.query_points_host_async(mid, h_pts, k, h_out, mfadvr.QUERY_BOTH, max_ctas=cap, stream=sq.cuda_stream)
        ctx.render_host(mid, cam, prm, tf, rgba=h_img.numpy(), stream=sr.cuda_stream)
        sq.synchronize()
        np.testing.assert_array_equal(h_out.numpy(), ref_out)
        np.testing.assert_array_equal(h_img.numpy(), ref_img)
    ctx.unload_model(mid)


def test_usage_example_runs(torch_cuda):
    """The usage example (tests/example_usage.py, which README.md quotes)
    runs as written and gives finite queries and a non-empty image."""
    import os
    import runpy
    scope = runpy.run_path(os.path.join(os.path.dirname(os.path.abspath(__file__)), "example_usage.py"))
    torch_cuda.cuda.synchronize()
    out, img = scope["out"], scope["img"]
    assert torch_cuda.isfinite(out).all() and torch_cuda.isfinite(img).all()
    assert (img[..., 3] > 0).any()
