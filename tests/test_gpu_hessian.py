"""GPU parity of the Hessian query (MFADVR_QUERY_HESSIAN: value, gradient and
the six second partials; the higher-order query of Sec. 3.1) against the FP64
oracle: first-order outputs within 1e-4 and second-order ones within 1e-3 of
their scale (max|P| m and max|P| m^2, m = 1 / smallest span width)."""
import numpy as np
import pytest

from _parity import dequantize

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


@pytest.mark.parametrize("p,n,storage,general,rational", [
    (1, (7, 8, 9), "f32", False, False), (2, (12, 10, 13), "f32", False, False),
    (3, (16, 18, 15), "f32", False, False), (3, (14, 13, 17), "f32", True, False),
    (3, (13, 15, 14), "f32", False, True), (3, (12, 14, 11), "f16", False, False),
    (4, (11, 12, 13), "f32", True, True), (5, (12, 11, 10), "bf16", False, False)])
def test_hessian_query(ctx, torch_cuda, orc, p, n, storage, general, rational):
    from paper_2204_11762_gb300 import mfadvr, workloads
    torch = torch_cuda
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(7000 + p * 11 + general + 2 * rational)
    ctrl = rng.normal(size=(n[2], n[1], n[0])).astype(np.float32)
    w = rng.uniform(0.5, 2.0, size=ctrl.shape).astype(np.float32) if rational else None
    kv = [workloads.graded_knots(rng, n[d], p) for d in range(3)] if general else None
    pts = rng.uniform(0, 1, size=(1500, 3)).astype(np.float32)
    pts[:3] = [[0, 0, 0], [1, 1, 1], [0.5, 0, 1]]
    mid = ctx.load_model(ctrl, p, storage=storage, knots=kv, weights=w)
    k = pts.shape[0]
    d_out = torch.full((k, 10), float("nan"), device=dev)
    d_sp = torch.full((k, 3), -1, dtype=torch.int32, device=dev)
    ctx.query_points(mid, torch.from_numpy(pts).to(dev), k, d_out, mfadvr.QUERY_HESSIAN, d_sp)
    torch.cuda.synchronize()
    got = d_out.cpu().numpy()
    if rational:
        q = (w.astype(np.float64) * ctrl.astype(np.float64)).astype(np.float32)
        wd = dequantize(w, storage)
        c_eff = dequantize(q, storage) / wd
    else:
        c_eff, wd = dequantize(ctrl, storage), None
    kv64 = [t.astype(np.float64) for t in kv] if kv else None
    ref = orc.eval_hessian(c_eff, p, pts, knot_vectors=kv64, weights=wd)
    _, ref_sp = orc.eval_points(c_eff, p, pts, knot_vectors=kv64, weights=wd)
    np.testing.assert_array_equal(d_sp.cpu().numpy(), ref_sp)
    pabs = float(np.abs(c_eff).max())
    hmin = min(float(np.diff(kv[d][p:n[d] + 1]).min()) for d in range(3)) if kv else 1.0 / (max(n) - p)
    m = 1.0 / hmin
    scale = np.array([pabs] + [pabs * m] * 3 + [pabs * m * m] * 6) * (4.0 if rational else 1.0)
    err = np.abs(got - ref) / np.maximum(np.abs(ref), scale)
    tol = np.array([1e-5] + [1e-4] * 3 + [1e-3] * 6)
    worst = (err / tol).max(axis=0)
    assert (worst <= 1.0).all(), f"error / tolerance per output: {worst}"
    # the first four outputs agree with the combined query
    both = ctx.query_points_host(mid, pts, mfadvr.QUERY_BOTH)
    np.testing.assert_allclose(got[:, :4], both, rtol=0, atol=1e-5 * scale[:4].max())
    ctx.unload_model(mid)
