"""The serving loop (mfadvr_serve_start / submit / wait) through the C ABI:
requests of different models, image sizes and cameras admitted by a frame
budget and batched into persistent launches replayed through CUDA graphs.
Every image must be the same whether its request ran alone (mfadvr_render)
or in the mix, and requests submitted while batches run must join later
batches."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _models(ctx, rng):
    from paper_2204_11762_gb300 import workloads
    out = []
    for p, n, st in [(3, (40, 44, 36), "f16"), (4, (30, 28, 33), "f16"), (3, (50, 30, 45), "f32"),
                     (2, (35, 40, 30), "bf16")]:
        ctrl = workloads.gaussian_sum_lattice(n, p, rng)
        out.append(ctx.load_model(ctrl, p, storage=st))
    return out


def _requests(torch, models, rng, count, sizes=(32, 64, 128)):
    from paper_2204_11762_gb300 import workloads
    dev = torch.device("cuda:0")
    reqs = []
    for _ in range(count):
        side = int(rng.choice(sizes))
        tf = workloads.transfer_function(rng, 256)
        reqs.append({"model_id": int(rng.choice(models)), "camera": workloads.sphere_camera(rng),
                     "params": {"width": side, "height": side, "step": 1 / 256, "max_opacity": 0.99,
                                "ref_step": 1 / 16, "shading": 1},
                     "tf_dev": torch.from_numpy(tf).to(dev), "tf_size": 256,
                     "rgba_dev": torch.full((side, side, 4), float("nan"), device=dev),
                     "nsamples_dev": torch.full((side, side), -1, dtype=torch.int32, device=dev)})
    return reqs


def _alone(ctx, torch, r):
    img = torch.empty_like(r["rgba_dev"])
    ns = torch.empty_like(r["nsamples_dev"])
    ctx.render(r["model_id"], r["camera"], r["params"], r["tf_dev"], r["tf_size"], img, ns)
    torch.cuda.synchronize()
    return img.cpu().numpy(), ns.cpu().numpy()


def test_results_same_alone_and_in_the_mix(torch_cuda):
    from paper_2204_11762_gb300 import mfadvr
    torch = torch_cuda
    rng = np.random.default_rng(21)
    with mfadvr.Context(0) as ctx:
        models = _models(ctx, rng)
        reqs = _requests(torch, models, rng, 24)
        ctx.serve_start(frame_budget_bytes=1 << 30, max_batch=8, max_in_flight=2)
        tickets = [ctx.submit(r) for r in reqs[:12]]
        time.sleep(0.002)  # the second wave arrives while the first runs
        tickets += [ctx.submit(r) for r in reqs[12:]]
        lats = [ctx.wait(t) for t in tickets]
        stats = ctx.serve_stats()
        ctx.serve_stop()
        assert all(l is not None and l >= 0 for l in lats)
        assert stats["launches"] >= 3  # 24 requests, at most 8 per batch
        assert stats["graph_updates"] + stats["graph_instantiations"] == stats["launches"]
        for r in reqs:
            img, ns = _alone(ctx, torch, r)
            np.testing.assert_array_equal(r["rgba_dev"].cpu().numpy(), img)
            np.testing.assert_array_equal(r["nsamples_dev"].cpu().numpy(), ns)


def test_budget_admits_one_at_a_time(torch_cuda):
    from paper_2204_11762_gb300 import mfadvr
    torch = torch_cuda
    rng = np.random.default_rng(22)
    with mfadvr.Context(0) as ctx:
        models = _models(ctx, rng)
        reqs = _requests(torch, models, rng, 6, sizes=(64,))
        # each request needs 64*64*20 bytes; the budget fits one
        ctx.serve_start(frame_budget_bytes=64 * 64 * 20, max_batch=8, max_in_flight=2)
        tickets = [ctx.submit(r) for r in reqs]
        for t in tickets:
            assert ctx.wait(t) is not None
        stats = ctx.serve_stats()
        ctx.serve_stop()
        assert stats["launches"] == len(reqs)
        for r in reqs:
            img, _ = _alone(ctx, torch, r)
            np.testing.assert_array_equal(r["rgba_dev"].cpu().numpy(), img)


def test_wait_poll_timeout_and_unknown_ticket(torch_cuda):
    from paper_2204_11762_gb300 import mfadvr, workloads
    torch = torch_cuda
    rng = np.random.default_rng(23)
    with mfadvr.Context(0) as ctx:
        models = _models(ctx, rng)
        big = _requests(torch, models, rng, 1, sizes=(1024,))[0]
        big["params"]["step"] = 1 / 2048
        ctx.serve_start()
        t = ctx.submit(big)
        first = ctx.wait(t, timeout_us=0)  # a 1024^2 frame is not done 0 us after submission
        lat = first if first is not None else ctx.wait(t)
        assert lat is not None
        with pytest.raises(mfadvr.MfadvrError) as e:
            ctx.wait(t)  # released
        assert e.value.status == mfadvr.ENOTFOUND
        with pytest.raises(mfadvr.MfadvrError) as e:
            ctx.submit(dict(big, model_id=12345))
        assert e.value.status == mfadvr.ENOTFOUND
        with pytest.raises(mfadvr.MfadvrError) as e:
            ctx.serve_start()
        assert e.value.status == mfadvr.EBUSY
        ctx.serve_stop()
        with pytest.raises(mfadvr.MfadvrError):
            ctx.submit(big)
