"""Batched rendering (mfadvr_render_batch) and the autotuner, through the C
ABI: every image of a batch -- mixed degrees, storage types, image sizes and
tile shapes -- must equal the image mfadvr_render gives for the same job on
its own (both follow Algorithm 1 with the same per-ray arithmetic)."""
import os

import numpy as np
import pytest

from _parity import assert_render_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _jobs(ctx, torch, specs, seed=5):
    from paper_2204_11762_gb300 import workloads
    rng = np.random.default_rng(seed)
    dev = torch.device("cuda:0")
    out = []
    for p, n, storage, (W, H) in specs:
        ctrl = workloads.gaussian_sum_lattice(n, p, rng)
        tf = workloads.transfer_function(rng, 256)
        cam = workloads.sphere_camera(rng)
        prm = {"width": W, "height": H, "step": 1 / 256, "max_opacity": 0.99, "ref_step": 1 / 16, "shading": 1}
        mid = ctx.load_model(ctrl, p, storage=storage)
        out.append({"model_id": mid, "camera": cam, "params": prm, "tf": tf, "ctrl": ctrl, "p": p,
                    "tf_dev": torch.from_numpy(tf).to(dev), "tf_size": tf.shape[0],
                    "rgba_dev": torch.full((H, W, 4), float("nan"), device=dev),
                    "nsamples_dev": torch.full((H, W), -1, dtype=torch.int32, device=dev)})
    return out


SPECS = [(3, (40, 36, 44), "f32", (96, 80)), (2, (30, 25, 33), "f32", (61, 47)), (4, (21, 24, 19), "bf16", (64, 64)),
         (3, (33, 29, 31), "f16", (40, 72)), (5, (18, 17, 20), "f32", (48, 40)), (3, (20, 22, 24), "f32", (128, 96)),
         (2, (16, 40, 18), "bf16", (33, 65))]


def test_batch_equals_single_renders(torch_cuda):
    from paper_2204_11762_gb300 import mfadvr
    torch = torch_cuda
    with mfadvr.Context(0) as ctx:
        jobs = _jobs(ctx, torch, SPECS)
        ctx.render_batch(jobs)
        torch.cuda.synchronize()
        batch = [(j["rgba_dev"].cpu().numpy(), j["nsamples_dev"].cpu().numpy()) for j in jobs]
        for j, (img, ns) in zip(jobs, batch):
            ctx.render(j["model_id"], j["camera"], j["params"], j["tf_dev"], j["tf_size"], j["rgba_dev"],
                       j["nsamples_dev"])
            torch.cuda.synchronize()
            np.testing.assert_array_equal(img, j["rgba_dev"].cpu().numpy())
            np.testing.assert_array_equal(ns, j["nsamples_dev"].cpu().numpy())


def test_batch_mixed_shading_equals_single_renders(torch_cuda):
    """Shaded and unshaded jobs of the same degree and storage run in separate
    groups (gradient and value-only kernels); each image equals its single
    render."""
    from paper_2204_11762_gb300 import mfadvr
    torch = torch_cuda
    with mfadvr.Context(0) as ctx:
        jobs = _jobs(ctx, torch, SPECS[:4] + SPECS[:3], seed=11)
        for j in jobs[::2]:
            j["params"] = dict(j["params"], shading=0)
        ctx.render_batch(jobs)
        torch.cuda.synchronize()
        batch = [(j["rgba_dev"].cpu().numpy(), j["nsamples_dev"].cpu().numpy()) for j in jobs]
        for j, (img, ns) in zip(jobs, batch):
            ctx.render(j["model_id"], j["camera"], j["params"], j["tf_dev"], j["tf_size"], j["rgba_dev"],
                       j["nsamples_dev"])
            torch.cuda.synchronize()
            np.testing.assert_array_equal(img, j["rgba_dev"].cpu().numpy())
            np.testing.assert_array_equal(ns, j["nsamples_dev"].cpu().numpy())


def test_batch_against_oracle(torch_cuda, orc):
    from _parity import dequantize
    from paper_2204_11762_gb300 import mfadvr
    torch = torch_cuda
    with mfadvr.Context(0) as ctx:
        jobs = _jobs(ctx, torch, SPECS[:4], seed=9)
        ctx.render_batch(jobs)
        torch.cuda.synchronize()
        for j, (p, n, storage, _) in zip(jobs, SPECS[:4]):
            deq = dequantize(j["ctrl"], storage)
            prm = dict(j["params"], tf=j["tf"], tf_lo=float(j["ctrl"].min()), tf_hi=float(j["ctrl"].max()))
            ref = orc.render(deq, p, j["camera"], prm)
            assert_render_parity(j["rgba_dev"].cpu().numpy(), j["nsamples_dev"].cpu().numpy(), ref)


def test_batch_of_one_and_repeated_models(torch_cuda):
    from paper_2204_11762_gb300 import mfadvr
    torch = torch_cuda
    with mfadvr.Context(0) as ctx:
        jobs = _jobs(ctx, torch, SPECS[:1])
        # the same model seen three times, from its own camera and two others
        extra = []
        for k, cam in enumerate([{"kind": 1, "eye": (2.1, 0.3, 1.2)}, {"kind": 0, "eye": (0.5, -1.0, 0.5),
                                                                        "up": (0, 0, 1), "ortho_height": 1.2}]):
            e = dict(jobs[0], camera=cam)
            e["rgba_dev"] = torch.empty_like(jobs[0]["rgba_dev"])
            e["nsamples_dev"] = torch.empty_like(jobs[0]["nsamples_dev"])
            extra.append(e)
        ctx.render_batch(jobs[:1])
        torch.cuda.synchronize()
        alone = jobs[0]["rgba_dev"].cpu().numpy()
        ctx.render_batch(jobs + extra)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(alone, jobs[0]["rgba_dev"].cpu().numpy())
        for e in extra:
            img = e["rgba_dev"].cpu().numpy()
            ctx.render(e["model_id"], e["camera"], e["params"], e["tf_dev"], e["tf_size"], e["rgba_dev"])
            torch.cuda.synchronize()
            np.testing.assert_array_equal(img, e["rgba_dev"].cpu().numpy())


def test_batch_rejects_bad_jobs(torch_cuda):
    from paper_2204_11762_gb300 import mfadvr
    torch = torch_cuda
    with mfadvr.Context(0) as ctx:
        jobs = _jobs(ctx, torch, SPECS[:2])
        bad = dict(jobs[1], model_id=999)
        with pytest.raises(mfadvr.MfadvrError) as e:
            ctx.render_batch([jobs[0], bad])
        assert e.value.status == mfadvr.ENOTFOUND
        one_entry = dict(jobs[1], tf_size=1)
        with pytest.raises(mfadvr.MfadvrError) as e:
            ctx.render_batch([jobs[0], one_entry])
        assert e.value.status == mfadvr.EINVAL
        with pytest.raises(mfadvr.MfadvrError) as e:
            ctx.render_batch([])
        assert e.value.status == mfadvr.EINVAL


def test_autotune_picks_a_shape_and_keeps_images(torch_cuda, tmp_path):
    from paper_2204_11762_gb300 import mfadvr
    torch = torch_cuda
    with mfadvr.Context(0) as ctx:
        jobs = _jobs(ctx, torch, SPECS[5:6])
        j = jobs[0]
        ctx.render(j["model_id"], j["camera"], j["params"], j["tf_dev"], j["tf_size"], j["rgba_dev"])
        torch.cuda.synchronize()
        before = j["rgba_dev"].cpu().numpy()
        best = ctx.autotune(j["model_id"], j["camera"], j["params"], j["tf_dev"], j["tf_size"], j["rgba_dev"])
        assert best["tile_w"] in (1, 2, 4, 8, 16, 32) and best["ctas_per_sm"] >= 0 and best["ms"] > 0
        ctx.render(j["model_id"], j["camera"], j["params"], j["tf_dev"], j["tf_size"], j["rgba_dev"])
        torch.cuda.synchronize()
        np.testing.assert_array_equal(before, j["rgba_dev"].cpu().numpy())
        path = os.path.join(tmp_path, "tuning.txt")
        ctx.tuning_save(path)
        line = open(path).read().split()
        assert int(line[4]) == best["tile_w"] and int(line[5]) == best["ctas_per_sm"]
    with mfadvr.Context(0) as ctx2:
        ctx2.tuning_load(path)
        open(path, "w").write("3 0 1 2 nonsense\n")
        with pytest.raises(mfadvr.MfadvrError):
            ctx2.tuning_load(path)


@pytest.mark.parametrize("kind", ["f32_power", "f32_bspline", "f16", "bf16", "p2", "p4", "p5", "graded_knots",
                                  "rational", "shading_off"])
def test_tile_order_leaves_every_kernel_kind_unchanged(torch_cuda, kind):
    """mfadvr_render takes the tiles of a 640 x 480 image (9600 tiles of 8 x 4)
    costliest first; mfadvr_render_batch takes them in job order.  Every
    render kernel kind gives the same bits both ways."""
    from paper_2204_11762_gb300 import mfadvr, workloads
    torch = torch_cuda
    rng = np.random.default_rng(910)
    p = {"p2": 2, "p4": 4, "p5": 5}.get(kind, 3)
    n = (23, 21, 25)
    ctrl = workloads.gaussian_sum_lattice(n, p, rng)
    kw = {}
    if kind in ("f16", "bf16"):
        kw["storage"] = kind
    if kind == "f32_bspline":
        kw["render_form"] = mfadvr.FORM_BSPLINE
    if kind == "graded_knots":
        kw["knots"] = [workloads.graded_knots(rng, n[a], p) for a in range(3)]
    if kind == "rational":
        kw["weights"] = rng.uniform(0.5, 2.0, size=ctrl.shape).astype(np.float32)
    tf = workloads.transfer_function(rng, 128)
    W, H = 640, 480
    prm = {"width": W, "height": H, "step": 1 / 128, "max_opacity": 0.97, "ref_step": 1 / 16,
           "shading": 0 if kind == "shading_off" else 1}
    dev = torch.device("cuda:0")
    with mfadvr.Context(0) as ctx:
        mid = ctx.load_model(ctrl, p, **kw)
        cam = workloads.sphere_camera(rng, fovy_deg=45.0)
        job = {"model_id": mid, "camera": cam, "params": prm, "tf_dev": torch.from_numpy(tf).to(dev),
               "tf_size": tf.shape[0], "rgba_dev": torch.full((H, W, 4), float("nan"), device=dev),
               "nsamples_dev": torch.full((H, W), -1, dtype=torch.int32, device=dev)}
        ctx.render_batch([job])
        torch.cuda.synchronize()
        img_b, ns_b = job["rgba_dev"].cpu().numpy(), job["nsamples_dev"].cpu().numpy()
        img = torch.full((H, W, 4), float("nan"), device=dev)
        ns = torch.full((H, W), -1, dtype=torch.int32, device=dev)
        ctx.render(mid, cam, prm, job["tf_dev"], tf.shape[0], img, ns)
        torch.cuda.synchronize()
        assert (ns_b > 0).mean() > 0.2
        np.testing.assert_array_equal(img.cpu().numpy(), img_b)
        np.testing.assert_array_equal(ns.cpu().numpy(), ns_b)


def test_ordered_batch_of_several_jobs_equals_single_renders(torch_cuda):
    """Three degree-3 jobs of different sizes, models and cameras in one
    launch (20800 tiles of 8 x 4: the group takes its tiles costliest first,
    each tile's cost from its own job's camera), and a degree-2 group with
    them: every image equals mfadvr_render's bit for bit."""
    from paper_2204_11762_gb300 import mfadvr
    torch = torch_cuda
    specs = [(3, (40, 36, 44), "f32", (640, 480)), (3, (30, 33, 28), "f32", (480, 320)),
             (3, (24, 26, 22), "f32", (512, 400)), (2, (30, 25, 33), "f32", (300, 200))]
    with mfadvr.Context(0) as ctx:
        jobs = _jobs(ctx, torch, specs, seed=17)
        ctx.render_batch(jobs)
        torch.cuda.synchronize()
        batch = [(j["rgba_dev"].cpu().numpy(), j["nsamples_dev"].cpu().numpy()) for j in jobs]
        for j, (img, ns) in zip(jobs, batch):
            assert not np.isnan(img).any() and (ns >= 0).all()
            ctx.render(j["model_id"], j["camera"], j["params"], j["tf_dev"], j["tf_size"], j["rgba_dev"],
                       j["nsamples_dev"])
            torch.cuda.synchronize()
            np.testing.assert_array_equal(img, j["rgba_dev"].cpu().numpy())
            np.testing.assert_array_equal(ns, j["nsamples_dev"].cpu().numpy())
