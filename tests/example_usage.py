"""The library's usage example: load a model, query points, render a frame.
README.md quotes this file; tests/test_gpu_eval.py runs it."""
import numpy as np, torch
from paper_2204_11762_gb300 import mfadvr, workloads

rng = np.random.default_rng(0)
ctrl = workloads.gaussian_sum_lattice((64, 64, 64), 3, rng)   # (n_w, n_v, n_u) float32
with mfadvr.Context(0) as ctx:
    mid = ctx.load_model(ctrl, 3)                             # storage=, knots=, weights=, render_form=
    pts = torch.rand(1 << 20, 3, device="cuda")
    out = torch.empty(1 << 20, 4, device="cuda")              # f, df/du, df/dv, df/dw
    ctx.eval_points(mid, pts, pts.shape[0], out)
    tf = torch.from_numpy(workloads.transfer_function(rng, 256)).cuda()
    img = torch.empty(512, 512, 4, device="cuda")
    ctx.render(mid, workloads.sphere_camera(rng),
               {"width": 512, "height": 512, "step": 1 / 1024, "max_opacity": 0.99, "shading": 1},
               tf, 256, img)
