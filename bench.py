#!/usr/bin/env python
"""Benchmark of the MFA-DVR hot path on GB300.

One step = one pass of the whole path over one batch of synthetic input:
  * mfadvr_render of the 1024^2 perspective frame of the degree-3, 128^3
    Gaussian-sum model (ray definition, box intersection, samples at step
    1/1024, span lookup, basis + derivatives, (p+1)^3 contraction, TF, Phong
    shading, front-to-back compositing with early termination), and
  * mfadvr_eval_points on 2^24 uniform parameter points (value + gradient).
The metric counts value+gradient queries: render samples actually composited
(exact, from the per-pixel sample counts) plus evaluated points, per second.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# DRAM bytes (read + write) of one render_kernel<3, PolyF32> launch (the power
# form) on the 128^3 workload from one ncu capture
# (profiles/render_kernel_gauss128_p3_persp1024.md), valid only for the kernel
# sources it was taken on.
RENDER_TRAFFIC = {"sources_sha256_16": "98fa770bb15a0f88", "bytes": 537079040}
RENDER_SOURCES = ("paper_2204_11762_gb300/csrc/render_kernels.cuh", "paper_2204_11762_gb300/csrc/mfa_basis.cuh",
                  "paper_2204_11762_gb300/csrc/mfa_internal.h")

METRIC = "MFA value+grad samples/s"
UNIT = "samples/s"
C_FMA = {p: 2 * (p + 1) ** 3 + 3 * (p + 1) ** 2 + 4 * (p + 1) for p in range(1, 6)}
# multiply-adds the power render form executes per value+gradient sample
# (Horner in u on packed pairs, padded when p is even, then in v and w)
POLY_FMA = {p: 2 * (p + 1) * ((p + 2) // 2) * (2 * p - 1) + (p + 1) * (3 * p - 1) + 4 * p - 1 for p in (1, 2, 3, 4)}
FORMS = {"auto": 0, "bspline": 1, "power": 2}
FP32_LANES_PER_SM = 128


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--form", default="auto", choices=sorted(FORMS),
                    help="render form of the model: span polynomials (power) or the B-spline basis")
    ap.add_argument("--workload", default="gauss128",
                    choices=["gauss128", "ml32", "noise512", "multi16", "serve48", "sweep", "variants"],
                    help="gauss128: 128^3 degree-3 render + 2^24 points (default); "
                         "ml32: the 32^3 Marschner-Lobb frame at 128x128, with the oracle's full frame; "
                         "noise512: 512^3 degree-4 render at 3840x2160; "
                         "multi16: one batched render of 16 models of degree 2-5; "
                         "serve48: 2000 Poisson requests over 48 resident models through the serving loop; "
                         "sweep: value / gradient / combined query time vs lattice size and degree; "
                         "variants: the default frame and points per storage, shading, knot kind, weights, query")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the 16-bit storage comparison")
    ap.add_argument("--image", type=int, default=0,
                    help="default workload: square frame of this side instead of 1024 (profiling small cases)")
    ap.add_argument("--no-configs", action="store_true",
                    help="default workload: skip the ml32, noise512 and serving-slice legs of the line")
    ap.add_argument("--serve-step", type=float, default=1.0 / 512, help="serve48: sample step")
    ap.add_argument("--serve-batch", type=int, default=32, help="serve48: requests per scheduling step")
    ap.add_argument("--serve-flights", type=int, default=3, help="serve48: batches in flight")
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def render_traffic():
    """ncu DRAM bytes per render launch, or None once the kernel changed."""
    import hashlib
    h = hashlib.sha256()
    try:
        for f in RENDER_SOURCES:
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
    except OSError:
        return None
    return RENDER_TRAFFIC["bytes"] if h.hexdigest()[:16] == RENDER_TRAFFIC["sources_sha256_16"] else None


def max_over_ranks(x: float, device=None) -> float:
    """Max of a per-rank float over the process group (identity at N = 1)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank_step: int, steps: int, max_ms: float, world: int) -> float:
    """Units all ranks processed / the slowest rank's timed region (weak
    scaling: every rank runs the same per-GPU workload)."""
    return world * units_per_rank_step * steps / (max_ms / 1000.0)


def measure_fma_peak(torch, dev, stream, iters=4096, reps=3):
    """FP32 multiply-add throughput of this GPU from the library's probe
    (mfadvr_probe_fma): best of `reps` launches, scalar and packed, timed with
    CUDA events on `stream`.  Returns TFLOP/s (2 FLOP per multiply-add) per
    form and the best."""
    from paper_2204_11762_gb300 import mfadvr
    sink = torch.zeros(1, dtype=torch.float32, device=dev)
    out = {}
    for packed in (False, True):
        best = 0.0
        for _ in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fmas = mfadvr.probe_fma(sink, iters, packed=packed, stream=stream)
            e1.record(stream)
            e1.synchronize()
            best = max(best, fmas * 2 / (e0.elapsed_time(e1) / 1000.0) / 1e12)
        out["packed" if packed else "scalar"] = best
    out["best"] = max(out.values())
    return out


def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [l.strip().split(", ") for l in self.file.read().splitlines() if l.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip() == "Active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on host cores
# ---------------------------------------------------------------------------

def _oracle_sample(wl, row_step, npts):
    """Oracle on every row_step-th row of the frame and the first npts points;
    returns (queries, seconds)."""
    import oracle
    t0 = time.perf_counter()
    r = oracle.render(wl["ctrl"], wl["degree"], wl["camera"], dict(wl["params"], tf=wl["tf"]), row_step=row_step)
    t1 = time.perf_counter()
    oracle.eval_points(wl["ctrl"], wl["degree"], wl["points"][:npts], with_spans=False)
    t2 = time.perf_counter()
    rs = int(r["nsamples"][::row_step].sum())
    return rs + npts, t2 - t0, rs, t1 - t0, t2 - t1


def run_reference(args, wl):
    rank, world, _ = _dist()
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    row_step, npts = 16, 1 << 20
    for _ in range(args.warmup):
        _oracle_sample(wl, row_step, npts)
    tot_q, tot_t = 0, 0.0
    for _ in range(args.steps):
        q, t, *_ = _oracle_sample(wl, row_step, npts)
        tot_q += q
        tot_t += t
    value = tot_q / tot_t
    sample = f"every {row_step}th row of the 1024^2 frame + the first 2^20 of the 2^24 points, per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(wl, args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _config(wl, args):
    return {"workload": f"gauss20_128cube_p3: {wl['params']['width']}x{wl['params']['height']} perspective render (60 deg, step 1/1024, O_max 0.99, "
                        "TF 256, opacity ref 1/16, shading) + eval_points on 2^24 uniform points",
            "model": f"MFA degree {wl['degree']}, 128^3 control points, clamped uniform knots",
            "storage": args.storage, "image": f"{wl['params']['width']}x{wl['params']['height']}",
            "eval_points": 1 << 24,
            "l2": "flushed between steps (256 MiB write outside the timed events)",
            "parallelism": f"replicas x{args.gpus} (independent frames per GPU)"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args, wl):
    import numpy as np
    import torch

    from paper_2204_11762_gb300 import mfadvr

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    ctx = mfadvr.Context(local)
    p = wl["degree"]
    mid = ctx.load_model(wl["ctrl"], p, storage=args.storage, render_form=FORMS[args.form])
    rows_bytes = int(np.prod(wl["ctrl"].shape)) * 32
    form = "power" if ctx.model_info(mid)["bytes"] > rows_bytes else "bspline"
    pts = wl["points"]
    npts = pts.shape[0]
    prm = wl["params"]
    W, H = prm["width"], prm["height"]
    d_pts = torch.from_numpy(pts).to(dev)
    d_out = torch.empty((npts, 4), dtype=torch.float32, device=dev)
    d_tf = torch.from_numpy(wl["tf"]).to(dev)
    d_img = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    d_ns = torch.empty((H, W), dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(m=mid):
        ctx.render(m, wl["camera"], prm, d_tf, wl["tf"].shape[0], d_img, d_ns, stream=stream)
        ctx.eval_points(m, d_pts, npts, d_out, None, stream=stream)

    # launch shape of the frame from the library's autotuner (untimed set-up;
    # later renders of this model and image size use the tuned shape)
    tuned = ctx.autotune(mid, wl["camera"], prm, d_tf, wl["tf"].shape[0], d_img, d_ns, stream=stream)
    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        step()
    torch.cuda.synchronize(dev)
    render_samples = int(d_ns.sum(dtype=torch.int64).item())

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize(dev)
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        ctx.render(mid, wl["camera"], prm, d_tf, wl["tf"].shape[0], d_img, d_ns, stream=stream)
        ev[k][1].record(stream)
        ctx.eval_points(mid, d_pts, npts, d_out, None, stream=stream)
        ev[k][2].record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    wall1 = time.perf_counter()
    clk = clocks.stop()
    render_ms = [e[0].elapsed_time(e[1]) for e in ev]
    eval_ms = [e[1].elapsed_time(e[2]) for e in ev]
    total_ms = sum(render_ms) + sum(eval_ms)
    fma_probe = measure_fma_peak(torch, dev, stream)  # after the timed region, same stream and clocks
    assert int(d_ns.sum(dtype=torch.int64).item()) == render_samples, "sample count changed between steps"

    total_ms = max_over_ranks(total_ms, dev)
    units_per_step = render_samples + npts
    value = whole_job_value(units_per_step, args.steps, total_ms, world)

    # ---- roofline of the dominant kernel (render: FP32 FMA pipe) ---------
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peaks = _measured_peaks()
    sm_max_mhz = (clk or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
    fma_peak_tflops = sms * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
    r_mean = statistics.mean(render_ms)
    e_mean = statistics.mean(eval_ms)
    render_tflops = render_samples * C_FMA[p] * 2 / (r_mean / 1000.0) / 1e12
    eval_tflops = npts * C_FMA[p] * 2 / (e_mean / 1000.0) / 1e12
    eval_io_bytes = npts * (12 + 16)
    dominant = "render" if r_mean >= e_mean else "eval_points"
    if dominant == "render":
        roof = {"kernel": "render_kernel", "bound": "alu", "achieved": render_tflops, "peak": fma_peak_tflops,
                "unit": "TFLOP/s", "frac": render_tflops / fma_peak_tflops,
                "traffic": render_traffic() if form == "power" else None,
                "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2 FLOP x {sm_max_mhz:.0f} MHz",
                "per_unit": f"{C_FMA[p]} FMA per sample (sum-factorised contraction, degree {p})",
                "render_form": form}
        roof["measured_peak"] = {"tflops": fma_probe["best"], "frac": render_tflops / fma_probe["best"],
                                 "scalar_tflops": fma_probe["scalar"], "packed_tflops": fma_probe["packed"],
                                 "source": "measured on this GPU in this run: mfadvr_probe_fma (8 independent "
                                           "FMA chains per thread, full occupancy), best of 3 launches per form, "
                                           "CUDA events on the bench stream right after the timed region"}
        if form == "power":
            ex = render_samples * POLY_FMA[p] * 2 / (r_mean / 1000.0) / 1e12
            roof["executed"] = {"fma_per_sample": POLY_FMA[p], "tflops": ex, "frac": ex / fma_peak_tflops,
                                "note": "the power form evaluates each cell's polynomial by Horner sums: "
                                        "an algebraic shortcut, so achieved/frac keep the algorithmic count"}
    else:
        roof = {"kernel": "eval_points_kernel", "bound": "alu", "achieved": eval_tflops, "peak": fma_peak_tflops,
                "unit": "TFLOP/s", "frac": eval_tflops / fma_peak_tflops, "traffic": None,
                "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2 FLOP x {sm_max_mhz:.0f} MHz",
                "per_unit": f"{C_FMA[p]} FMA per point"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.storage == "f32" else
            f"f32 (storage {args.storage})", "data": "synthetic", "config": _config(wl, args),
            "gpu_launches": 4 * args.steps,  # tile costs, tile order, render, point query
            "frames_per_s": world * 1000.0 / r_mean,
            "render": {"samples_per_frame": render_samples, "ms_mean": r_mean,
                       "ms_p50": statistics.median(render_ms),
                       "ms_p99": sorted(render_ms)[min(len(render_ms) - 1, int(0.99 * len(render_ms)))],
                       "samples_per_s": render_samples / (r_mean / 1000.0), "tflops": render_tflops},
            "eval_points": {"points": npts, "ms_mean": e_mean, "points_per_s": npts / (e_mean / 1000.0),
                            "tflops": eval_tflops, "io_gbs": eval_io_bytes / (e_mean / 1000.0) / 1e9,
                            "fma_frac": eval_tflops / fma_peak_tflops,
                            "hbm_frac": (eval_io_bytes / (e_mean / 1000.0) / 1e9) / peaks["hbm_gbs"]
                            if "hbm_gbs" in peaks else None},
            "roofline": roof, "clocks": clk, "wall_s": wall1 - wall0}
    line["config"]["render_form"] = (f"{form}: span polynomials, Horner sums" if form == "power" else
                                     f"{form}: basis and sum-factorised contraction")
    line["config"]["launch"] = (f"{tuned['tile_w']}x{32 // tuned['tile_w']} ray tiles, "
                                f"{tuned['ctas_per_sm'] or 'max'} CTAs/SM (library autotuner, untimed set-up)")

    # ---- mixed precision: same step with 16-bit storage ------------------
    if not args.no_mixed and args.storage == "f32":
        mixed = {}
        for st in ("f16", "bf16"):
            m2 = ctx.load_model(wl["ctrl"], p, storage=st)
            ctx.autotune(m2, wl["camera"], prm, d_tf, wl["tf"].shape[0], d_img, d_ns, stream=stream)
            for _ in range(3):
                flush.zero_()
                step(m2)
            ev2 = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
            for k in range(args.steps):
                flush.zero_()
                ev2[k][0].record(stream)
                ctx.render(m2, wl["camera"], prm, d_tf, wl["tf"].shape[0], d_img, d_ns, stream=stream)
                ev2[k][1].record(stream)
                ctx.eval_points(m2, d_pts, npts, d_out, None, stream=stream)
                ev2[k][2].record(stream)
            torch.cuda.synchronize(dev)
            rs2 = int(d_ns.sum(dtype=torch.int64).item())
            rm = statistics.mean([e[0].elapsed_time(e[1]) for e in ev2])
            em = statistics.mean([e[1].elapsed_time(e[2]) for e in ev2])
            mixed[st] = {"value": (rs2 + npts) / ((rm + em) / 1000.0), "render_ms": rm, "eval_ms": em,
                         "render_samples_per_s": rs2 / (rm / 1000.0)}
            ctx.unload_model(m2)
        line["mixed_precision"] = mixed

    # ---- end to end through the host-buffer entry points -----------------
    if not args.no_e2e:
        h_pts = torch.from_numpy(pts).pin_memory()
        h_out = torch.empty((npts, 4), dtype=torch.float32).pin_memory()
        h_img = torch.empty((H, W, 4), dtype=torch.float32).pin_memory()
        h_tf = torch.from_numpy(wl["tf"]).pin_memory()
        tf_np = h_tf.numpy()
        img_np = h_img.numpy()
        k2 = max(3, min(args.steps, 10))
        # One step: the point query, queued first on its own stream, reads the
        # points from and writes the results to the pinned buffers over the
        # host link on a few SMs; the frame renders beside it on the others
        # and is written to the pinned image.  Both calls are the library's
        # host-buffer entry points; the step ends when both streams are done.
        q_stream = torch.cuda.Stream(device=dev)

        def e2e_step(cap):
            ctx.query_points_host_async(mid, h_pts, npts, h_out, max_ctas=cap, stream=q_stream.cuda_stream)
            ctx.render_host(mid, wl["camera"], prm, tf_np, rgba=img_np, stream=stream)
            q_stream.synchronize()

        # untimed set-up: the share of the GPU the point query gets
        trial = {}
        for cap in (16, 24, 32, 48, 64, 0):
            e2e_step(cap)
            t0 = time.perf_counter()
            for _ in range(3):
                e2e_step(cap)
            trial[cap] = time.perf_counter() - t0
        cap = min(trial, key=trial.get)
        for _ in range(2):
            e2e_step(cap)
        barrier()
        t0 = time.perf_counter()
        for _ in range(k2):
            e2e_step(cap)
        t1 = time.perf_counter()
        dt = max_over_ranks(t1 - t0, dev)
        line["e2e"] = {"value": whole_job_value(units_per_step, k2, dt * 1000.0, world), "unit": UNIT,
                       "h2d_bytes_per_step": npts * 12 + wl["tf"].nbytes,
                       "d2h_bytes_per_step": npts * 16 + H * W * 16, "steps": k2,
                       "ms_per_step": 1000 * dt / k2,
                       "overlap": {"query_max_ctas": cap, "query_stream": "separate, queued before the frame"}}

    # ---- CPU baseline: the oracle on a bounded sample, rank 0 at N = 1 ---
    if not args.no_cpu_baseline and world == 1:
        q, t, rs, tr, te = _oracle_sample(wl, 2, 1 << 22)
        line["cpu_baseline"] = {"value": q / t, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
                                "sample": "every 2nd row of the 1024^2 frame + the first 2^22 of the 2^24 points",
                                "render_samples_per_s": rs / tr, "eval_points_per_s": (1 << 22) / te}

    ctx.close()
    del d_pts, d_out, d_img, d_ns
    torch.cuda.empty_cache()

    # ---- the other named configurations, bounded, rank 0 at N = 1 --------
    if not args.no_configs and world == 1:
        t0 = time.perf_counter()
        configs = {"ml32": leg_ml32(torch, dev, local, flush, stream)}
        configs["noise512"] = leg_noise512(torch, dev, local, flush, stream)
        torch.cuda.empty_cache()
        configs["serve_slice"] = leg_serve_slice(torch, dev, local, args)
        configs["wall_s"] = time.perf_counter() - t0
        line["configs"] = configs
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_noise512(args, wl):
    """Render-only step: the 512^3 degree-4 value-noise model at 3840x2160,
    step 1/2048, TF 1024; FP32 and BF16 storage."""
    import torch

    from paper_2204_11762_gb300 import mfadvr

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    ctx = mfadvr.Context(local)
    p = wl["degree"]
    prm = wl["params"]
    W, H = prm["width"], prm["height"]
    d_tf = torch.from_numpy(wl["tf"]).to(dev)
    d_img = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    d_ns = torch.empty((H, W), dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    steps = max(3, min(args.steps, 40))
    out = {}
    for st in ("f32", "bf16"):
        # FP32 with --form auto renders in the power form here too: its cells
        # (84 GB) exceed AUTO's 4 GiB default, so the form is requested
        form = FORMS["power"] if st == "f32" and args.form == "auto" else FORMS[args.form]
        mid = ctx.load_model(wl["ctrl"], p, storage=st, render_form=form if st == "f32" else FORMS["auto"])
        # untimed set-up: the library's autotuner picks the launch shape
        ctx.autotune(mid, wl["camera"], prm, d_tf, wl["tf"].shape[0], d_img, d_ns, stream=stream)
        for _ in range(max(args.warmup, 3) if st == "f32" else 2):
            flush.zero_()
            ctx.render(mid, wl["camera"], prm, d_tf, wl["tf"].shape[0], d_img, d_ns, stream=stream)
        torch.cuda.synchronize(dev)
        samples = int(d_ns.sum(dtype=torch.int64).item())
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        clocks = ClockSampler(local)
        clocks.start()
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            ctx.render(mid, wl["camera"], prm, d_tf, wl["tf"].shape[0], d_img, d_ns, stream=stream)
            b.record(stream)
        torch.cuda.synchronize(dev)
        clk = clocks.stop()
        ms = [a.elapsed_time(b) for a, b in ev]
        out[st] = {"samples": samples, "ms": ms, "clocks": clk}
        ctx.unload_model(mid)
    r = out["f32"]
    r_ms = statistics.mean(r["ms"])
    total_ms = max_over_ranks(sum(r["ms"]), dev)
    value = whole_job_value(r["samples"], steps, total_ms, world)
    props = torch.cuda.get_device_properties(dev)
    clk = r["clocks"] or {}
    sm_max = clk.get("sm_max_mhz") or _measured_peaks().get("sm_max_mhz") or 2070.0
    peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    tflops = r["samples"] * C_FMA[p] * 2 / (r_ms / 1000.0) / 1e12
    b = out["bf16"]
    b_ms = statistics.mean(b["ms"])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": total_ms / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "noise512_p4: 3840x2160 perspective render (60 deg, step 1/2048, O_max 0.99, "
                                   "TF 1024, opacity ref 1/16, shading)",
                       "model": "MFA degree 4, 512^3 control points (5-octave value noise), clamped uniform knots",
                       "l2": "flushed between steps; the 4 GiB FP32 row array exceeds L2"},
            "gpu_launches": 3 * steps,  # tile costs, tile order, render
            "frames_per_s": world * 1000.0 / r_ms,
            "render": {"samples_per_frame": r["samples"], "ms_mean": r_ms, "ms_p50": statistics.median(r["ms"]),
                       "ms_p99": sorted(r["ms"])[min(len(r["ms"]) - 1, int(0.99 * len(r["ms"])))]},
            "roofline": {"kernel": "render_kernel<4, PolyF32>" if args.form != "bspline" else "render_kernel<4, float>",
                         "bound": "alu", "achieved": tflops, "peak": peak,
                         "unit": "TFLOP/s", "frac": tflops / peak, "traffic": None,
                         "per_unit": f"{C_FMA[p]} FMA per sample (degree {p})"},
            "mixed_precision": {"bf16": {"render_ms": b_ms, "samples_per_s": b["samples"] / (b_ms / 1000.0),
                                         "samples_per_frame": b["samples"], "vs_f32": r_ms / b_ms}},
            "clocks": r["clocks"]}
    ctx.close()
    if not args.no_cpu_baseline and world == 1:
        # the oracle on every 64th row of the frame, on all host cores
        import oracle
        oracle.build()
        row_step = 64
        t0 = time.perf_counter()
        ro = oracle.render(wl["ctrl"], p, wl["camera"], dict(prm, tf=wl["tf"]), row_step=row_step)
        t = time.perf_counter() - t0
        rs = int(ro["nsamples"][::row_step].sum())
        line["cpu_baseline"] = {"value": rs / t, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
                                "sample": f"every {row_step}th row of the 3840x2160 frame ({rs} samples, {t:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_ml32(args, wl):
    """The small case: the 32^3 degree-3 Marschner-Lobb model (Eq. 2) at
    128x128 orthographic, step 1/256.  Render time on the GPU (launch shape
    from the autotuner), the oracle's full frame on the host cores, and the
    largest pixel difference between the two (either branch of a tied
    decision accepted)."""
    import numpy as np
    import torch

    import oracle
    from paper_2204_11762_gb300 import mfadvr

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = mfadvr.Context(local)
    p, prm = wl["degree"], wl["params"]
    W, H = prm["width"], prm["height"]
    d_tf = torch.from_numpy(wl["tf"]).to(dev)
    d_img = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    d_ns = torch.empty((H, W), dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    mid = ctx.load_model(wl["ctrl"], p)
    ctx.autotune(mid, wl["camera"], prm, d_tf, wl["tf"].shape[0], d_img, d_ns, stream=stream)
    steps = max(3, args.steps)
    for _ in range(max(args.warmup, 3)):
        ctx.render(mid, wl["camera"], prm, d_tf, wl["tf"].shape[0], d_img, d_ns, stream=stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    clocks = ClockSampler(local)
    clocks.start()
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        ctx.render(mid, wl["camera"], prm, d_tf, wl["tf"].shape[0], d_img, d_ns, stream=stream)
        b.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    img, ns = d_img.cpu().numpy(), d_ns.cpu().numpy()
    samples = int(ns.sum(dtype=np.int64))
    ctx.close()
    oracle.build()
    t0 = time.perf_counter()
    ref = oracle.render(wl["ctrl"], p, wl["camera"], dict(prm, tf=wl["tf"]))
    t_oracle = time.perf_counter() - t0
    err = np.minimum(np.abs(img - ref["rgba"]).max(-1), np.abs(img - ref["rgba_alt"]).max(-1))
    r_ms = statistics.mean(ms)
    line = {"metric": METRIC, "value": samples / (r_ms / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "ms_per_step": r_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "ml32_p3: 128x128 orthographic render of the 32^3 Marschner-Lobb model "
                                   "(Eq. 2, f_M 6, alpha 0.25, + N(0, 0.01)), step 1/256, TF 256, shading",
                       "l2": "flushed between steps (the model fits L2)"},
            "gpu_launches": 3 * steps,  # tile costs, tile order, render
            "render": {"samples_per_frame": samples, "ms_mean": r_ms, "ms_p50": statistics.median(ms)},
            "parity": {"max_pixel_err": float(err.max()), "tolerance": 2e-3},
            "cpu_baseline": {"value": int(ref["nsamples"].sum()) / t_oracle, "unit": UNIT,
                             "cores": os.cpu_count() or 1, "kind": "oracle",
                             "sample": f"the full frame ({t_oracle:.2f} s)"},
            "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_multi16(args, jobs):
    """One mfadvr_render_batch call over 16 models (degrees 2-5, lattices
    64..256 per axis, images 512^2..2048^2), launch shapes from the
    autotuner, under FP32, FP16 and BF16 storage; errors against the FP64
    oracle on bounded samples (4096 points per model for value/gradient,
    every 128th row of every image for pixels)."""
    import numpy as np
    import torch

    import oracle
    from paper_2204_11762_gb300 import mfadvr

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    steps = max(3, min(args.steps, 20))
    rng = np.random.default_rng(7)
    pts = [rng.uniform(0, 1, size=(4096, 3)).astype(np.float32) for _ in jobs]
    ref_eval, ref_img = [], []
    for j, pp in zip(jobs, pts):
        r, _ = oracle.eval_points(j["ctrl"], j["degree"], pp)
        ref_eval.append(r)
        ref_img.append(oracle.render(j["ctrl"], j["degree"], j["camera"], dict(j["params"], tf=j["tf"]),
                                     row_step=128))
    results = {}
    for st in ("f32", "f16", "bf16"):
        ctx = mfadvr.Context(local)
        batch, tunes = [], []
        for j in jobs:
            W, H = j["params"]["width"], j["params"]["height"]
            mid = ctx.load_model(j["ctrl"], j["degree"], storage=st)
            e = {"model_id": mid, "camera": j["camera"], "params": j["params"],
                 "tf_dev": torch.from_numpy(j["tf"]).to(dev), "tf_size": j["tf"].shape[0],
                 "rgba_dev": torch.empty((H, W, 4), device=dev),
                 "nsamples_dev": torch.empty((H, W), dtype=torch.int32, device=dev)}
            tunes.append(ctx.autotune(mid, e["camera"], e["params"], e["tf_dev"], e["tf_size"], e["rgba_dev"],
                                      e["nsamples_dev"], stream=stream))
            batch.append(e)
        for _ in range(3):
            flush.zero_()
            ctx.render_batch(batch, stream=stream)
        torch.cuda.synchronize(dev)
        samples = sum(int(e["nsamples_dev"].sum(dtype=torch.int64).item()) for e in batch)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            ctx.render_batch(batch, stream=stream)
            b.record(stream)
        torch.cuda.synchronize(dev)
        ms = [a.elapsed_time(b) for a, b in ev]
        # errors against the FP64 oracle of the FP32 lattice
        verr, gerr, perr = [], [], []
        for j, e, pp, r, ri in zip(jobs, batch, pts, ref_eval, ref_img):
            d_p = torch.from_numpy(pp).to(dev)
            d_o = torch.empty((pp.shape[0], 4), device=dev)
            ctx.eval_points(e["model_id"], d_p, pp.shape[0], d_o, None, stream=stream)
            torch.cuda.synchronize(dev)
            got = d_o.cpu().numpy().astype(np.float64)
            pabs = float(np.abs(j["ctrl"]).max())
            m = max(int(x) - j["degree"] for x in j["ncp"])
            verr.append(np.abs(got[:, 0] - r[:, 0]) / pabs)
            gerr.append(np.abs(got[:, 1:] - r[:, 1:]).max(axis=1) / (pabs * m))
            img = e["rgba_dev"].cpu().numpy()[::128]
            perr.append(np.abs(img - ri["rgba"][::128]).max(axis=-1).ravel())
        v, g, px = np.concatenate(verr), np.concatenate(gerr), np.concatenate(perr)
        results[st] = {"samples": samples, "ms_mean": statistics.mean(ms), "ms_p50": statistics.median(ms),
                       "samples_per_s": samples / (statistics.mean(ms) / 1000.0),
                       "err_value": {"max": float(v.max()), "rms": float(np.sqrt((v ** 2).mean()))},
                       "err_grad": {"max": float(g.max()), "rms": float(np.sqrt((g ** 2).mean()))},
                       "err_pixel": {"max": float(px.max()), "rms": float(np.sqrt((px ** 2).mean()))},
                       "tuning": [f"{t['tile_w']}x{32 // t['tile_w']}/{t['ctas_per_sm']}" for t in tunes]}
        ctx.close()
        del batch
    f32 = results["f32"]
    line = {"metric": METRIC, "value": f32["samples_per_s"], "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": 3, "ms_per_step": f32["ms_mean"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "multi16: one batched render of 16 models (degree 2-5, lattices 64..256 per "
                                   "axis, Gaussian sums), images 512^2..2048^2, step 1/1024, autotuned shapes",
                       "models": [f"p{j['degree']} {j['ncp'][0]}x{j['ncp'][1]}x{j['ncp'][2]} "
                                  f"{j['params']['width']}^2" for j in jobs],
                       "errors": "value/|P|max, gradient/(|P|max m), pixel abs; vs FP64 oracle of the FP32 "
                                 "lattice; 4096 points per model, every 128th row"},
            "gpu_launches": 4 * steps, "storage": results,
            "mixed_precision": {st: {"samples_per_s": results[st]["samples_per_s"],
                                     "vs_f32": results[st]["samples_per_s"] / f32["samples_per_s"]}
                                for st in ("f16", "bf16")}}
    if rank == 0:
        print(json.dumps(line), flush=True)


SWEEP_DEGREES = (1, 2, 3, 4, 5)
SWEEP_SIZES = (32, 64, 128, 256, 512)
SWEEP_MODES = (("value", 1), ("gradient", 2), ("both", 3), ("hessian", 4))


def run_sweep(args):
    """Query-time sweep of the MFA parameter study (Sec. 4.3.3, Fig. 12): the
    time of one value query, one gradient query, one combined query and one
    Hessian query (Sec. 3.1's higher-order query), per point, for the Gaussian
    beam (Eq. 1) on n^3 control points, n in {32..512}, degrees 1-5, over 2^24
    U[0,1]^3 points (inputs larger than L2).  The headline value is the
    combined query at degree 3 on 256^3, the paper's beam size."""
    import numpy as np
    import torch

    from paper_2204_11762_gb300 import mfadvr, workloads

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    npts = 1 << 24
    steps = max(3, min(args.steps, 20))
    rng = np.random.default_rng(workloads.seed_for(6))
    pts = workloads.uniform_points(rng, npts)
    d_pts = torch.from_numpy(pts).to(dev)
    d_out = torch.empty((npts, 10), device=dev)
    table, launches = {}, 0
    clocks = ClockSampler(local)
    clocks.start()
    with mfadvr.Context(local) as ctx:
        for n in SWEEP_SIZES:
            for p in SWEEP_DEGREES:
                # control points at the degree's Greville abscissae
                mid = ctx.load_model(workloads.gaussian_beam_lattice((n, n, n), p), p)
                row = {}
                for name, q in SWEEP_MODES:
                    for _ in range(3):
                        ctx.query_points(mid, d_pts, npts, d_out, q, stream=stream)
                    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                          for _ in range(steps)]
                    for e0, e1 in ev:
                        e0.record(stream)
                        ctx.query_points(mid, d_pts, npts, d_out, q, stream=stream)
                        e1.record(stream)
                    torch.cuda.synchronize(dev)
                    launches += steps
                    ms = statistics.median(e0.elapsed_time(e1) for e0, e1 in ev)
                    row[name] = {"ns_per_query": ms * 1e6 / npts, "queries_per_s": npts / (ms / 1000.0),
                                 "tflops": npts * _query_fma(p, q) * 2 / (ms / 1000.0) / 1e12}
                table[f"p{p}_n{n}"] = row
                ctx.unload_model(mid)
    clk = clocks.stop()
    head = table["p3_n256"]["both"]
    props = torch.cuda.get_device_properties(dev)
    sm_max = (clk or {}).get("sm_max_mhz") or _measured_peaks().get("sm_max_mhz") or 2070.0
    peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    peak_src = f"derived: {props.multi_processor_count} SMs x 128 FP32 lanes x 2 FLOP x {sm_max:.0f} MHz"
    line = {"metric": METRIC, "value": head["queries_per_s"], "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": 3, "ms_per_step": npts / head["queries_per_s"] * 1000.0, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "sweep: query time of mfadvr_query_points (value / gradient / both / hessian) on the "
                                   "Gaussian beam (Eq. 1) at the Greville abscissae, n^3 control points for n in "
                                   f"{list(SWEEP_SIZES)}, degrees {list(SWEEP_DEGREES)}, 2^24 U[0,1]^3 points; "
                                   "headline: both, degree 3, 256^3",
                       "l2": "inputs larger than L2 (2^24 points: 201 MB in, 268 MB out)"},
            "gpu_launches": launches,
            "roofline": {"kernel": "eval_points_kernel", "bound": "alu", "achieved": head["tflops"], "peak": peak,
                         "unit": "TFLOP/s", "frac": head["tflops"] / peak, "traffic": None,
                         "peak_source": peak_src,
                         "per_unit": "192 FMA per combined query (degree 3); the kernel is bound by the L1/L2 "
                                     "sector rate of the control-point gathers"},
            "clocks": clk, "sweep": table}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_variants(args):
    """The default workload (128^3 Gaussian sum, 1024^2 frame at step 1/1024,
    2^24 points) on each model and query variant the library supports: FP32 /
    FP16 / BF16 storage, FP32 in both render forms (span polynomials, the
    default here, and the B-spline basis), shading off (value-only kernel), graded non-uniform
    knots (span widths U[0.2, 1.8] normalised, all axes), rational weights
    U[0.5, 2], and the value-only, gradient-only and Hessian point queries.
    Render and query times are medians of CUDA-event timings with the L2
    flushed between launches; launch shapes from the autotuner."""
    import numpy as np
    import torch

    from paper_2204_11762_gb300 import mfadvr, workloads

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    wl = workloads.gaussian_sum_workload()
    p, prm = wl["degree"], wl["params"]
    H, W = prm["height"], prm["width"]
    rng = np.random.default_rng(workloads.seed_for(7))
    knots = [workloads.graded_knots(rng, 128, p) for _ in range(3)]
    weights = rng.uniform(0.5, 2.0, size=wl["ctrl"].shape).astype(np.float32)
    npts = wl["points"].shape[0]
    d_pts = torch.from_numpy(wl["points"]).to(dev)
    d_out = torch.empty((npts, 10), device=dev)
    d_tf = torch.from_numpy(wl["tf"]).to(dev)
    d_img = torch.empty((H, W, 4), device=dev)
    d_ns = torch.empty((H, W), dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    steps = max(3, min(args.steps, 20))

    def timed(fn):
        for _ in range(3):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize(dev)
        return statistics.median(a.elapsed_time(b) for a, b in ev)

    variants = [("f32", {}, 1), ("f32 B-spline form", {"render_form": FORMS["bspline"]}, 1),
                ("f16", {"storage": "f16"}, 1), ("bf16", {"storage": "bf16"}, 1),
                ("f32 shading off", {}, 0), ("f32 B-spline form, shading off", {"render_form": FORMS["bspline"]}, 0),
                ("f32 graded knots", {"knots": knots}, 1),
                ("f32 graded knots, B-spline form", {"knots": knots, "render_form": FORMS["bspline"]}, 1),
                ("f32 rational", {"weights": weights}, 1),
                ("f32 rational, B-spline form", {"weights": weights, "render_form": FORMS["bspline"]}, 1)]
    table, launches = {}, 0
    clocks = ClockSampler(local)
    clocks.start()
    with mfadvr.Context(local) as ctx:
        for name, kw, shading in variants:
            mid = ctx.load_model(wl["ctrl"], p, **kw)
            pv = dict(prm, shading=shading)
            ctx.autotune(mid, wl["camera"], pv, d_tf, wl["tf"].shape[0], d_img, d_ns, stream=stream)
            r_ms = timed(lambda: ctx.render(mid, wl["camera"], pv, d_tf, wl["tf"].shape[0], d_img, d_ns,
                                            stream=stream))
            samples = int(d_ns.sum(dtype=torch.int64).item())
            q_ms = timed(lambda: ctx.query_points(mid, d_pts, npts, d_out, 3, stream=stream))
            launches += 4 * steps  # tile costs, tile order, render; point query
            row = {"render_ms": r_ms, "samples": samples, "render_samples_per_s": samples / (r_ms / 1e3),
                   "query_both_ms": q_ms, "query_points_per_s": npts / (q_ms / 1e3)}
            if name == "f32":
                for qn, q in (("value", 1), ("gradient", 2), ("hessian", 4)):
                    ms = timed(lambda: ctx.query_points(mid, d_pts, npts, d_out, q, stream=stream))
                    launches += steps
                    row[f"query_{qn}_ms"] = ms
                    row[f"query_{qn}_tflops"] = npts * _query_fma(p, q) * 2 / (ms / 1e3) / 1e12
            table[name] = row
            ctx.unload_model(mid)
    clk = clocks.stop()
    head = table["f32"]
    props = torch.cuda.get_device_properties(dev)
    sm_max = (clk or {}).get("sm_max_mhz") or _measured_peaks().get("sm_max_mhz") or 2070.0
    peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    tflops = head["samples"] * C_FMA[p] * 2 / (head["render_ms"] / 1e3) / 1e12
    line = {"metric": METRIC, "value": (head["samples"] + npts) / ((head["render_ms"] + head["query_both_ms"]) / 1e3),
            "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": 3,
            "ms_per_step": head["render_ms"] + head["query_both_ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "variants: the 128^3 degree-3 Gaussian-sum frame (1024^2, step 1/1024) and 2^24 "
                                   "points per storage type, shading, knot kind, rational weights and query kind",
                       "l2": "flushed between launches (256 MiB write outside the timed events)"},
            "gpu_launches": launches,
            "roofline": {"kernel": "render_kernel", "bound": "alu", "achieved": tflops, "peak": peak,
                         "unit": "TFLOP/s", "frac": tflops / peak, "traffic": None,
                         "peak_source": f"derived: {props.multi_processor_count} SMs x 128 FP32 lanes x 2 FLOP x "
                                        f"{sm_max:.0f} MHz", "per_unit": f"{C_FMA[p]} FMA per sample"},
            "clocks": clk, "variants": table}
    if rank == 0:
        print(json.dumps(line), flush=True)


def _query_fma(p, mode):
    a = p + 1
    return {1: a ** 3 + a * a + a, 2: 2 * a ** 3 + 3 * a * a + 3 * a, 3: 2 * a ** 3 + 3 * a * a + 4 * a,
            4: 3 * a ** 3 + 6 * a * a + 10 * a}[mode]


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(q * len(xs)))]


def serve_legs(ctx, torch, dev, local, mods, reqs, prm, args, err_requests=0, capacity=False):
    """One request stream through three renderers, each replayed in real time
    (every request submitted at its arrival time): the serving loop with FP16
    models, the serving loop with FP32 models, and serial plain-FP32 rendering
    (one request at a time, synchronously, in arrival order: a request waits
    for all earlier ones).  Latency = completion - arrival.  err_requests > 0:
    the FP16-served images of that many of the stream's 256^2 requests are
    compared with the FP64 oracle of the FP32 lattice (every 2nd row).
    capacity: also the saturated case, every request available at once (the
    stream submitted back to back), for the served FP16 and the serial FP32
    renderers: the samples/s each sustains when the GPU is the bottleneck."""
    import numpy as np

    import oracle
    tfs = [torch.from_numpy(m["tf"]).to(dev) for m in mods]
    pool = 8
    bufs = {side: [(torch.empty((side, side, 4), device=dev), torch.empty((side, side), dtype=torch.int32, device=dev))
                   for _ in range(pool)] for side in sorted({r["side"] for r in reqs})}
    check = [i for i, r in enumerate(reqs) if r["side"] == 256][:err_requests]

    def job(r, ids, rgba, ns):
        return {"model_id": ids[r["model"]], "camera": r["camera"],
                "params": dict(prm, width=r["side"], height=r["side"]), "tf_dev": tfs[r["model"]],
                "tf_size": 256, "rgba_dev": rgba, "nsamples_dev": ns}

    resident = {}  # HBM bytes of the loaded models, per storage type
    kept = {}      # host copies of the checked requests' images

    def served(storage, paced=True):
        ids = [ctx.load_model(m["ctrl"], m["degree"], storage=storage) for m in mods]
        arr = [r["arrival"] if paced else 0.0 for r in reqs]  # unpaced: every request there at once
        resident[storage] = sum(ctx.model_info(i)["bytes"] for i in ids)
        ctx.serve_start(frame_budget_bytes=2 << 30, max_batch=args.serve_batch, max_in_flight=args.serve_flights)
        # the clock sampler starts before the warm-up: its first nvidia-smi
        # start-up on a box can hold the driver for seconds
        clocks = ClockSampler(local)
        clocks.start()
        for k in range(len(mods)):  # warm-up: graphs, every model once
            r = dict(reqs[0], model=k, side=256)
            ctx.wait(ctx.submit(job(r, ids, *bufs[256][k % pool])))
        warm = []  # and an unmeasured burst of the stream's first requests (every size and buffer)
        for i, r in enumerate(reqs[:min(300, len(reqs))]):
            warm.append(ctx.submit(job(r, ids, *bufs[r["side"]][i % pool])))
            if len(warm) >= pool:
                ctx.wait(warm.pop(0))
        for t in warm:
            ctx.wait(t)
        samples = torch.zeros((), dtype=torch.int64, device=dev)
        for side in bufs:  # the client's own reduction kernels load before the replay
            samples += bufs[side][0][1].sum(dtype=torch.int64) * 0
        torch.cuda.synchronize(dev)
        owner = {side: [None] * pool for side in bufs}
        used = {side: 0 for side in bufs}
        submit_t, lat = {}, {}

        def retire(i, side, slot):
            lat[i] = ctx.wait(submit_t[i][1]) / 1e6 + (submit_t[i][0] - arr[i])
            if storage == "f16" and i in check:
                kept[i] = bufs[side][slot][0].cpu().numpy()
            return bufs[side][slot][1].sum(dtype=torch.int64)

        t0 = time.perf_counter()
        for i, r in enumerate(reqs):
            target = t0 + arr[i]
            while True:
                dt = target - time.perf_counter()
                if dt <= 0:
                    break
                if dt > 0.0015:
                    time.sleep(dt - 0.001)
            side = r["side"]
            slot = used[side] % pool
            used[side] += 1
            prev = owner[side][slot]
            rgba, ns = bufs[side][slot]
            if prev is not None:  # the buffer's previous request must be done
                samples += retire(prev, side, slot)
            submit_t[i] = (time.perf_counter() - t0, ctx.submit(job(r, ids, rgba, ns)))
            owner[side][slot] = i
        for side in bufs:
            for slot, prev in enumerate(owner[side]):
                if prev is not None and prev not in lat:
                    samples += retire(prev, side, slot)
        clk = clocks.stop()
        stats = ctx.serve_stats()
        ctx.serve_stop()
        torch.cuda.synchronize(dev)
        for m in ids:
            ctx.unload_model(m)
        n = int(samples.item())
        lats = [lat[i] for i in range(len(reqs))]
        makespan = max(arr[i] + lats[i] for i in range(len(reqs))) - arr[0]
        client_wait = max(submit_t[i][0] - arr[i] for i in range(len(reqs)))
        return {"latency_ms_p50": 1000 * _pct(lats, 0.50), "latency_ms_p99": 1000 * _pct(lats, 0.99),
                "latency_ms_max": 1000 * max(lats), "samples": n, "makespan_s": makespan,
                "samples_per_s": n / makespan, "frames_per_s": len(reqs) / makespan,
                "client_submit_delay_ms_max": 1000 * client_wait, "clocks": clk, **stats}

    srv16 = served("f16")
    srv32 = served("f32")

    # serial plain FP32: one request at a time, synchronously, each started
    # at its arrival (paced) or at once, and when the previous one is done
    ids32 = [ctx.load_model(m["ctrl"], m["degree"]) for m in mods]
    stream = torch.cuda.current_stream(dev)
    for k in range(len(mods)):  # warm-up
        j = job(dict(reqs[0], model=k, side=256), ids32, *bufs[256][0])
        ctx.render(j["model_id"], j["camera"], j["params"], j["tf_dev"], 256, j["rgba_dev"], j["nsamples_dev"],
                   stream=stream)
    torch.cuda.synchronize(dev)

    def serial_run(paced=True):
        arr = [r["arrival"] if paced else 0.0 for r in reqs]
        acc = torch.zeros((), dtype=torch.int64, device=dev)
        clocks = ClockSampler(local)
        clocks.start()
        slat, busy = [], 0.0
        t0 = time.perf_counter()
        for r, a in zip(reqs, arr):
            while time.perf_counter() - t0 < a:
                pass
            rgba, ns = bufs[r["side"]][0]
            j = job(r, ids32, rgba, ns)
            ts = time.perf_counter()
            ctx.render(j["model_id"], j["camera"], j["params"], j["tf_dev"], 256, rgba, ns, stream=stream)
            acc += ns.sum(dtype=torch.int64)
            stream.synchronize()
            te = time.perf_counter()
            busy += te - ts
            slat.append(te - t0 - a)
        clk = clocks.stop()
        n = int(acc.item())
        makespan = max(a + l for a, l in zip(arr, slat)) - arr[0]
        return {"latency_ms_p50": 1000 * _pct(slat, 0.50), "latency_ms_p99": 1000 * _pct(slat, 0.99),
                "latency_ms_max": 1000 * max(slat), "samples": n, "busy_s": busy, "makespan_s": makespan,
                "samples_per_s": n / makespan, "frames_per_s": len(reqs) / makespan, "clocks": clk,
                "replay": ("real time" if paced else "all requests at once") +
                          ", synchronous, one request at a time"}

    serial = serial_run()
    serial_cap = serial_run(paced=False) if capacity else None
    busy = serial["busy_s"]
    for m in ids32:
        ctx.unload_model(m)
    span = reqs[-1]["arrival"] - reqs[0]["arrival"]
    out = {"served_f16": srv16, "served_f32": srv32, "serial_f32": serial, "resident_model_bytes": resident,
           "offered_load_serial_f32": busy / span if span > 0 else None,
           "f16_vs_serial_f32_samples_per_s": srv16["samples_per_s"] / serial["samples_per_s"]}
    if capacity:
        cap16 = served("f16", paced=False)
        out["saturated"] = {"served_f16": cap16, "serial_f32": serial_cap,
                            "f16_vs_serial_f32_samples_per_s": cap16["samples_per_s"] / serial_cap["samples_per_s"],
                            "what": "every request available at once: the samples/s each renderer sustains "
                                    "when the GPU is the bottleneck"}
    if check:
        oracle.build()
        worst, rms = 0.0, []
        for i in check:
            r = reqs[i]
            m = mods[r["model"]]
            ref = oracle.render(m["ctrl"], m["degree"], r["camera"],
                                dict(prm, width=256, height=256, tf=m["tf"]), row_step=2)
            rows = np.arange(0, 256, 2)
            e = np.minimum(np.abs(kept[i] - ref["rgba"]).max(-1), np.abs(kept[i] - ref["rgba_alt"]).max(-1))[rows]
            worst = max(worst, float(e.max()))
            rms.append(float(np.sqrt(np.mean(e * e))))
        out["f16_pixel_error_vs_oracle"] = {"max": worst, "rms": float(np.mean(rms)), "requests": len(check),
                                            "rows": "every 2nd row of each 256^2 image",
                                            "reference": "FP64 oracle of the FP32 lattice"}
    return out


def _fp32_peak(torch, dev, clk):
    props = torch.cuda.get_device_properties(dev)
    sm_max = (clk or {}).get("sm_max_mhz") or _measured_peaks().get("sm_max_mhz") or 2070.0
    return props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12


def _timed_frames(ctx, torch, dev, local, mid, wl, prm, d_tf, d_img, d_ns, flush, stream, frames, warm):
    """Autotuned launch shape (untimed), `warm` untimed frames, then `frames`
    frames timed with CUDA events, the L2 flushed before each.  Returns
    (ms list, composited samples per frame, clocks)."""
    ctx.autotune(mid, wl["camera"], prm, d_tf, wl["tf"].shape[0], d_img, d_ns, stream=stream)
    for _ in range(warm):
        flush.zero_()
        ctx.render(mid, wl["camera"], prm, d_tf, wl["tf"].shape[0], d_img, d_ns, stream=stream)
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(frames)]
    clocks = ClockSampler(local)
    clocks.start()
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        ctx.render(mid, wl["camera"], prm, d_tf, wl["tf"].shape[0], d_img, d_ns, stream=stream)
        b.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    return [a.elapsed_time(b) for a, b in ev], int(d_ns.sum(dtype=torch.int64).item()), clk


def leg_ml32(torch, dev, local, flush, stream, frames=20):
    """The small case: 32^3 degree-3 Marschner-Lobb model at 128x128
    orthographic, step 1/256: frame time and the largest pixel error against
    the oracle's full frame."""
    import numpy as np

    import oracle
    from paper_2204_11762_gb300 import mfadvr, workloads
    wl = workloads.small_ml_workload()
    prm = wl["params"]
    W, H = prm["width"], prm["height"]
    ctx = mfadvr.Context(local)
    d_tf = torch.from_numpy(wl["tf"]).to(dev)
    d_img = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    d_ns = torch.empty((H, W), dtype=torch.int32, device=dev)
    mid = ctx.load_model(wl["ctrl"], wl["degree"])
    ms, samples, clk = _timed_frames(ctx, torch, dev, local, mid, wl, prm, d_tf, d_img, d_ns, flush, stream,
                                     frames, 3)
    img = d_img.cpu().numpy()
    ctx.close()
    oracle.build()
    t0 = time.perf_counter()
    ref = oracle.render(wl["ctrl"], wl["degree"], wl["camera"], dict(prm, tf=wl["tf"]))
    t_oracle = time.perf_counter() - t0
    err = np.minimum(np.abs(img - ref["rgba"]).max(-1), np.abs(img - ref["rgba_alt"]).max(-1))
    r_ms = statistics.mean(ms)
    return {"workload": "ml32_p3: 128x128 orthographic, 32^3 Marschner-Lobb (Eq. 2) + N(0, 0.01), step 1/256, "
                        "TF 256, shading",
            "frames": frames, "render_ms": r_ms, "samples_per_frame": samples,
            "samples_per_s": samples / (r_ms / 1000.0), "frames_per_s": 1000.0 / r_ms,
            "max_pixel_err_vs_oracle": float(err.max()), "tolerance": 2e-3,
            "oracle_full_frame_s": t_oracle, "oracle_cores": os.cpu_count() or 1, "clocks": clk}


def leg_noise512(torch, dev, local, flush, stream, frames=3):
    """The large single model: 512^3 degree-4 value noise at 3840x2160, step
    1/2048, TF 1024, in FP32 and in BF16 storage: frame times, the roofline
    fraction, and the pixel error against the oracle of the FP32 lattice on
    every 540th row."""
    import numpy as np

    import oracle
    from paper_2204_11762_gb300 import mfadvr, workloads
    wl = workloads.value_noise_workload(512)
    p, prm = wl["degree"], wl["params"]
    W, H = prm["width"], prm["height"]
    ctx = mfadvr.Context(local)
    d_tf = torch.from_numpy(wl["tf"]).to(dev)
    d_img = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    d_ns = torch.empty((H, W), dtype=torch.int32, device=dev)
    out, imgs = {}, {}
    # FP32 in the power form, requested (its cells take 84 GB, beyond the
    # AUTO default's 4 GiB), and in the B-spline form; BF16 (B-spline form)
    for st, storage, form in (("f32", "f32", FORMS["power"]), ("f32_bspline", "f32", FORMS["bspline"]),
                              ("bf16", "bf16", FORMS["auto"])):
        mid = ctx.load_model(wl["ctrl"], p, storage=storage, render_form=form)
        resident = ctx.model_info(mid)["bytes"]
        ms, samples, clk = _timed_frames(ctx, torch, dev, local, mid, wl, prm, d_tf, d_img, d_ns, flush, stream,
                                         frames, 2)
        imgs[st] = d_img.cpu().numpy()
        ctx.unload_model(mid)
        r_ms = statistics.mean(ms)
        tflops = samples * C_FMA[p] * 2 / (r_ms / 1000.0) / 1e12
        peak = _fp32_peak(torch, dev, clk)
        out[st] = {"render_ms": r_ms, "samples_per_frame": samples, "samples_per_s": samples / (r_ms / 1000.0),
                   "tflops": tflops, "frac": tflops / peak, "resident_model_bytes": resident, "clocks": clk}
    ctx.close()
    oracle.build()
    rows = np.arange(0, H, 540)
    ref = oracle.render(wl["ctrl"], p, wl["camera"], dict(prm, tf=wl["tf"]), row_step=540)
    for st in out:
        e = np.minimum(np.abs(imgs[st] - ref["rgba"]).max(-1), np.abs(imgs[st] - ref["rgba_alt"]).max(-1))[rows]
        out[st]["pixel_err_vs_oracle"] = {"max": float(e.max()), "rms": float(np.sqrt(np.mean(e * e)))}
    out["bf16"]["vs_f32"] = out["f32"]["render_ms"] / out["bf16"]["render_ms"]
    out["f32_bspline"]["vs_f32"] = out["f32"]["render_ms"] / out["f32_bspline"]["render_ms"]
    return {"workload": "noise512_p4: 3840x2160 perspective, 512^3 value noise, step 1/2048, TF 1024, shading",
            "frames": frames, "per_unit": f"{C_FMA[p]} FMA per sample", "error_rows": "every 540th row",
            **out}


def leg_serve_slice(torch, dev, local, args, models=8, requests=200):
    """A bounded slice of the serving workload: the stream's first `models`
    models (degree 3-4, lattices 96^3..384^3) and `requests` Poisson requests
    at 200/s, replayed in real time through the serving loop with FP16 and
    with FP32 models and through serial plain-FP32 rendering."""
    from paper_2204_11762_gb300 import mfadvr, workloads
    mods, reqs, prm = workloads.serving_workload(models=models, requests=requests)
    prm = dict(prm, step=args.serve_step)
    ctx = mfadvr.Context(local)
    legs = serve_legs(ctx, torch, dev, local, mods, reqs, prm, args, err_requests=4, capacity=True)
    ctx.close()
    return {"workload": f"serve slice: {requests} requests, Poisson 200/s, {models} resident models "
                        f"(degree 3-4, lattices {min(m['ncp'][0] for m in mods)}^3.."
                        f"{max(m['ncp'][0] for m in mods)}^3), images {{256,512,1024,2048}}^2, "
                        f"step {args.serve_step:g}",
            "frame_budget_bytes": 2 << 30, "max_batch": args.serve_batch, "max_in_flight": args.serve_flights,
            **legs}


def run_serve48(args, wl):
    """Real-time replay of a Poisson request stream (2000 requests at 200/s,
    48 resident models of degree 3-4, images 256^2..2048^2) through the
    serving loop with FP16 models and with FP32 models, against serial
    plain-FP32 rendering of the same stream, also replayed in real time."""
    import torch

    from paper_2204_11762_gb300 import mfadvr

    mods, reqs, prm = wl
    prm = dict(prm, step=args.serve_step)
    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = mfadvr.Context(local)
    legs = serve_legs(ctx, torch, dev, local, mods, reqs, prm, args, err_requests=8, capacity=True)
    ctx.close()
    srv16 = legs["served_f16"]
    line = {"metric": METRIC, "value": srv16["samples_per_s"], "unit": UNIT, "n_gpus": world,
            "steps": len(reqs), "warmup": len(mods), "ms_per_step": 1000 * srv16["makespan_s"] / len(reqs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (storage f16)",
            "data": "synthetic",
            "config": {"workload": f"serve48: {len(reqs)} requests, Poisson 200/s, {len(mods)} resident models "
                                   f"(degree 3-4, lattices 96^3..384^3, FP16), images {{256,512,1024,2048}}^2, "
                                   f"step {args.serve_step:g}",
                       "frame_budget_bytes": 2 << 30, "max_batch": args.serve_batch,
                       "max_in_flight": args.serve_flights},
            **legs, "gpu_launches": srv16["launches"]}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = _args()
    from paper_2204_11762_gb300 import workloads
    if args.workload == "ml32":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle reference arm is timed on the "
                                                                   "default workload only"}))
            return
        run_ml32(args, workloads.small_ml_workload())
        return
    if args.workload == "noise512":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle reference arm is timed on the "
                                                                   "default workload only"}))
            return
        run_noise512(args, workloads.value_noise_workload(512))
        return
    if args.workload == "serve48":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle reference arm is timed on the "
                                                                   "default workload only"}))
            return
        run_serve48(args, workloads.serving_workload())
        return
    if args.workload == "multi16":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle reference arm is timed on the "
                                                                   "default workload only"}))
            return
        run_multi16(args, workloads.multi_model_workload())
        return
    if args.workload == "variants":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle reference arm is timed on the "
                                                                   "default workload only"}))
            return
        run_variants(args)
        return
    if args.workload == "sweep":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle reference arm is timed on the "
                                                                   "default workload only"}))
            return
        run_sweep(args)
        return
    wl = workloads.gaussian_sum_workload()
    if args.image:
        wl["params"] = dict(wl["params"], width=args.image, height=args.image)
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
