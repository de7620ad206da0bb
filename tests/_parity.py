"""Comparison helpers for GPU-vs-oracle parity tests.

Tolerances: values 1e-5 relative and gradients 1e-4 relative, both
normalised by the model's scale (|a - b| / max(|b|, max|P|) for values,
|a - b| / max(|g_b|, max|P| * max_d m_d) for gradients) so that zero
crossings do not blow the ratio up; pixels 2e-3 absolute per RGBA channel;
knot spans exact.
"""
import numpy as np

VALUE_RTOL = 1e-5
GRAD_RTOL = 1e-4
PIXEL_ATOL = 2e-3


def storage_scale(amax: float, storage: str) -> float:
    """The library's per-model scale of a 16-bit array with largest
    magnitude amax: BF16 amax; FP16 the power of two putting amax in
    [2^14, 2^15); 1 for an all-zero array."""
    if not amax > 0:
        return 1.0
    if storage == "bf16":
        return float(np.float32(amax))
    _, e = np.frexp(np.float32(amax))
    return float(np.ldexp(np.float32(1.0), int(e) - 15))


def dequantize(ctrl: np.ndarray, storage: str) -> np.ndarray:
    """The lattice a 16-bit model actually holds: P/s rounded to the storage
    type (s = storage_scale(max|P|), P * (1/s) in FP32, round to nearest
    even), times s, in float64."""
    ctrl = np.asarray(ctrl, dtype=np.float32)
    if storage == "f32":
        return ctrl.astype(np.float64)
    s = np.float32(storage_scale(float(np.abs(ctrl).max()), storage))
    inv = np.float32(1.0) / s
    q = (ctrl * inv).astype(np.float32)
    if storage == "f16":
        qq = q.astype(np.float16).astype(np.float64)
    elif storage == "bf16":
        import torch
        qq = torch.from_numpy(q).to(torch.bfloat16).to(torch.float64).numpy()
    else:
        raise ValueError(storage)
    return qq * np.float64(s)


def eval_errors(got: np.ndarray, ref: np.ndarray, ctrl: np.ndarray, n, p):
    """Max normalised value and gradient errors."""
    pabs = float(np.abs(ctrl).max()) or 1.0
    m = max(int(x) - p for x in n)
    verr = np.abs(got[:, 0] - ref[:, 0]) / np.maximum(np.abs(ref[:, 0]), pabs)
    gn = np.linalg.norm(ref[:, 1:], axis=1)
    gerr = np.abs(got[:, 1:] - ref[:, 1:]).max(axis=1) / np.maximum(gn, pabs * m)
    return float(verr.max(initial=0.0)), float(gerr.max(initial=0.0))


def assert_eval_parity(got, ref, ctrl, n, p, spans=None, ref_spans=None, vtol=VALUE_RTOL, gtol=GRAD_RTOL):
    if spans is not None:
        bad = np.nonzero((spans != ref_spans).any(axis=1))[0]
        assert bad.size == 0, f"{bad.size} span mismatches, first at {bad[:5]}: {spans[bad[:5]]} vs {ref_spans[bad[:5]]}"
    ve, ge = eval_errors(got, ref, ctrl, n, p)
    assert ve <= vtol, f"value error {ve:.3e} > {vtol}"
    assert ge <= gtol, f"gradient error {ge:.3e} > {gtol}"
    return ve, ge


def pixel_errors(img: np.ndarray, ref: dict, rows=None):
    """Per-pixel max channel error against the oracle, taking a tied sample
    count either way where the oracle flagged one."""
    a = ref["rgba"]
    b = ref["rgba_alt"]
    if rows is not None:
        img, a, b = img[rows], a[rows], b[rows]
    e1 = np.abs(img - a).max(axis=-1)
    e2 = np.abs(img - b).max(axis=-1)
    return np.minimum(e1, e2)


def assert_render_parity(img, ns, ref, rows=None, atol=PIXEL_ATOL):
    err = pixel_errors(img, ref, rows)
    worst = np.unravel_index(np.argmax(err), err.shape)
    assert err.max() <= atol, f"pixel error {err.max():.3e} at {worst} > {atol}"
    if ns is not None:
        lo, hi = ref["ns_lo"], ref["ns_hi"]
        if rows is not None:
            ns, lo, hi = ns[rows], lo[rows], hi[rows]
        ok = (ns >= lo) & (ns <= hi)
        assert ok.all(), f"{(~ok).sum()} pixels with a sample count outside the tied range"
    return float(err.max())


def tie_stats(img, ns, ref, rows):
    """How often the tie windows of the oracle are used on the sampled rows:
    hit pixels, pixels whose GPU sample count differs from the exact FP64
    stop (nsamples), pixels whose allowed range [ns_lo, ns_hi] holds more
    than one count, and the largest opacity difference on the pixels that
    stopped elsewhere."""
    exact, lo, hi = ref["nsamples"][rows], ref["ns_lo"][rows], ref["ns_hi"][rows]
    g = ns[rows]
    hit = exact > 0
    moved = (g != exact) & hit
    da = np.abs(img[rows][..., 3] - ref["rgba"][rows][..., 3])
    return {"hit": int(hit.sum()), "off_exact": int(moved.sum()), "wide": int(((hi > lo) & hit).sum()),
            "tied_count": int((ref["nambig"][rows] != 0).sum()),
            "max_samples_off": int(np.abs(g - exact)[moved].max(initial=0)),
            "max_dA_off_exact": float(da[moved].max(initial=0.0))}


def assert_ties_rare(img, ns, ref, rows, limit=1e-3):
    """At most `limit` of the hit pixels may stop away from the exact FP64
    sample count (each still inside its tie range and its pixel within the
    tolerance, which assert_render_parity checks)."""
    st = tie_stats(img, ns, ref, rows)
    assert st["off_exact"] <= limit * st["hit"], f"tie windows used too often: {st}"
    return st
