"""Shared parity helpers for GPU-vs-oracle tests.

Tolerance (FP32 paths): per pad, max_i |U_gpu,i - U_ref,i| <= 1e-5 * max_i |U_ref,i| + 1e-7 mm,
the reading of "1e-5 relative" used throughout.  Contact sets must agree bit for bit except
at nodes whose oracle signed distance is within 1e-6 mm of the surface; where such a node
differs, the oracle is re-run with the GPU's contact set so that displacements are still
compared on identical masks.

Reverse mode (FP32), entry by entry: |g - g_ref| <= ADJ_EPS * (|g_ref| + max |g_ref|), the
maximum taken over the entry's block (one parameter layer, the object-pose gradients, dL/du_hat
or dL/dpenetration).  Each entry is a sum of terms a_t.  Terms that pass through the reverse
propagation GEMM carry two BF16 splits (hi + lo, three products), i.e. a relative error of at
most 2^-16 each; every other term is a short FP32 expression (a few u = 2^-24); the FP32
sums of the kernels run at most ~10^3 sequential additions deep (warp shuffles, then per-CTA
and per-partial loops), a first-order bound of 10^3 u = 6e-5 of sum |a_t|.  ADJ_EPS = 1e-4
covers 2^-16 + 6e-5 of the scale above; rounding errors of random sign grow as the square root
of the depth, and the measured worst entry sits near 4e-6.
"""
from __future__ import annotations

import numpy as np

import oracle as O

REL_TOL = 1e-5
ABS_TOL = 1e-7
BAND = 1e-6


def oracle_forward_matching(scene, theta, mode, gpu_mask, nthreads=0):
    """Oracle forward; if the GPU contact set differs only inside the band, recompute the
    oracle on the GPU's set.  Returns (ref, n_band_diffs).  Raises on a difference outside
    the band."""
    ref = O.forward(scene, theta, mode=mode, nthreads=nthreads)
    diff = ref["mask"] != gpu_mask
    if diff.any():
        outside = diff & (np.abs(ref["phi"]) >= BAND)
        if outside.any():
            idx = np.nonzero(outside)[0][:10]
            raise AssertionError(f"contact mismatch outside the {BAND} mm band at nodes {idx}, "
                                 f"phi={ref['phi'][idx]}")
        ref = O.forward(scene, theta, mode=mode, mask_override=gpu_mask, nthreads=nthreads)
    return ref, int(diff.sum())


def pad_errors(scene, got, want):
    """Per-pad normwise error and scale: (max |dU|, max |U_ref|) for every pad instance."""
    offs = scene.node_offsets
    d = np.linalg.norm(np.asarray(got, np.float64) - want, axis=1)
    r = np.linalg.norm(want, axis=1)
    errs = np.maximum.reduceat(d, offs[:-1]) if len(d) else d
    scale = np.maximum.reduceat(r, offs[:-1]) if len(r) else r
    return errs, scale


def assert_disp_close(scene, got, want, rel=REL_TOL, abs_=ABS_TOL):
    errs, scale = pad_errors(scene, got, want)
    bad = errs > rel * scale + abs_
    if bad.any():
        i = int(np.argmax(errs / (rel * scale + abs_)))
        raise AssertionError(f"{int(bad.sum())} pads out of tolerance; worst pad {i}: "
                             f"err {errs[i]:.3e} scale {scale[i]:.3e}")
    return float(np.max(errs / np.maximum(scale, 1e-30))) if len(errs) else 0.0


ADJ_EPS = 1e-4

# The reverse mode of the residual network (Sec. III-A 2) takes discrete decisions: each ReLU's
# gate, and each channel's max-pool maximiser.  Where a pre-activation lies within rounding of
# zero, or two features within rounding of each other, FP32 and FP64 may decide differently;
# both are correct to FP32, and the gradient jumps there.  Every quantity those decisions read
# is FP32-accurate on the GPU (per-type tables evaluated in FP64 and rounded once; the reverse
# mode's recomputed encoder uses three-part BF16 splits, 2^-24 per operand; or the FP32
# forward's own record), i.e. within a few 1e-7 of its scale.  Reverse-mode parity therefore
# drops the upstream gradient of every pad with a decision margin below DECISION_MARGIN
# (relative to the scale of the terms each decision sums, as the oracle reports it).
DECISION_MARGIN = 1e-6


def condition_upstream(scene, theta, G, mask, mode=O.MODE_FULL, uhat=None):
    """(G with the rows of pads that hold a near-kink decision zeroed, their pad indices).
    The margins come from the oracle's decision report on the given contact set."""
    G = np.array(G, np.float64, copy=True)
    if mode not in (O.MODE_FULL, O.MODE_RESIDUAL_ONLY):
        return G, []
    mg = O.decision_margin(scene, theta, mask_override=mask, uhat_override=uhat)
    offs = scene.node_offsets
    dropped = [int(p) for p in np.nonzero(mg.min(axis=1) < DECISION_MARGIN)[0]]
    for p in dropped:
        G[offs[p]:offs[p + 1]] = 0.0
    return G, dropped


def grad_blocks(got, ref, param_slices):
    """(name, got, ref) blocks of a reverse-mode result: each parameter layer, object pose,
    dL/du_hat, dL/dpenetration (whichever both sides hold)."""
    out = []
    if "params" in got:
        for k, (s, n, _) in param_slices.items():
            out.append((k, got["params"][s:s + n], ref["params"][s:s + n]))
    for k in ("obj_pose", "uhat", "pen"):
        if k in got and k in ref:
            out.append((k, got[k], ref[k]))
    return out


def assert_grads_close(got, ref, param_slices, eps=ADJ_EPS):
    """Entry-by-entry reverse-mode parity (see the module docstring); returns the worst
    ratio |g - g_ref| / (|g_ref| + max |g_ref|) over all blocks."""
    worst = 0.0
    for name, g, r in grad_blocks(got, ref, param_slices):
        g = np.asarray(g, np.float64).ravel()
        r = np.asarray(r, np.float64).ravel()
        scale = np.abs(r).max() if r.size else 0.0
        if scale == 0.0:
            assert np.all(g == 0.0), f"{name}: oracle gradient is zero, GPU max |g| = {np.abs(g).max()}"
            continue
        ratio = np.abs(g - r) / (np.abs(r) + scale)
        i = int(np.argmax(ratio))
        assert ratio[i] <= eps, (f"{name}: entry {i} got {g[i]:.6e} want {r[i]:.6e} "
                                 f"(block max {scale:.3e}); ratio {ratio[i]:.2e} > {eps}")
        worst = max(worst, float(ratio[i]))
    return worst
