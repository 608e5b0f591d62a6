"""Shared parity helpers for GPU-vs-oracle tests.

Tolerance (FP32 paths): per pad, max_i |U_gpu,i - U_ref,i| <= 1e-5 * max_i |U_ref,i| + 1e-7 mm,
the reading of "1e-5 relative" used throughout.  Contact sets must agree bit for bit except
at nodes whose oracle signed distance is within 1e-6 mm of the surface; where such a node
differs, the oracle is re-run with the GPU's contact set so that displacements are still
compared on identical masks.
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
