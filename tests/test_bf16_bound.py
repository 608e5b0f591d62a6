"""The entry-wise error bound of the BF16 propagation contraction (Eq. 1), checked on the host:
a contraction that rounds Omega and u_hat to BF16 exactly as the tensor-core path does (round
to nearest, FP32 products and sums) must stay inside the bound that
`tests/test_gpu_bf16.py::propagation_bound` derives, and a contraction whose Omega is off by
2^-6 (twice the bound's 2^-7 rounding term, every entry the same way) must not."""
import numpy as np
import torch

import oracle as O
from paper_2604_20295_gb300 import etac as X
from paper_2604_20295_gb300 import inputs as I
from tests.test_gpu_bf16 import propagation_bound


def _bf16(a):
    return torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()


def _contract(scene, theta, ref, round_fn):
    alpha = float(theta[0])
    offs = scene.node_offsets
    mask = ref["mask"]
    out = np.zeros_like(ref["disp"])
    for p in range(len(scene.pad_type)):
        a, b = offs[p], offs[p + 1]
        act = mask[a:b] > 0
        if not act.any():
            continue
        pos = scene.types[scene.pad_type[p]].pos.astype(np.float64)
        om = np.exp(-alpha * np.linalg.norm(pos[:, None, :] - pos[None, act, :], axis=2))
        u = ref["disp"][a:b][act]
        out[a:b] = (round_fn(om.astype(np.float32)) @ round_fn(u.astype(np.float32))).astype(np.float32)
    return out


def _case():
    sc = I.hand_scene(64, seed=3).subset(np.arange(8))
    th = I.make_params(0)
    ref = O.forward(sc, th, mode=X.MODE_LINEAR_ONLY)
    return sc, th, ref


def test_bf16_rounded_contraction_stays_inside_the_bound():
    sc, th, ref = _case()
    sim = _contract(sc, th, ref, _bf16)
    bound = propagation_bound(sc, th, ref["mask"], ref)
    pas = ref["mask"] == 0
    err = np.abs(sim - ref["disp"])[pas]
    assert (ref["mask"] > 0).sum() > 0
    assert np.all(err <= bound[pas])
    # the bound is not loose by orders of magnitude: some entry comes within a factor of 4
    assert (err / np.maximum(bound[pas], 1e-300)).max() > 0.25


def test_a_contraction_off_by_twice_the_rounding_breaks_the_bound():
    sc, th, ref = _case()
    # Omega scaled by (1 + 2^-6), no rounding at all
    sim = _contract(sc, th, ref, lambda a: a.astype(np.float64) * (1.0 + 2.0 ** -6))
    bound = propagation_bound(sc, th, ref["mask"], ref)
    pas = ref["mask"] == 0
    assert np.any(np.abs(sim - ref["disp"])[pas] > bound[pas])
