"""GPU taxel regressor (etac_regress) against the FP64 oracle, both precisions: hand pads (512
and 2,048 nodes: 4 and 16 tiles of 128), uneven pads, ragged pads (37, 21, 45 nodes), a field
from a GPU step, no attention output, repeatability, and the full 4,096-env hand layout checked
on sampled envs (the launch the bench times).

Tolerances, per pad, max_k |y_k - y_ref,k| <= tol * max_k |y_ref,k| + atol:
- FP32 rung: FP32 dot products of length <= 256 through seven layers and a softmax give a
  relative error of a few 1e-6; tol 1e-4, atol 1e-6; attention weights within 1e-4 relative.
- Tensor-core path (BF16 operands, FP32 accumulation) against the oracle run on the same
  weights rounded to BF16 (a different, exactly representable model; the oracle's arithmetic is
  unchanged): what remains is the rounding of the four stored activations h1, h2, h3, f to BF16
  (2^-9 relative each), tanh.approx (about 2^-11) and x's two-part split (2^-17).  To first
  order each rounding perturbs the output by 2^-9 times the output's sensitivity to that layer;
  summed over four layers with random signs, tol = 4 * 2^-9 ~ 8e-3 of the output scale; atol
  1e-5.  Attention weights: 8e-3 of the pad's largest weight (a score error d moves a weight by
  the factor exp(d)).
- Against the oracle on the FP32 weights the weight rounding adds 2^-9 relative per weight, in
  dot products of 64-256 random-sign terms: the same order again; tol 2e-2.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_20295_gb300 import build as B
from paper_2604_20295_gb300 import etac as X
from paper_2604_20295_gb300 import inputs as I

pytestmark = pytest.mark.gpu

REL32, ABS32 = 1e-4, 1e-6
REL_TC, ABS_TC = 8e-3, 1e-5           # against the oracle on BF16-rounded weights
REL_TC_F32W = 2e-2                    # against the oracle on the FP32 weights


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    X.lib()


def bf16_round(a):
    """Round-to-nearest-even to BF16, returned as float64 (exact)."""
    return torch.as_tensor(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def tc_weights(rp):
    """The regressor as the tensor-core path evaluates it: the five per-node layers' weights
    (R1, R2, R3, R4, A1) rounded to BF16, biases and the A2, H1, H2 layers unchanged."""
    out = np.asarray(rp, np.float64).copy()
    sl = I.regressor_param_slices()
    for k in ("WR1", "WR2", "WR3", "WR4", "WA1"):
        s, n, _ = sl[k]
        out[s:s + n] = bf16_round(out[s:s + n])
    return out


def taxel_ratio(got, want, rel, abs_):
    """Worst per-pad ratio of |dy| to its allowance (<= 1 passes)."""
    scale = np.abs(want).max(axis=1, keepdims=True)
    return float((np.abs(got - want) / (rel * scale + abs_)).max())


def attn_ratio(scene, got, want, rel):
    offs = scene.node_offsets
    amax = np.maximum.reduceat(want, offs[:-1])
    allow = rel * np.repeat(amax, np.diff(offs)) + 1e-9
    return float((np.abs(got - want) / allow).max())


def _scene(name):
    if name == "hand":
        return I.hand_scene(16, seed=3).subset([0, 7, 11])
    if name == "uneven":
        return I.uneven_scene(8, seed=4).subset([1, 5])
    if name == "many":
        return I.hand_scene(6, seed=8)
    types = [I.flat_pad(1, 37, 1.0), I.flat_pad(3, 7, 0.5), I.curved_pad(5, 9, 1.0, 8.0)]
    return I.custom_scene(types, [0, 1, 2], {0: (I.OBJ_SPHERE, (4.0, 0, 0), (0, 0, 3.5, 0, 0, 0, 1))},
                          [(0, 0, 0, 0, 0, 0, 1)] * 3, 1, 1)


def _run(scene, disp32, rp, want_attn=True, precision=X.PREC_BF16):
    sim = X.TactileSim(scene)
    try:
        d = torch.as_tensor(np.ascontiguousarray(disp32, np.float32)).cuda()
        y, a = sim.regress(rp, disp=d, want_attn=want_attn, precision=precision)
        torch.cuda.synchronize()
        assert sim.poll_status() == 0
        return y.cpu().numpy().astype(np.float64), None if a is None else a.cpu().numpy()
    finally:
        sim.close()


@pytest.mark.parametrize("scene", ["hand", "uneven", "ragged"])
def test_fp32_rung_matches_the_oracle(scene):
    sc = _scene(scene)
    disp = O.forward(sc, I.make_params(1))["disp"].astype(np.float32)
    rp = I.make_regressor_params(3)
    ref = O.regress(sc, disp.astype(np.float64), rp.astype(np.float64))
    y, a = _run(sc, disp, rp, precision=X.PREC_FP32)
    assert taxel_ratio(y, ref["taxels"], REL32, ABS32) <= 1.0
    np.testing.assert_allclose(a, ref["attn"], rtol=REL32, atol=1e-9)


@pytest.mark.parametrize("scene", ["hand", "uneven", "ragged", "many"])
def test_tensor_core_path_matches_the_oracle(scene):
    sc = _scene(scene)
    disp = O.forward(sc, I.make_params(1))["disp"].astype(np.float32)
    rp = I.make_regressor_params(3)
    y, a = _run(sc, disp, rp)
    d64 = disp.astype(np.float64)
    ref_bw = O.regress(sc, d64, tc_weights(rp))
    ref = O.regress(sc, d64, rp.astype(np.float64))
    r_bw = taxel_ratio(y, ref_bw["taxels"], REL_TC, ABS_TC)
    r_fw = taxel_ratio(y, ref["taxels"], REL_TC_F32W, ABS_TC)
    r_at = attn_ratio(sc, a, ref_bw["attn"], REL_TC)
    print(f"{scene}: taxels {r_bw:.3f} of the BF16-weight bound, {r_fw:.3f} of the FP32-weight "
          f"bound; attention {r_at:.3f} of its bound")
    assert r_bw <= 1.0 and r_fw <= 1.0 and r_at <= 1.0
    # the softmax weights of every pad sum to one
    s = np.add.reduceat(a.astype(np.float64), sc.node_offsets[:-1])
    assert np.all(np.abs(s - 1.0) < 1e-5)


def test_tensor_core_path_on_a_gpu_step_field_repeatable_and_without_attention():
    sc = I.hand_scene(8, seed=6)
    rp = I.make_regressor_params(9)
    sim = X.TactileSim(sc)
    try:
        sim.set_model(I.make_params(0), X.MODE_FULL, X.PREC_BF16, X.ALGO_BATCHED)
        disp = sim.step().clone()
        y1, a1 = sim.regress(rp)
        y2, a2 = sim.regress(rp, want_attn=False)
        y3, a3 = sim.regress(rp)
        y4, _ = sim.regress(rp, precision=X.PREC_FP32)
        torch.cuda.synchronize()
        assert sim.poll_status() == 0
        assert a2 is None and torch.equal(y1, y2) and torch.equal(y1, y3) and torch.equal(a1, a3)
        got_y, got_a = y1.cpu().numpy().astype(np.float64), a1.cpu().numpy()
        y32 = y4.cpu().numpy().astype(np.float64)
        d = disp.cpu().numpy().astype(np.float64)
    finally:
        sim.close()
    ref = O.regress(sc, d, tc_weights(rp))
    assert taxel_ratio(got_y, ref["taxels"], REL_TC, ABS_TC) <= 1.0
    assert attn_ratio(sc, got_a, ref["attn"], REL_TC) <= 1.0
    ref32 = O.regress(sc, d, rp.astype(np.float64))
    assert taxel_ratio(y32, ref32["taxels"], REL32, ABS32) <= 1.0


def test_tensor_core_path_at_full_size_on_sampled_envs():
    """The 4,096-env hand layout (18.9 M nodes, 24,576 pads over every SM's two slots), on the
    BF16 step's field; three envs (18 pads) are checked against the oracle."""
    sc = I.hand_scene(4096, seed=2)
    rp = I.make_regressor_params(0)
    sim = X.TactileSim(sc)
    try:
        sim.set_model(I.make_params(0), X.MODE_FULL, X.PREC_BF16, X.ALGO_BATCHED)
        disp = sim.step()
        y, a = sim.regress(rp)
        torch.cuda.synchronize()
        assert sim.poll_status() == 0
        envs = [0, 2047, 4095]
        P = sc.pads_per_env
        offs = sc.node_offsets
        rows = np.concatenate([np.arange(offs[e * P], offs[(e + 1) * P]) for e in envs])
        pads = np.concatenate([np.arange(e * P, (e + 1) * P) for e in envs])
        d = disp[torch.as_tensor(rows, device=disp.device)].cpu().numpy().astype(np.float64)
        got_y = y[torch.as_tensor(pads, device=y.device)].cpu().numpy().astype(np.float64)
        got_a = a[torch.as_tensor(rows, device=a.device)].cpu().numpy()
        assert torch.isfinite(y).all()
    finally:
        sim.close()
    sub = sc.subset(envs)
    ref = O.regress(sub, d, tc_weights(rp))
    assert taxel_ratio(got_y, ref["taxels"], REL_TC, ABS_TC) <= 1.0
    assert attn_ratio(sub, got_a, ref["attn"], REL_TC) <= 1.0
