"""GPU taxel regressor (etac_regress, plain FP32) against the FP64 oracle: hand pads, uneven
pads with ragged chunks, the field of a GPU step, without attention output, repeatability.

Tolerance: FP32 dot products of length <= 256 through seven layers and a softmax give a
relative error of a few 1e-6; per pad, max |dy| <= 1e-4 * max |y_ref| + 1e-6 and attention
weights within 1e-4 relative."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_20295_gb300 import build as B
from paper_2604_20295_gb300 import etac as X
from paper_2604_20295_gb300 import inputs as I

pytestmark = pytest.mark.gpu

REL, ABS = 1e-4, 1e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    X.lib()


def _check(got_y, got_a, ref):
    scale = np.abs(ref["taxels"]).max(axis=1, keepdims=True)
    assert np.all(np.abs(got_y - ref["taxels"]) <= REL * scale + ABS)
    if got_a is not None:
        np.testing.assert_allclose(got_a, ref["attn"], rtol=REL, atol=1e-9)


def _run(scene, disp32, rp, want_attn=True):
    sim = X.TactileSim(scene)
    try:
        d = torch.as_tensor(np.ascontiguousarray(disp32, np.float32)).cuda()
        y, a = sim.regress(rp, disp=d, want_attn=want_attn)
        torch.cuda.synchronize()
        return y.cpu().numpy().astype(np.float64), None if a is None else a.cpu().numpy()
    finally:
        sim.close()


@pytest.mark.parametrize("scene", ["hand", "uneven", "ragged"])
def test_regressor_matches_the_oracle(scene):
    if scene == "hand":
        sc = I.hand_scene(16, seed=3).subset([0, 7, 11])
    elif scene == "uneven":
        sc = I.uneven_scene(8, seed=4).subset([1, 5])
    else:
        types = [I.flat_pad(1, 37, 1.0), I.flat_pad(3, 7, 0.5), I.curved_pad(5, 9, 1.0, 8.0)]
        sc = I.custom_scene(types, [0, 1, 2], {0: (I.OBJ_SPHERE, (4.0, 0, 0), (0, 0, 3.5, 0, 0, 0, 1))},
                            [(0, 0, 0, 0, 0, 0, 1)] * 3, 1, 1)
    disp = O.forward(sc, I.make_params(1))["disp"].astype(np.float32)
    rp = I.make_regressor_params(3)
    ref = O.regress(sc, disp.astype(np.float64), rp.astype(np.float64))
    y, a = _run(sc, disp, rp)
    _check(y, a, ref)


def test_regressor_on_a_gpu_step_field_and_without_attention():
    sc = I.hand_scene(8, seed=6)
    rp = I.make_regressor_params(9)
    sim = X.TactileSim(sc)
    try:
        sim.set_model(I.make_params(0), X.MODE_FULL, X.PREC_BF16, X.ALGO_BATCHED)
        disp = sim.step().clone()
        y1, a1 = sim.regress(rp)
        y2, a2 = sim.regress(rp, want_attn=False)
        y3, _ = sim.regress(rp)
        torch.cuda.synchronize()
        assert a2 is None and torch.equal(y1, y2) and torch.equal(y1, y3)
        got_y, got_a, d = y1.cpu().numpy(), a1.cpu().numpy(), disp.cpu().numpy()
    finally:
        sim.close()
    ref = O.regress(sc, d.astype(np.float64), rp.astype(np.float64))
    _check(got_y.astype(np.float64), got_a, ref)
