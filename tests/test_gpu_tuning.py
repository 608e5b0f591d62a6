"""GPU tests of the measured tile / block shape choice (etac_autotune, etac_set_tuning): every
propagation-GEMM shape (32, 64 or 80 instances per tile, both tile orders) and every node range
of the reverse mode's decoder stage must give the oracle's results within the same bounds as
the default shapes; the autotuner returns candidates it timed and leaves a valid choice in
effect."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_20295_gb300 import build as B
from paper_2604_20295_gb300 import etac as X
from paper_2604_20295_gb300 import inputs as I
from tests import parity as PT

pytestmark = pytest.mark.gpu
BF16_REL = 2e-2


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    X.lib()
    assert torch.cuda.is_available()


def _scene():
    # 16 pad types (8x8 .. 64x64), partial 32- and 64-instance tiles
    return I.uneven_scene(40, seed=5).subset(np.arange(0, 40, 3))


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _forward_check(sim, sc, th):
    sim.step()
    torch.cuda.synchronize()
    disp, mask = sim.disp.cpu().numpy(), sim.mask.cpu().numpy()
    ref, _ = PT.oracle_forward_matching(sc, th, X.MODE_FULL, mask)
    errs, scale = PT.pad_errors(sc, disp, ref["disp"])
    assert np.all(errs <= BF16_REL * scale + 1e-6), (errs / np.maximum(scale, 1e-30)).max()
    return mask


def _backward_check(sim, sc, th, G, mask):
    G, dropped = PT.condition_upstream(sc, th, G, mask)
    assert len(dropped) <= sc.num_envs * sc.pads_per_env // 2
    g = sim.backward(torch.as_tensor(np.asarray(G, np.float32)).cuda())
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}
    ref = O.backward(sc, th, G, mode=X.MODE_FULL, mask_override=mask)
    ref["obj_pose"] = ref["obj_pose"].reshape(got["obj_pose"].shape)
    PT.assert_grads_close(got, ref, I.param_slices())


@pytest.mark.parametrize("gi,order", [(64, 0), (64, 1), (80, 0), (80, 1), (32, 0), (32, 1)])
def test_every_gemm_shape_matches_oracle(gi, order):
    sc = _scene()
    th = I.make_params(1)
    G = np.random.default_rng(3).normal(size=(sc.total_nodes, 3))
    sim = X.TactileSim(sc)
    try:
        sim.set_model(th, X.MODE_FULL, X.PREC_BF16, X.ALGO_BATCHED)
        sim.set_tuning(gi, order, 0)
        mask = _forward_check(sim, sc, th)
        _backward_check(sim, sc, th, G, mask)
        assert sim.poll_status() == 0
    finally:
        sim.close()


@pytest.mark.parametrize("node_range", [16, 48, 128, 256])
def test_every_backward_node_range_matches_oracle(node_range):
    sc = I.hand_scene(64, seed=7).subset([0, 5, 9, 20])
    th = I.make_params(0)
    G = np.random.default_rng(1).normal(size=(sc.total_nodes, 3))
    sim = X.TactileSim(sc)
    try:
        sim.set_model(th, X.MODE_FULL, X.PREC_FP32, X.ALGO_BATCHED)
        sim.set_tuning(64, 0, node_range)
        sim.step()
        torch.cuda.synchronize()
        _backward_check(sim, sc, th, G, sim.mask.cpu().numpy())
    finally:
        sim.close()


def test_autotune_picks_a_timed_candidate_and_stays_correct():
    sc = I.hand_scene(96, seed=11)
    th = I.make_params(0)
    G = np.random.default_rng(4).normal(size=(sc.total_nodes, 3))
    sim = X.TactileSim(sc)
    try:
        sim.set_model(th, X.MODE_FULL, X.PREC_BF16, X.ALGO_BATCHED)
        t = sim.autotune(torch.as_tensor(np.asarray(G, np.float32)).cuda())
        print("autotune:", t)
        assert len(t["fwd"]) == 6 and len(t["bwd"]) == 4
        best = min(t["fwd"], key=lambda c: c[2])
        assert (t["gemm_inst_per_tile"], t["gemm_tile_order"]) == best[:2]
        assert t["bwd_node_range"] == min(t["bwd"], key=lambda c: c[1])[0]
        assert all(ms > 0 for _, _, ms in t["fwd"]) and all(ms > 0 for _, ms in t["bwd"])
        assert len(t["front"]) >= 1 and all(ms > 0 for _, ms in t["front"])
        assert t["front_ctas_per_sm"] == min(t["front"], key=lambda c: c[1])[0]
        sub = [0, 17, 50, 95]
        scs = sc.subset(sub)
        sim.step()
        torch.cuda.synchronize()
        offs = sc.node_offsets
        idx = np.concatenate([np.arange(offs[e * 6], offs[e * 6 + 6]) for e in sub])
        disp, mask = sim.disp.cpu().numpy()[idx], sim.mask.cpu().numpy()[idx]
        ref, _ = PT.oracle_forward_matching(scs, th, X.MODE_FULL, mask)
        errs, scale = PT.pad_errors(scs, disp, ref["disp"])
        assert np.all(errs <= BF16_REL * scale + 1e-6)
        assert sim.poll_status() == 0
    finally:
        sim.close()


def test_set_tuning_rejects_bad_shapes():
    sc = I.hand_scene(4, seed=1)
    sim = X.TactileSim(sc)
    try:
        sim.set_model(I.make_params(0), X.MODE_FULL, X.PREC_BF16, X.ALGO_BATCHED)
        with pytest.raises(X.EtacError):
            sim.set_tuning(48, 0, 0)
        with pytest.raises(X.EtacError):
            sim.set_tuning(64, 2, 0)
        with pytest.raises(X.EtacError):
            sim.set_tuning(64, 0, 40)
        with pytest.raises(X.EtacError):
            sim.set_tuning(64, 0, 0, front_ctas_per_sm=99)
        sim.set_tuning(32, 1, 64)   # valid; the context keeps working
        sim.step()
        torch.cuda.synchronize()
        assert sim.poll_status() == 0
    finally:
        sim.close()


def test_tuning_cache_applies_a_stored_choice(tmp_path):
    """A choice stored under the tuning key (GPU, pad-type histogram, objects, model) is
    applied by a later context of the same key without timing, and the step stays correct;
    another workload has another key."""
    cache = str(tmp_path / "tuning.json")
    sc = I.hand_scene(48, seed=12)
    th = I.make_params(0)
    first = X.TactileSim(sc)
    try:
        first.set_model(th, X.MODE_FULL, X.PREC_BF16, X.ALGO_BATCHED)
        t1 = first.autotune(cache=cache)
        assert not t1["cached"]
        key = first.tuning_key(False)
    finally:
        first.close()
    again = X.TactileSim(sc)
    try:
        again.set_model(th, X.MODE_FULL, X.PREC_BF16, X.ALGO_BATCHED)
        assert again.tuning_key(False) == key
        t2 = again.autotune(cache=cache)
        assert t2["cached"]
        for k in ("gemm_inst_per_tile", "gemm_tile_order", "front_ctas_per_sm"):
            assert t2[k] == t1[k]
        mask = _forward_check(again, sc, th)
        assert mask.any()
    finally:
        again.close()
    other = X.TactileSim(I.uneven_scene(4, seed=1))
    try:
        other.set_model(th, X.MODE_FULL, X.PREC_BF16, X.ALGO_BATCHED)
        assert other.tuning_key(False) != key
    finally:
        other.close()
