"""Omega (Eq. 1) on the fly in the batched FP32 step, and pads of continuous, per-instance pitch
(every pad its own type, so per-type tables cannot be shared: the continuous-pitch variant of
the uneven 8x8 .. 64x64 workload).

- The on-the-fly kernel evaluates exp(-alpha |p_j - p_i|) with the per-type table's own FP32
  expression, so on shared types it reproduces the table step bit for bit.
- On continuous-pitch scenes, the batched step (Omega on the fly) and the plain step match the
  FP64 oracle (contacts bit-exact outside the 1e-6 mm band, displacements within 1e-5 of the
  pad's scale, as every FP32 parity test), and so does the reverse mode.
- Where the tables would exceed 4 GiB the library chooses on the fly by itself and refuses an
  explicit request for the table; the autotuner times both sources where the table fits.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_20295_gb300 import build as B
from paper_2604_20295_gb300 import etac as X
from paper_2604_20295_gb300 import inputs as I
from tests import parity as PT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    X.lib()


def _step(scene, theta, algo=X.ALGO_BATCHED, omega=X.OMEGA_AUTO, mode=X.MODE_FULL):
    sim = X.TactileSim(scene)
    try:
        sim.set_model(theta, mode, X.PREC_FP32, algo)
        if algo == X.ALGO_BATCHED:
            sim.set_tuning(omega_source=omega)
        sim.step()
        torch.cuda.synchronize()
        assert sim.poll_status() == 0
        return sim.disp.cpu().numpy().astype(np.float64), sim.mask.cpu().numpy()
    finally:
        sim.close()


@pytest.mark.parametrize("mode", [X.MODE_FULL, X.MODE_LINEAR_ONLY])
def test_on_the_fly_omega_equals_the_table_bitwise(mode):
    sc = I.uneven_scene(12, seed=7)
    th = I.make_params(2)
    d_tab, m_tab = _step(sc, th, omega=X.OMEGA_TABLE, mode=mode)
    d_otf, m_otf = _step(sc, th, omega=X.OMEGA_ON_THE_FLY, mode=mode)
    np.testing.assert_array_equal(m_tab, m_otf)
    np.testing.assert_array_equal(d_tab, d_otf)
    assert m_tab.sum() > 0


@pytest.mark.parametrize("algo", [X.ALGO_BATCHED, X.ALGO_PLAIN])
def test_continuous_pitch_matches_the_oracle(algo):
    sc = I.uneven_continuous_scene(10, seed=3)
    th = I.make_params(1)
    omega = X.OMEGA_ON_THE_FLY if algo == X.ALGO_BATCHED else X.OMEGA_AUTO
    disp, mask = _step(sc, th, algo=algo, omega=omega)
    ref, _ = PT.oracle_forward_matching(sc, th, X.MODE_FULL, mask)
    PT.assert_disp_close(sc, disp, ref["disp"])
    assert mask.sum() > 0


def test_continuous_pitch_reverse_mode_matches_the_oracle():
    sc = I.uneven_continuous_scene(6, seed=11)
    th = I.make_params(3)
    G = np.random.default_rng(2).normal(size=(sc.total_nodes, 3))
    sim = X.TactileSim(sc)
    try:
        sim.set_model(th, X.MODE_FULL, X.PREC_FP32, X.ALGO_BATCHED)
        sim.set_tuning(omega_source=X.OMEGA_ON_THE_FLY)
        sim.step()
        mask = sim.mask.cpu().numpy()
        Gc, _ = PT.condition_upstream(sc, th, G, mask)
        g = sim.backward(torch.as_tensor(Gc, dtype=torch.float32).cuda())
        torch.cuda.synchronize()
        assert sim.poll_status() == 0
        got = {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}
    finally:
        sim.close()
    PT.oracle_forward_matching(sc, th, X.MODE_FULL, mask)
    ref = O.backward(sc, th, Gc, mask_override=mask)
    ref["obj_pose"] = ref["obj_pose"].reshape(got["obj_pose"].shape)
    PT.assert_grads_close(got, ref, I.param_slices())


def test_large_continuous_scene_chooses_on_the_fly_and_refuses_the_table():
    """512 envs of per-instance pads: the Omega tables would take about 55 GB, so the library
    evaluates Omega on the fly; an explicit request for the table is refused.  Sampled envs
    against the oracle."""
    sc = I.uneven_continuous_scene(512, seed=4)
    th = I.make_params(0)
    sim = X.TactileSim(sc)
    try:
        sim.set_model(th, X.MODE_FULL, X.PREC_FP32, X.ALGO_BATCHED)
        with pytest.raises(X.EtacError) as e:
            sim.set_tuning(omega_source=X.OMEGA_TABLE)
        assert e.value.status == 7
        sim.step()
        torch.cuda.synchronize()
        assert sim.poll_status() == 0
        envs = np.array([0, 255, 511])
        offs = sc.node_offsets
        rows = np.concatenate([np.arange(offs[e * 6], offs[e * 6 + 6]) for e in envs])
        disp = sim.disp.cpu().numpy()[rows].astype(np.float64)
        mask = sim.mask.cpu().numpy()[rows]
    finally:
        sim.close()
    sub = sc.subset(envs)
    ref, _ = PT.oracle_forward_matching(sub, th, X.MODE_FULL, mask)
    PT.assert_disp_close(sub, disp, ref["disp"])


def test_autotune_times_both_omega_sources():
    sc = I.uneven_scene(16, seed=2)
    sim = X.TactileSim(sc)
    try:
        sim.set_model(I.make_params(0), X.MODE_FULL, X.PREC_FP32, X.ALGO_BATCHED)
        r = sim.autotune()
        assert r["omega_source"] in (X.OMEGA_TABLE, X.OMEGA_ON_THE_FLY)
        assert r["omega_ms"][0] > 0 and r["omega_ms"][1] > 0
        sim.step()
        torch.cuda.synchronize()
        assert sim.poll_status() == 0
    finally:
        sim.close()
