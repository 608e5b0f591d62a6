"""Failure detection without a GPU fault: a bounded device wait that runs out.

The propagation GEMM's MMA issuer waits (bounded, on an mbarrier) for the loads of each K
block.  The test hook etac_test_withhold_load makes the load producer of one GEMM tile skip
issuing its loads, so that wait can only end by running out; nothing faults and no copy is
left in flight.  The launch must return, etac_poll_status must report ETAC_ERR_TIMEOUT, and
the context must stay usable: the next normal step matches the oracle and reports no error."""
import time

import numpy as np
import pytest
import torch

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


def _check_against_oracle(sim, sc, th):
    disp, mask = sim.disp.cpu().numpy().astype(np.float64), sim.mask.cpu().numpy()
    ref, _ = PT.oracle_forward_matching(sc, th, X.MODE_FULL, mask)
    errs, scale = PT.pad_errors(sc, disp, ref["disp"])
    assert np.all(errs <= BF16_REL * scale + 1e-6), (errs / np.maximum(scale, 1e-30)).max()


@pytest.mark.parametrize("tile", [0, 1])
def test_withheld_load_times_out_and_the_context_recovers(tile):
    sc = I.hand_scene(8, seed=9)
    th = I.make_params(0)
    sim = X.TactileSim(sc)
    try:
        sim.set_model(th, X.MODE_FULL, X.PREC_BF16, X.ALGO_BATCHED)
        sim.step()
        assert sim.poll_status() == 0
        X.etac_test_withhold_load(sim.ctx, tile, 1_000_000)       # 1 ms wait limit
        t0 = time.perf_counter()
        sim.step()
        torch.cuda.synchronize()
        elapsed = time.perf_counter() - t0
        status = sim.poll_status()
        assert status == 5, X.STATUS_NAMES.get(status, status)       # ETAC_ERR_TIMEOUT
        assert elapsed < 1.0, elapsed                                 # gave up after ~ms
        X.etac_test_withhold_load(sim.ctx, -1, 0)
        sim.disp.fill_(float("nan"))
        sim.step()
        torch.cuda.synchronize()
        assert sim.poll_status() == 0
        _check_against_oracle(sim, sc, th)
    finally:
        sim.close()


def test_withhold_hook_checks_its_arguments():
    sc = I.hand_scene(2, seed=1)
    sim = X.TactileSim(sc)
    try:
        with pytest.raises(X.EtacError) as e:
            X.etac_test_withhold_load(sim.ctx, 0, 0)       # no model yet
        assert e.value.status == 2
        sim.set_model(I.make_params(0), X.MODE_FULL, X.PREC_FP32, X.ALGO_BATCHED)
        with pytest.raises(X.EtacError) as e:
            X.etac_test_withhold_load(sim.ctx, 0, 0)       # not a BF16 model
        assert e.value.status == 2
        sim.set_model(I.make_params(0), X.MODE_FULL, X.PREC_BF16, X.ALGO_BATCHED)
        for bad in ((-2, 0), (1 << 20, 0), (0, 3_000_000_000)):
            with pytest.raises(X.EtacError) as e:
                X.etac_test_withhold_load(sim.ctx, *bad)
            assert e.value.status == 1
    finally:
        sim.close()
