"""The no-allocation forward entry point (etac_step_forward_noalloc).

Callers that may not allocate device memory while they run -- an application that hands
the whole device heap to its own pool allocator, a real-time loop, or a plugin whose host
program gives it device pointers and no allocator -- use this entry point: its scratch lives
in a static device array in the library.  On two calls in a row (the second call reuses the
array the first one left behind), in every mode, it must give the regular batched FP32 entry
point's contact set, penetration and active counts exactly and its displacements within the
FP32 parity tolerance, and the FP64 oracle's results within that same tolerance.  Geometry
arrays whose device-side values disagree with the host sizes must leave the outputs untouched
and report ETAC_ERR_INVALID_ARG in the status word.  This file is collected last so that a
stop at the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2604_20295_gb300 import build as B
from paper_2604_20295_gb300 import etac as X
from paper_2604_20295_gb300 import inputs as I
from tests import parity as PT

pytestmark = pytest.mark.gpu
MODES = [X.MODE_FULL, X.MODE_LINEAR_ONLY, X.MODE_RESIDUAL_ONLY, X.MODE_PENETRATION_ONLY]


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    assert torch.cuda.is_available()


def _regular(scene, theta, mode):
    sim = X.TactileSim(scene)
    try:
        sim.set_model(theta, mode, X.PREC_FP32, X.ALGO_BATCHED)
        sim.step()
        torch.cuda.synchronize()
        return dict(disp=sim.disp.cpu().numpy().astype(np.float64), mask=sim.mask.cpu().numpy(),
                    pen=sim.pen.cpu().numpy(), count=sim.count.cpu().numpy())
    finally:
        sim.close()


class _Inputs:
    """Device copies of a scene's geometry and step inputs, as a caller that cannot allocate
    would already hold them."""

    def __init__(self, sc, theta, type_off=None, pad_type=None):
        dev = torch.device("cuda", torch.cuda.current_device())
        d = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).to(dev)
        self.tn = np.ascontiguousarray(sc.type_num_nodes, np.int32)
        to = np.concatenate([[0], np.cumsum(self.tn)]) if type_off is None else type_off
        self.type_off = d(to, torch.int32)
        self.type_pos = d(sc.type_pos, torch.float32)
        self.type_nrm = d(sc.type_nrm, torch.float32)
        self.pad_type = d(sc.pad_type if pad_type is None else pad_type, torch.int32)
        self.pad_off = d(sc.node_offsets, torch.int64)
        self.params = d(theta, torch.float32)
        self.ins = [d(sc.obj_type, torch.int32), d(sc.obj_dims, torch.float32),
                    d(sc.obj_pose, torch.float32), d(sc.pad_pose, torch.float32)]
        self.pads = X.etac_noalloc_pads(len(sc.types), self.tn.ctypes.data,
                                        self.type_off.data_ptr(), self.type_pos.data_ptr(),
                                        self.type_nrm.data_ptr(), sc.num_envs, sc.pads_per_env,
                                        sc.max_objects, self.pad_type.data_ptr(),
                                        self.pad_off.data_ptr())
        self.sin = X.etac_step_in(*[t.data_ptr() for t in self.ins])

    def call(self, sc, mode):
        dev = self.params.device
        out = dict(disp=torch.full((sc.total_nodes, 3), float("nan"), device=dev),
                   mask=torch.full((sc.total_nodes,), 7, dtype=torch.uint8, device=dev),
                   pen=torch.full((sc.total_nodes,), float("nan"), device=dev),
                   count=torch.full((sc.num_envs * sc.pads_per_env,), -1, dtype=torch.int32,
                                    device=dev))
        status = torch.full((1,), -1, dtype=torch.int32, device=dev)
        sout = X.etac_step_out(out["disp"].data_ptr(), out["mask"].data_ptr(),
                               out["pen"].data_ptr(), out["count"].data_ptr())
        X.etac_step_forward_noalloc(self.pads, mode, self.params.data_ptr(), self.sin, sout,
                                    status.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in out.items()}
        got["disp"] = got["disp"].astype(np.float64)
        return got, int(status.item())


@pytest.mark.parametrize("mode", MODES)
def test_noalloc_matches_regular_entry_point_and_oracle_twice(mode):
    th = I.make_params(0)
    # (the 16-type uneven workload needs ~280 MB of Omega tables, beyond the static scratch)
    scenes = [I.sphere_press_scene(64, seed=4), I.hand_scene(8, seed=5)]
    for sc in scenes:
        inp = _Inputs(sc, th)
        want = _regular(sc, th, mode)
        ref, _ = PT.oracle_forward_matching(sc, th, mode, want["mask"])
        for call in range(2):
            got, status = inp.call(sc, mode)
            assert status == 0
            np.testing.assert_array_equal(got["mask"], want["mask"])
            np.testing.assert_array_equal(got["count"], want["count"])
            np.testing.assert_array_equal(got["pen"], want["pen"])
            PT.assert_disp_close(sc, got["disp"], want["disp"])
            PT.assert_disp_close(sc, got["disp"], ref["disp"])
            np.testing.assert_array_equal(got["count"], ref["active_count"])


def test_noalloc_device_side_geometry_checks():
    """type_off values that disagree with the host node counts, and a pad type out of range,
    are caught on the device before any indexed access: nothing is written and the status
    word reads ETAC_ERR_INVALID_ARG.  A valid call afterwards is unaffected."""
    th = I.make_params(0)
    sc = I.hand_scene(4, seed=1)
    good = np.concatenate([[0], np.cumsum(sc.type_num_nodes)])
    bad_off = good.copy()
    bad_off[1] += 32                                    # sums no longer match the host counts
    bad_type = np.array(sc.pad_type, np.int32).copy()
    bad_type[3] = len(sc.types)                         # out of range
    for kw in (dict(type_off=bad_off), dict(pad_type=bad_type)):
        got, status = _Inputs(sc, th, **kw).call(sc, X.MODE_FULL)
        assert status == X.ERR_INVALID_ARG
        assert np.isnan(got["disp"]).all() and np.isnan(got["pen"]).all()
        assert (got["mask"] == 7).all() and (got["count"] == -1).all()
    got, status = _Inputs(sc, th).call(sc, X.MODE_FULL)
    assert status == 0
    PT.assert_disp_close(sc, got["disp"], _regular(sc, th, X.MODE_FULL)["disp"])


def test_noalloc_rejects_batches_beyond_its_scratch():
    # 16 pad types of 4096 nodes need 16 * 4096^2 * 4 bytes of Omega alone (> 32 MiB)
    tn = np.full(16, 4096, np.int32)
    one = torch.zeros(4, dtype=torch.int64, device="cuda")
    pads = X.etac_noalloc_pads(16, tn.ctypes.data, one.data_ptr(), one.data_ptr(),
                               one.data_ptr(), 1, 1, 1, one.data_ptr(), one.data_ptr())
    sin = X.etac_step_in(one.data_ptr(), one.data_ptr(), one.data_ptr(), one.data_ptr())
    sout = X.etac_step_out(one.data_ptr(), None, None, None)
    with pytest.raises(X.EtacError) as e:
        X.etac_step_forward_noalloc(pads, 0, one.data_ptr(), sin, sout, 0, 0)
    assert e.value.status == 1 and "bytes of scratch" in str(e.value)
