"""The no-allocation forward entry point (etac_step_forward_noalloc).

Callers that may not allocate device memory while they run -- an application that hands
the whole device heap to its own pool allocator, a real-time loop, or a plugin whose host
program gives it device pointers and no allocator -- use this entry point: its scratch lives
in a static device array in the library.  It must give the same displacements as the regular batched FP32 entry point, on
two calls in a row (the second call reuses the array the first one left behind).  This file
is collected last so that a stop at the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2604_20295_gb300 import build as B
from paper_2604_20295_gb300 import etac as X
from paper_2604_20295_gb300 import inputs as I
from tests import parity as PT

pytestmark = pytest.mark.gpu


def _regular(scene, theta):
    sim = X.TactileSim(scene)
    try:
        sim.set_model(theta, X.MODE_FULL, X.PREC_FP32, X.ALGO_BATCHED)
        sim.step()
        torch.cuda.synchronize()
        return sim.disp.cpu().numpy().astype(np.float64), sim.mask.cpu().numpy()
    finally:
        sim.close()


def test_noalloc_matches_regular_entry_point_twice():
    B.build()
    assert torch.cuda.is_available()
    dev = torch.device("cuda", torch.cuda.current_device())
    th = I.make_params(0)
    scenes = [I.sphere_press_scene(64, seed=4), I.hand_scene(8, seed=5)]
    for sc in scenes:
        tn = np.ascontiguousarray(sc.type_num_nodes, np.int32)
        d = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).to(dev)
        type_off = d(np.concatenate([[0], np.cumsum(tn)]), torch.int32)
        type_pos = d(sc.type_pos, torch.float32)
        type_nrm = d(sc.type_nrm, torch.float32)
        pad_type = d(sc.pad_type, torch.int32)
        pad_off = d(sc.node_offsets, torch.int64)
        params = d(th, torch.float32)
        ins = [d(sc.obj_type, torch.int32), d(sc.obj_dims, torch.float32),
               d(sc.obj_pose, torch.float32), d(sc.pad_pose, torch.float32)]
        pads = X.etac_noalloc_pads(len(sc.types), tn.ctypes.data, type_off.data_ptr(),
                                   type_pos.data_ptr(), type_nrm.data_ptr(), sc.num_envs,
                                   sc.pads_per_env, sc.max_objects, pad_type.data_ptr(),
                                   pad_off.data_ptr())
        sin = X.etac_step_in(*[t.data_ptr() for t in ins])
        want, want_mask = _regular(sc, th)
        for call in range(2):
            disp = torch.full((sc.total_nodes, 3), float("nan"), device=dev)
            mask = torch.zeros(sc.total_nodes, dtype=torch.uint8, device=dev)
            sout = X.etac_step_out(disp.data_ptr(), mask.data_ptr(), None, None)
            X.etac_step_forward_noalloc(pads, X.MODE_FULL, params.data_ptr(), sin, sout,
                                        torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            got = disp.cpu().numpy().astype(np.float64)
            np.testing.assert_array_equal(mask.cpu().numpy(), want_mask)
            PT.assert_disp_close(sc, got, want)


def test_noalloc_rejects_batches_beyond_its_scratch():
    B.build()
    # 16 pad types of 4096 nodes need 16 * 4096^2 * 4 bytes of Omega alone (> 32 MiB)
    tn = np.full(16, 4096, np.int32)
    one = torch.zeros(4, dtype=torch.int64, device="cuda")
    pads = X.etac_noalloc_pads(16, tn.ctypes.data, one.data_ptr(), one.data_ptr(),
                               one.data_ptr(), 1, 1, 1, one.data_ptr(), one.data_ptr())
    sin = X.etac_step_in(one.data_ptr(), one.data_ptr(), one.data_ptr(), one.data_ptr())
    sout = X.etac_step_out(one.data_ptr(), None, None, None)
    with pytest.raises(X.EtacError) as e:
        X.etac_step_forward_noalloc(pads, 0, one.data_ptr(), sin, sout, 0)
    assert e.value.status == 1 and "bytes of scratch" in str(e.value)
