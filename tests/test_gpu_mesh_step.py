"""Mesh objects in the tactile step (ETac Sec. III-A "Overview": contact by signed distance
between the nodes and object meshes): the hand layout pressed into seeded rock meshes
(inputs.mesh_scene) through every forward path and the reverse mode, against the FP64 oracle,
which evaluates the mesh's signed distance from its definition (every triangle, winding-number
sign).  Contact sets must agree outside the 1e-6 mm band, displacements within the FP32
tolerance (BF16: 2e-2 per pad), the reverse mode entry by entry (tests.parity), including the
object-pose gradients through the mesh SDF's Hessian (edges and vertices)."""
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
    assert torch.cuda.is_available()


def _run(sc, th, algo, prec, mode=X.MODE_FULL, meshes=None):
    sim = X.TactileSim(sc)
    try:
        sim.set_model(th, mode, prec, algo)
        sim.set_meshes(meshes)
        sim.step()
        torch.cuda.synchronize()
        return dict(disp=sim.disp.cpu().numpy().astype(np.float64), mask=sim.mask.cpu().numpy(),
                    pen=sim.pen.cpu().numpy().astype(np.float64),
                    count=sim.count.cpu().numpy(), status=sim.poll_status())
    finally:
        sim.close()


@pytest.mark.parametrize("algo,prec", [(X.ALGO_PLAIN, X.PREC_FP32), (X.ALGO_BATCHED, X.PREC_FP32),
                                       (X.ALGO_BATCHED, X.PREC_BF16)])
@pytest.mark.parametrize("mode", [X.MODE_FULL, X.MODE_PENETRATION_ONLY])
def test_mesh_contact_matches_oracle(algo, prec, mode):
    sc = I.mesh_scene(12, seed=3)
    th = I.make_params(0)
    got = _run(sc, th, algo, prec, mode)
    assert got["status"] == 0
    assert got["mask"].sum() > 0
    ref, nband = PT.oracle_forward_matching(sc, th, mode, got["mask"])
    np.testing.assert_array_equal(got["count"], ref["active_count"])
    act = got["mask"] == 1
    # penetration: the distance to the surface, FP64 or FP32 (nodes certainly inside)
    np.testing.assert_allclose(got["pen"][act], ref["pen"][act], rtol=1e-5, atol=2e-5)
    if prec == X.PREC_FP32:
        PT.assert_disp_close(sc, got["disp"], ref["disp"])
    else:
        errs, scale = PT.pad_errors(sc, got["disp"], ref["disp"])
        assert np.all(errs <= 2e-2 * scale + 1e-6), (errs / np.maximum(scale, 1e-30)).max()
        np.testing.assert_allclose(got["disp"][act], ref["disp"][act], rtol=1e-5, atol=1e-4)


def test_mesh_reverse_mode_matches_oracle():
    sc = I.mesh_scene(6, seed=5)
    th = I.make_params(0)
    G = np.random.default_rng(3).normal(size=(sc.total_nodes, 3))
    sim = X.TactileSim(sc)
    try:
        sim.set_model(th, X.MODE_FULL, X.PREC_FP32, X.ALGO_BATCHED)
        sim.set_meshes()
        sim.step()
        torch.cuda.synchronize()
        mask = sim.mask.cpu().numpy()
        G, dropped = PT.condition_upstream(sc, th, G, mask)
        assert len(dropped) <= sc.num_envs * sc.pads_per_env // 2
        g = sim.backward(torch.as_tensor(np.asarray(G, np.float32)).cuda())
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}
        assert sim.poll_status() == 0
    finally:
        sim.close()
    ref = O.backward(sc, th, G, mask_override=mask)
    ref["obj_pose"] = ref["obj_pose"].reshape(got["obj_pose"].shape)
    assert np.abs(ref["obj_pose"]).max() > 0
    PT.assert_grads_close(got, ref, I.param_slices())


def test_mesh_index_outside_the_list_leaves_the_slot_empty():
    """An OBJ_MESH object whose index names no registered mesh is an empty slot: its pads
    output zero, as the oracle gives for an env without objects."""
    sc = I.mesh_scene(4, seed=2)
    th = I.make_params(0)
    got = _run(sc, th, X.ALGO_BATCHED, X.PREC_FP32, meshes=[])   # no meshes registered
    assert got["status"] == 0
    assert not got["mask"].any() and np.all(got["disp"] == 0.0)


def test_set_meshes_checks_its_arguments():
    sc = I.mesh_scene(2, seed=1)
    sim = X.TactileSim(sc)
    try:
        with pytest.raises(X.EtacError) as e:
            X.lib()  # the library is loaded
            st = X.lib().etac_set_meshes(sim.ctx, None, 2, None)
            X._check(sim.ctx, st, "etac_set_meshes")
        assert e.value.status == 1
        with pytest.raises(X.EtacError) as e:
            X.etac_set_meshes(sim.ctx, [0])
        assert e.value.status == 1
    finally:
        sim.close()
