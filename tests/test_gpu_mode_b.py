"""Mode B: the contact result supplied by the caller (etac_step_in.active_mask_in /
active_disp_in).  Eq. 1 and Eq. 4 take the active nodes' local displacements U_a as their
input; an external contact pipeline can hand them over directly.  Every forward path (plain
FP32, batched FP32, batched BF16) in every mode must match the oracle run with the same mask
and u_hat overrides, and both reverse-mode implementations must match the oracle's reverse
mode entry by entry (dL/du_hat and the parameter gradients; pose and penetration gradients are
zero).  Passive entries of the supplied u_hat are ignored."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_20295_gb300 import build as B
from paper_2604_20295_gb300 import etac as X
from paper_2604_20295_gb300 import inputs as I
from tests import parity as PT

pytestmark = pytest.mark.gpu
MODES = [X.MODE_FULL, X.MODE_LINEAR_ONLY, X.MODE_RESIDUAL_ONLY, X.MODE_PENETRATION_ONLY]
SCENES = {
    "hand": lambda: I.hand_scene(6, seed=11).subset([0, 2, 5]),
    "uneven": lambda: I.uneven_scene(12, seed=6).subset([3, 7]),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    X.lib()
    assert torch.cuda.is_available()


def _given(sc, seed):
    """A seeded active set (about a fifth of each pad's nodes, one pad left without contact)
    and u_hat (N(0, 0.5) mm), with garbage in the passive entries."""
    rng = np.random.default_rng(seed)
    mask = (rng.random(sc.total_nodes) < 0.2).astype(np.uint8)
    offs = sc.node_offsets
    mask[offs[1]:offs[2]] = 0
    uh = rng.normal(0.0, 0.5, size=(sc.total_nodes, 3)).astype(np.float32)
    uh_in = uh.copy()
    uh_in[mask == 0] = 1e3
    return mask, uh.astype(np.float64) * mask[:, None], uh_in


@pytest.mark.parametrize("name", sorted(SCENES))
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("algo,prec", [(X.ALGO_PLAIN, X.PREC_FP32), (X.ALGO_BATCHED, X.PREC_FP32),
                                       (X.ALGO_BATCHED, X.PREC_BF16)])
def test_given_contact_forward_matches_oracle(name, mode, algo, prec):
    sc = SCENES[name]()
    th = I.make_params(0)
    mask, uh, uh_in = _given(sc, 5)
    ref = O.forward(sc, th, mode=mode, mask_override=mask, uhat_override=uh)
    sim = X.TactileSim(sc)
    try:
        sim.set_model(th, mode, prec, algo)
        sim.pen.fill_(float("nan"))
        sim.step(uhat_in=torch.as_tensor(uh_in).cuda(), mask_in=torch.as_tensor(mask).cuda())
        torch.cuda.synchronize()
        assert sim.poll_status() == 0
        disp = sim.disp.cpu().numpy().astype(np.float64)
        np.testing.assert_array_equal(sim.mask.cpu().numpy(), mask)
        np.testing.assert_array_equal(sim.count.cpu().numpy(), ref["active_count"])
        assert np.all(sim.pen.cpu().numpy() == 0.0)
    finally:
        sim.close()
    if prec == X.PREC_FP32:
        PT.assert_disp_close(sc, disp, ref["disp"])
    else:
        errs, scale = PT.pad_errors(sc, disp, ref["disp"])
        assert np.all(errs <= 2e-2 * scale + 1e-6), (errs / np.maximum(scale, 1e-30)).max()
        act = mask == 1
        np.testing.assert_allclose(disp[act], uh[act], rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("name", sorted(SCENES))
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("algo", [X.ALGO_PLAIN, X.ALGO_BATCHED])
def test_given_contact_reverse_matches_oracle(name, mode, algo):
    sc = SCENES[name]()
    th = I.make_params(0)
    mask, uh, uh_in = _given(sc, 8)
    G = np.random.default_rng(2).normal(size=(sc.total_nodes, 3))
    G, dropped = PT.condition_upstream(sc, th, G, mask, mode, uhat=uh)
    assert len(dropped) <= sc.num_envs * sc.pads_per_env // 2
    ref = O.backward(sc, th, G, mode=mode, mask_override=mask, uhat_override=uh)
    sim = X.TactileSim(sc)
    try:
        sim.set_model(th, mode, X.PREC_FP32, algo)
        sim.step(uhat_in=torch.as_tensor(uh_in).cuda(), mask_in=torch.as_tensor(mask).cuda())
        g = sim.backward(torch.as_tensor(np.asarray(G, np.float32)).cuda())
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}
        assert sim.poll_status() == 0
    finally:
        sim.close()
    assert np.all(got["obj_pose"] == 0.0) and np.all(got["pen"] == 0.0)
    assert np.all(ref["obj_pose"] == 0.0) and np.all(ref["pen"] == 0.0)
    got.pop("obj_pose"), got.pop("pen")
    PT.assert_grads_close(got, ref, I.param_slices())


def test_given_contact_needs_both_buffers():
    sc = I.hand_scene(2, seed=1)
    sim = X.TactileSim(sc)
    try:
        sim.set_model(I.make_params(0), X.MODE_FULL, X.PREC_FP32, X.ALGO_BATCHED)
        u = torch.zeros(sc.total_nodes, 3, device="cuda")
        for sin in (X.etac_step_in(None, None, None, None, u.data_ptr(), None),
                    X.etac_step_in(None, None, None, None, None, sim.mask.data_ptr())):
            with pytest.raises(X.EtacError) as e:
                X.etac_step_forward(sim.ctx, sin, sim.step_out(), 0)
            assert e.value.status == 1 and "together" in str(e.value)
    finally:
        sim.close()
