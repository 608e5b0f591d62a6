"""GPU tests of the BF16 tensor-core algorithm (tcgen05 propagation GEMM with the decoder fused
in its epilogue) against the FP64 oracle.  Contact sets are computed exactly as in the FP32
algorithms and must match bit for bit (outside the 1e-6 mm band); active nodes keep u_hat in
FP32.  Passive displacements carry BF16 operand rounding (Omega, u_hat, h0, beta, D2 with FP32
accumulation): the bound used here is 2e-2 of the pad's largest displacement, and the measured
max / RMS errors are printed (they are reported per configuration)."""
import numpy as np
import pytest
import torch

from paper_2604_20295_gb300 import build as B
from paper_2604_20295_gb300 import etac as X
from paper_2604_20295_gb300 import inputs as I
from tests import parity as PT
from tests.test_gpu_forward import run

pytestmark = pytest.mark.gpu
BF16_REL = 2e-2


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    X.lib()
    assert torch.cuda.is_available()


def check_bf16(scene, theta, mode=X.MODE_FULL):
    got = run(scene, theta, mode, algo=X.ALGO_BATCHED, precision=X.PREC_BF16)
    assert got["status"] == 0, got["status"]
    ref, _ = PT.oracle_forward_matching(scene, theta, mode, got["mask"])
    errs, scale = PT.pad_errors(scene, got["disp"], ref["disp"])
    rel = errs / np.maximum(scale, 1e-30)
    assert np.all(errs <= BF16_REL * scale + 1e-6), f"worst pad rel err {rel.max():.3e}"
    act = got["mask"] > 0
    # active nodes keep u_hat in FP32 (not BF16); away from surfaces and ties it is evaluated in
    # plain FP32, whose coordinate rounding bounds the absolute error by ~1e-4 mm
    du = np.linalg.norm(got["disp"][act] - ref["disp"][act], axis=1)
    assert np.all(du <= 1e-5 * np.linalg.norm(ref["disp"][act], axis=1) + 1e-4), du.max()
    d = np.linalg.norm(got["disp"] - ref["disp"], axis=1)
    print(f"BF16 {scene.name} mode {mode}: max err {d.max():.3e} mm, rms {np.sqrt((d**2).mean()):.3e}"
          f" mm, worst pad rel {rel.max():.3e}")
    return got, ref


@pytest.mark.parametrize("mode", [X.MODE_FULL, X.MODE_LINEAR_ONLY, X.MODE_RESIDUAL_ONLY,
                                  X.MODE_PENETRATION_ONLY])
def test_bf16_sphere_press_100_steps(mode):
    check_bf16(I.sphere_press_scene(100, seed=0), I.make_params(0), mode)


def propagation_bound(scene, theta, mask, ref):
    """Entry-wise bound on the BF16 propagation term (Eq. 1, Omega U_a) of every passive node,
    derived from the arithmetic of the tensor-core contraction: Omega (an FP32 exp, within
    1e-6 relative) and u_hat are each rounded once to BF16 (8 significant bits, round to
    nearest: relative error at most 2^-8 each, so a product is within 2^-7 + 2^-16 of its
    exact value); the products are exact in FP32 and summed in FP32 (m terms: at most
    m 2^-24 relative of the sum of magnitudes); u_hat itself comes from FP32 arithmetic,
    within 1e-5 |u_hat| + 1e-4 mm of the oracle's.  So
        |L_ic - L_ref,ic| <= (2^-7 + 2^-16 + 1e-5 + 1e-6 + m 2^-24) sum_j Omega_ij |u_jc|
                             + 1e-4 sum_j Omega_ij
    over the pad's m active nodes j, with the oracle's u_hat."""
    alpha = float(theta[0])
    offs = scene.node_offsets
    bound = np.zeros((scene.total_nodes, 3))
    for p in range(len(scene.pad_type)):
        a, b = offs[p], offs[p + 1]
        act = mask[a:b] > 0
        m = int(act.sum())
        if m == 0:
            continue
        pos = scene.types[scene.pad_type[p]].pos.astype(np.float64)
        om = np.exp(-alpha * np.linalg.norm(pos[:, None, :] - pos[None, act, :], axis=2))
        u = np.abs(ref["disp"][a:b][act])
        rel = 2.0 ** -7 + 2.0 ** -16 + 1e-5 + 1e-6 + m * 2.0 ** -24
        bound[a:b] = rel * (om @ u) + 1e-4 * om.sum(1)[:, None]
    return bound


@pytest.mark.parametrize("which", ["sphere_press", "hand"])
def test_bf16_propagation_within_its_rounding_bound(which):
    """The tensor-core contraction alone (LINEAR_ONLY: passive nodes get Omega U_a), entry by
    entry against the bound its BF16 operands and FP32 sums imply."""
    if which == "sphere_press":
        sc = I.sphere_press_scene(100, seed=0)
    else:
        sc = I.hand_scene(256, seed=3).subset(np.random.default_rng(1).choice(256, 24, replace=False))
    th = I.make_params(0)
    got = run(sc, th, X.MODE_LINEAR_ONLY, algo=X.ALGO_BATCHED, precision=X.PREC_BF16)
    assert got["status"] == 0
    ref, _ = PT.oracle_forward_matching(sc, th, X.MODE_LINEAR_ONLY, got["mask"])
    pas = got["mask"] == 0
    bound = propagation_bound(sc, th, got["mask"], ref)
    err = np.abs(got["disp"] - ref["disp"])[pas]
    b = bound[pas]
    worst = float((err / np.maximum(b, 1e-300)).max()) if err.size else 0.0
    print(f"BF16 propagation {which}: worst error / derived bound {worst:.3f}")
    assert np.all(err <= b), f"worst error / bound {worst:.3f}"
    assert (got["mask"] > 0).sum() > 0


def test_bf16_hand_scene_sampled_envs():
    full = I.hand_scene(512, seed=3)
    sc = full.subset(np.random.default_rng(0).choice(512, 40, replace=False))
    check_bf16(sc, I.make_params(0))


def test_bf16_partial_tiles_and_uneven_types():
    """Instance counts that do not fill a 64-instance tile, 8x8 .. 64x64 pads (16 types)."""
    full = I.uneven_scene(40, seed=5)
    check_bf16(full.subset(np.arange(0, 40, 3)), I.make_params(1))


def test_bf16_full_size_sampled_outputs():
    full = I.hand_scene(4096, seed=2)
    th = I.make_params(0)
    got = run(full, th, algo=X.ALGO_BATCHED, precision=X.PREC_BF16)
    assert got["status"] == 0
    offs = full.node_offsets
    for e in np.sort(np.random.default_rng(1).choice(4096, 12, replace=False)):
        sub = full.subset([e])
        a, b = offs[e * 6], offs[e * 6 + 6]
        ref, _ = PT.oracle_forward_matching(sub, th, 0, got["mask"][a:b])
        errs, scale = PT.pad_errors(sub, got["disp"][a:b], ref["disp"])
        assert np.all(errs <= BF16_REL * scale + 1e-6)


def test_bf16_repeat_is_bitwise_deterministic():
    sc = I.hand_scene(70, seed=9)
    a = run(sc, I.make_params(0), algo=X.ALGO_BATCHED, precision=X.PREC_BF16)
    b = run(sc, I.make_params(0), algo=X.ALGO_BATCHED, precision=X.PREC_BF16, steps=3)
    assert np.array_equal(a["disp"], b["disp"])


def test_bf16_step_after_other_steps_on_the_context():
    """The BF16 front kernel rewrites only the B-operand entries of nodes that are or were
    active.  Steps on other inputs, and an FP32 model's forward and reverse mode on the same
    context in between, must leave the next BF16 step bitwise equal to a fresh context's."""
    sa, sb = I.hand_scene(16, seed=31), I.hand_scene(16, seed=32)
    th = I.make_params(0)
    sim = X.TactileSim(sa)
    try:
        def load(sc):
            for k in ("obj_type", "obj_dims", "obj_pose", "pad_pose"):
                getattr(sim, k).copy_(torch.as_tensor(getattr(sc, k)))
        sim.set_model(th, X.MODE_FULL, X.PREC_BF16, X.ALGO_BATCHED)
        sim.step()
        load(sb)
        sim.set_model(th, X.MODE_FULL, X.PREC_FP32, X.ALGO_BATCHED)
        sim.step()
        sim.backward(torch.ones(sb.total_nodes, 3, device="cuda"))
        sim.set_model(th, X.MODE_FULL, X.PREC_BF16, X.ALGO_BATCHED)
        for sc in (sb, sa):
            load(sc)
            sim.step()
            torch.cuda.synchronize()
            got = sim.disp.cpu().numpy()
            fresh = X.TactileSim(sc)
            try:
                fresh.set_model(th, X.MODE_FULL, X.PREC_BF16, X.ALGO_BATCHED)
                fresh.step()
                torch.cuda.synchronize()
                assert np.array_equal(got, fresh.disp.cpu().numpy())
            finally:
                fresh.close()
    finally:
        sim.close()
