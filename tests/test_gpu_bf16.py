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
