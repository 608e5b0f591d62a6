"""GPU parity of the FP32 forward algorithms against the FP64 oracle, through the C ABI:
the plain algorithm (one CTA per pad, literal Eq. 1 / Eq. 4) and the batched algorithm (one
persistent launch, per-type tables, factored network).  Contact sets bit-exact outside the
1e-6 mm band, displacements within 1e-5 normwise per pad."""
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
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def run(scene, theta, mode=X.MODE_FULL, algo=X.ALGO_PLAIN, precision=X.PREC_FP32, steps=1):
    sim = X.TactileSim(scene)
    try:
        sim.set_model(theta, mode, precision, algo)
        for _ in range(steps):
            sim.step()
        torch.cuda.synchronize()
        out = dict(disp=sim.disp.cpu().numpy().astype(np.float64), mask=sim.mask.cpu().numpy(),
                   pen=sim.pen.cpu().numpy().astype(np.float64), count=sim.count.cpu().numpy(),
                   status=sim.poll_status())
    finally:
        sim.close()
    return out


ALGOS = [X.ALGO_PLAIN, X.ALGO_BATCHED]


def check(scene, theta, mode=X.MODE_FULL, **kw):
    got = run(scene, theta, mode, **kw)
    ref, nband = PT.oracle_forward_matching(scene, theta, mode, got["mask"])
    err = PT.assert_disp_close(scene, got["disp"], ref["disp"])
    act = got["mask"] > 0
    np.testing.assert_allclose(got["pen"][act], ref["pen"][act], rtol=1e-5, atol=1e-7)
    assert np.all(got["pen"][~act] == 0)
    np.testing.assert_array_equal(got["count"], ref["active_count"])
    assert got["status"] == 0
    return got, ref, err, nband


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("mode", [X.MODE_FULL, X.MODE_LINEAR_ONLY, X.MODE_RESIDUAL_ONLY,
                                  X.MODE_PENETRATION_ONLY])
def test_sphere_press_100_steps(mode, algo):
    """16x16 flat pad, sphere r = 5 mm pressed 0-2 mm, 100 seeded steps (one env each)."""
    sc = I.sphere_press_scene(100, seed=0)
    got, ref, err, _ = check(sc, I.make_params(0), mode, algo=algo)
    assert got["mask"].sum() > 100


@pytest.mark.parametrize("algo", ALGOS)
def test_hand_scene_sampled_envs(algo):
    """Curved 16x32 fingertips + flat 32x64 palm, random primitives; 40 sampled envs."""
    full = I.hand_scene(512, seed=3)
    sc = full.subset(np.random.default_rng(0).choice(512, 40, replace=False))
    got, ref, err, nband = check(sc, I.make_params(0), algo=algo)
    frac = got["count"] / sc.pad_nodes
    assert 0.05 < frac.mean() < 0.45


@pytest.mark.parametrize("algo", ALGOS)
def test_hand_scene_full_size_sampled_outputs(algo):
    """4,096 environments (18.9 M nodes) in one launch, the benchmark's configuration;
    outputs of sampled envs vs oracle."""
    full = I.hand_scene(4096, seed=2)
    th = I.make_params(0)
    got = run(full, th, algo=algo)
    envs = np.sort(np.random.default_rng(1).choice(4096, 12, replace=False))
    offs = full.node_offsets
    for e in envs:
        sub = full.subset([e])
        a, b = offs[e * 6], offs[e * 6 + 6]
        ref, _ = PT.oracle_forward_matching(sub, th, 0, got["mask"][a:b])
        PT.assert_disp_close(sub, got["disp"][a:b], ref["disp"])
        np.testing.assert_array_equal(got["count"][e * 6:e * 6 + 6], ref["active_count"])


@pytest.mark.parametrize("algo", ALGOS)
def test_uneven_pads_and_multiple_objects(algo):
    """Pads of 8x8 .. 64x64 nodes at 0.5-2 mm pitch, 1-3 primitives per env (union SDF)."""
    full = I.uneven_scene(64, seed=5)
    sc = full.subset(np.arange(0, 64, 4))
    check(sc, I.make_params(1), algo=algo)


@pytest.mark.parametrize("algo", ALGOS)
def test_no_contact_gives_zero_and_edge_sizes(algo):
    """Objects far away: zero displacement, zero counts; single-node and 1xN pads."""
    types = [I.flat_pad(1, 1, 1.0), I.flat_pad(1, 7, 1.0), I.flat_pad(5, 3, 0.5)]
    objs = {0: (I.OBJ_SPHERE, (3, 0, 0), (0, 0, 50, 0, 0, 0, 1)),
            1: (I.OBJ_BOX, (2, 2, 2), (0.1, 0.1, 1.5, 0, 0, 0, 1))}
    poses = [[0, 0, 0, 0, 0, 0, 1]] * 6
    sc = I.custom_scene(types, [0, 1, 2, 0, 1, 2], objs, poses, 2, 1)
    got, ref, _, _ = check(sc, I.make_params(2), algo=algo)
    assert np.all(got["disp"][:sc.node_offsets[3]] == 0)
    assert got["count"][3:].sum() > 0


@pytest.mark.parametrize("algo", ALGOS)
def test_nonfinite_pose_is_latched(algo):
    """A NaN object pose zeroes that env's pads and latches ETAC_ERR_NONFINITE; other envs
    are unaffected."""
    sc = I.sphere_press_scene(4, seed=1)
    sc.obj_pose[7 * 2 + 1] = np.nan
    got = run(sc, I.make_params(0), algo=algo)
    assert got["status"] == 6
    offs = sc.node_offsets
    assert np.all(got["disp"][offs[2]:offs[3]] == 0)
    good = sc.subset([0, 1, 3])
    ref = O.forward(good, I.make_params(0))
    g = np.concatenate([got["disp"][offs[0]:offs[2]], got["disp"][offs[3]:offs[4]]])
    PT.assert_disp_close(good, g, ref["disp"])


@pytest.mark.parametrize("algo", ALGOS)
def test_repeat_is_bitwise_deterministic(algo):
    sc = I.hand_scene(16, seed=9)
    a = run(sc, I.make_params(0), algo=algo)
    b = run(sc, I.make_params(0), algo=algo, steps=2)
    assert np.array_equal(a["disp"], b["disp"]) and np.array_equal(a["mask"], b["mask"])


@pytest.mark.parametrize("algo,prec", [(a, X.PREC_FP32) for a in ALGOS] +
                         [(X.ALGO_BATCHED, X.PREC_BF16)])
def test_cuda_graph_replay_with_new_inputs(algo, prec):
    """The step captured once in a CUDA graph and replayed after the input poses are
    overwritten in place gives the same result as an eager step on those inputs (the BF16
    step is four launches; the FP32 steps one)."""
    sc0 = I.hand_scene(24, seed=21)
    sc1 = I.hand_scene(24, seed=22)
    th = I.make_params(0)
    sim = X.TactileSim(sc0)
    try:
        sim.set_model(th, X.MODE_FULL, prec, algo)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            sim.step()          # warm-up outside capture
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                sim.step()
        torch.cuda.current_stream().wait_stream(s)
        for sc in (sc1, sc0, sc1):
            sim.obj_type.copy_(torch.as_tensor(sc.obj_type))
            sim.obj_dims.copy_(torch.as_tensor(sc.obj_dims))
            sim.obj_pose.copy_(torch.as_tensor(sc.obj_pose))
            sim.pad_pose.copy_(torch.as_tensor(sc.pad_pose))
            sim.disp.zero_()
            g.replay()
            torch.cuda.synchronize()
            got = sim.disp.cpu().numpy().astype(np.float64)
            eager = run(sc, th, algo=algo, precision=prec)
            assert np.array_equal(got, eager["disp"])
    finally:
        sim.close()


def test_fp64_forward_matches_oracle():
    """The FP64 instantiation (used only by finite-difference checks) equals the oracle to
    ~1e-12 on small pads with every primitive type."""
    for ot in (I.OBJ_SPHERE, I.OBJ_BOX, I.OBJ_CYLINDER, I.OBJ_CAPSULE):
        sc = I.grad_scene(ot)
        th = I.make_params(7).astype(np.float64)
        sim = X.TactileSim(sc)
        try:
            dev = sim.device
            disp = torch.zeros(sc.total_nodes, 3, dtype=torch.float64, device=dev)
            args = [torch.as_tensor(a, dtype=torch.float64, device=dev) for a in
                    (sc.obj_dims, sc.obj_pose, sc.pad_pose, th)]
            X.etac_forward_f64(sim.ctx, X.etac_model_desc(64, 0, 0, 0), sim.obj_type.data_ptr(),
                               *[a.data_ptr() for a in args], disp.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            got = disp.cpu().numpy()
        finally:
            sim.close()
        ref = O.forward(sc, th)
        np.testing.assert_allclose(got, ref["disp"], rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("prec", [X.PREC_FP32, X.PREC_BF16])
def test_step_into_alternate_output_buffer(prec):
    """A step written into a caller's buffer equals the step into the context's own buffer, and
    a buffer of the wrong shape or type is rejected before anything runs."""
    sc = I.hand_scene(12, seed=31)
    sim = X.TactileSim(sc)
    try:
        sim.set_model(I.make_params(0), X.MODE_FULL, prec, X.ALGO_BATCHED)
        sim.step()
        torch.cuda.synchronize()
        ref = sim.disp.clone()
        alt = torch.full_like(sim.disp, float("nan"))
        out = sim.step(disp=alt)
        torch.cuda.synchronize()
        assert out is alt and torch.equal(alt, ref)
        with pytest.raises(X.EtacError):
            sim.step(disp=torch.empty(3, 3, device=sim.disp.device))
        with pytest.raises(X.EtacError):
            sim.step(disp=torch.empty_like(sim.disp, dtype=torch.float64))
    finally:
        sim.close()
