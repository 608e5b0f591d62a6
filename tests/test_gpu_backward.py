"""GPU reverse mode (hand-written FP32 adjoint, etac_step_backward) against the FP64 oracle's
reverse mode and against FP64 central finite differences (step 1e-6) of the GPU FP64 forward
on a 1-env 8x8 pad.  Gradients: object pose (translation + left world-frame rotation), per-node
penetration / u_hat, every propagation-model parameter."""
import math

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


def gpu_grads(scene, theta, G, mode=X.MODE_FULL, algo=X.ALGO_BATCHED, prec=X.PREC_FP32,
              condition=False):
    """Forward + reverse mode on the GPU.  With ``condition`` the upstream gradient of pads
    whose max-pool choice is a near-tie is zeroed first (tests.parity.condition_upstream);
    the gradient used is returned as out["G"]."""
    sim = X.TactileSim(scene)
    try:
        sim.set_model(theta, mode, prec, algo)
        sim.step()
        torch.cuda.synchronize()
        mask = sim.mask.cpu().numpy()
        dropped = []
        if condition:
            G, dropped = PT.condition_upstream(scene, theta, G, mask, mode)
        g = sim.backward(torch.as_tensor(np.asarray(G, np.float32)).cuda())
        torch.cuda.synchronize()
        out = {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}
        out["mask"] = mask
        out["status"] = sim.poll_status()
        out["G"], out["dropped"] = np.asarray(G, np.float64), dropped
    finally:
        sim.close()
    return out


SCENES = {
    "sphere-press": lambda: I.sphere_press_scene(48, seed=3),
    "hand": lambda: I.hand_scene(64, seed=7).subset([0, 5, 9]),
    "uneven": lambda: I.uneven_scene(16, seed=2).subset([1, 4]),
}


@pytest.mark.parametrize("name", sorted(SCENES))
@pytest.mark.parametrize("mode", [X.MODE_FULL, X.MODE_LINEAR_ONLY, X.MODE_RESIDUAL_ONLY,
                                  X.MODE_PENETRATION_ONLY])
def test_backward_matches_oracle(name, mode):
    """Every entry of every gradient against the oracle's reverse mode (tests.parity:
    |g - g_ref| <= 1e-4 (|g_ref| + block max))."""
    sc = SCENES[name]()
    th = I.make_params(0)
    G = np.random.default_rng(1).normal(size=(sc.total_nodes, 3))
    got = gpu_grads(sc, th, G, mode, condition=True)
    assert got["status"] == 0
    npads = sc.num_envs * sc.pads_per_env
    assert len(got["dropped"]) <= npads // 2, got["dropped"]
    PT.oracle_forward_matching(sc, th, mode, got["mask"])
    ref = O.backward(sc, th, got.pop("G"), mode=mode, mask_override=got["mask"])
    ref["obj_pose"] = ref["obj_pose"].reshape(got["obj_pose"].shape)
    worst = PT.assert_grads_close(got, ref, I.param_slices())
    print(f"{name} mode {mode}: worst entry ratio {worst:.2e}, "
          f"{len(got['dropped'])} of {npads} pads dropped (decisions within 1e-6 of their kinks)")


def _f64_forward(sim, sc, th, obj_pose):
    dev = sim.device
    disp = torch.zeros(sc.total_nodes, 3, dtype=torch.float64, device=dev)
    ten = [torch.as_tensor(np.asarray(v, np.float64), device=dev) for v in
           (sc.obj_dims, obj_pose, sc.pad_pose, th)]
    X.etac_forward_f64(sim.ctx, X.etac_model_desc(64, 0, 0, 0), sim.obj_type.data_ptr(),
                       *[t.data_ptr() for t in ten], disp.data_ptr(),
                       torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return disp.cpu().numpy()


@pytest.mark.parametrize("ot", [I.OBJ_SPHERE, I.OBJ_BOX, I.OBJ_CYLINDER, I.OBJ_CAPSULE])
def test_backward_vs_fp64_central_differences(ot):
    """1 env, 8x8 pad: FP64 central differences (h = 1e-6) of the GPU FP64 forward vs the GPU
    FP32 adjoint and vs the oracle adjoint, for the 6 pose components, alpha and 24 sampled
    weights; penetration gradient vs central differences of the oracle with u_hat = d n."""
    sc = I.grad_scene(ot, seed=0)
    th = I.make_params(7).astype(np.float64)
    fw = O.forward(sc, th)
    assert fw["mask"].sum() > 0
    assert np.min(np.abs(fw["phi"])) > 1e-4, "seed puts a node on the contact boundary"
    G = np.random.default_rng(5).normal(size=(sc.total_nodes, 3))
    got = gpu_grads(sc, th.astype(np.float32), G, algo=X.ALGO_PLAIN)
    ref = O.backward(sc, th, G)
    h = 1e-6
    sim = X.TactileSim(sc)
    try:
        sim.set_model(th.astype(np.float32), X.MODE_FULL, X.PREC_FP32, X.ALGO_PLAIN)
        op = sc.obj_pose.astype(np.float64)
        L = lambda pose, theta=th: float((_f64_forward(sim, sc, theta, pose) * G).sum())
        fd_pose = np.zeros(6)
        for a in range(6):
            def pose(sgn):
                o = op.copy()
                if a < 3:
                    o[a] += sgn * h
                else:
                    ax = np.zeros(3)
                    ax[a - 3] = 1.0
                    o[3:] = I._qmul(I._axis_angle(ax, sgn * h), o[3:] / np.linalg.norm(o[3:]))
                return o
            fd_pose[a] = (L(pose(1)) - L(pose(-1))) / (2 * h)
        rng = np.random.default_rng(11)
        idx = [0] + list(rng.choice(np.arange(1, th.size), 24, replace=False))
        fd_par = []
        for k in idx:
            tp, tm = th.copy(), th.copy()
            tp[k] += h
            tm[k] -= h
            fd_par.append((L(op, tp) - L(op, tm)) / (2 * h))
        fd_par = np.array(fd_par)
    finally:
        sim.close()
    scale_p = max(np.abs(fd_pose).max(), 1e-3)
    np.testing.assert_allclose(ref["obj_pose"][0], fd_pose, atol=1e-6 * scale_p, rtol=1e-6)
    np.testing.assert_allclose(got["obj_pose"][0], fd_pose, atol=2e-4 * scale_p, rtol=2e-4)
    scale = max(np.abs(fd_par).max(), 1e-3)
    np.testing.assert_allclose(ref["params"][idx], fd_par, atol=1e-6 * scale, rtol=1e-6)
    np.testing.assert_allclose(got["params"][idx], fd_par, atol=2e-4 * scale, rtol=2e-4)
    # penetration: u_hat_j = d_j n_j with n_j the outward normal; perturb d_j of active nodes
    act = np.nonzero(fw["mask"])[0]
    nrm = fw["disp"][act] / fw["pen"][act][:, None]
    fd_pen = []
    for j_local, j in enumerate(act[:12]):
        def lpen(sgn):
            uh = fw["disp"] * fw["mask"][:, None]
            uh = uh.copy()
            uh[j] = (fw["pen"][j] + sgn * h) * nrm[j_local]
            return float((O.forward(sc, th, mask_override=fw["mask"], uhat_override=uh)["disp"] * G).sum())
        fd_pen.append((lpen(1) - lpen(-1)) / (2 * h))
    fd_pen = np.array(fd_pen)
    sp = max(np.abs(fd_pen).max(), 1e-3)
    np.testing.assert_allclose(got["pen"][act[:12]], fd_pen, atol=2e-4 * sp, rtol=2e-4)


def test_backward_is_bitwise_deterministic():
    sc = I.hand_scene(12, seed=4)
    th = I.make_params(0)
    G = np.random.default_rng(2).normal(size=(sc.total_nodes, 3))
    a = gpu_grads(sc, th, G)
    b = gpu_grads(sc, th, G)
    for k in ("params", "obj_pose", "uhat", "pen"):
        assert np.array_equal(a[k], b[k]), k


def test_autograd_function_and_quaternion_gradient():
    """ETacStep.apply: dL/dparams equals the direct reverse mode; dL/d(quaternion) equals
    FP64 central differences in the raw quaternion components."""
    sc = I.grad_scene(I.OBJ_CAPSULE, seed=2)
    th = I.make_params(3)
    G = torch.as_tensor(np.random.default_rng(8).normal(size=(sc.total_nodes, 3)), dtype=torch.float32).cuda()
    sim = X.TactileSim(sc)
    try:
        sim.set_model(th, X.MODE_FULL, X.PREC_FP32, X.ALGO_BATCHED)
        Step = X.make_step_function()
        p = torch.as_tensor(th).cuda().requires_grad_(True)
        pose = torch.as_tensor(sc.obj_pose).cuda().requires_grad_(True)
        disp = Step.apply(sim, p, pose)
        (disp * G).sum().backward()
        direct = sim.backward(G)
        torch.testing.assert_close(p.grad, direct["params"])
        gq = pose.grad.cpu().numpy().astype(np.float64)
        sim64 = X.TactileSim(sc)
        sim64.set_model(th, X.MODE_FULL, X.PREC_FP32, X.ALGO_PLAIN)
        Gn = G.cpu().numpy().astype(np.float64)
        op = sc.obj_pose.astype(np.float64)
        h = 1e-6
        for a in range(7):
            o1, o2 = op.copy(), op.copy()
            o1[a] += h
            o2[a] -= h
            fd = (float((_f64_forward(sim64, sc, th.astype(np.float64), o1) * Gn).sum()) -
                  float((_f64_forward(sim64, sc, th.astype(np.float64), o2) * Gn).sum())) / (2 * h)
            assert abs(gq[a] - fd) <= 2e-4 * max(1.0, abs(fd)), (a, gq[a], fd)
        sim64.close()
    finally:
        sim.close()


def test_fit_reduces_loss():
    """Eq. 5 calibration on oracle targets: Adam on the MSE of passive displacements lowers
    the loss and moves alpha toward the target model's."""
    from paper_2604_20295_gb300 import fit as F
    sc = I.sphere_press_scene(64, seed=12)
    th0, th_t = I.make_params(0), I.make_params(42)
    target = O.forward(sc, th_t)["disp"]
    hist = F.fit(sc, th0, target, iters=40, lr=3e-3)
    assert hist["loss"][-1] < 0.5 * hist["loss"][0], hist["loss"][::10]
    assert abs(hist["params"][0] - th_t[0]) < abs(th0[0] - th_t[0])


def test_backward_refuses_a_step_that_is_not_the_last():
    """The context keeps only its last forward's state: differentiating an earlier step id
    fails with ETAC_ERR_STATE and enqueues nothing; the last id (and 0) work."""
    sc = I.sphere_press_scene(8, seed=1)
    th = I.make_params(0)
    G = torch.as_tensor(np.random.default_rng(3).normal(size=(sc.total_nodes, 3)),
                        dtype=torch.float32).cuda()
    sim = X.TactileSim(sc)
    try:
        sim.set_model(th, X.MODE_FULL, X.PREC_FP32, X.ALGO_BATCHED)
        assert sim.last_step() == 0
        sim.step()
        first = sim.last_step()
        sim.step()
        second = sim.last_step()
        assert second == first + 1
        with pytest.raises(X.EtacError) as e:
            sim.backward(G, step_id=first)
        assert e.value.status == 2 and "not the last forward" in str(e.value)
        a = sim.backward(G, step_id=second)
        b = sim.backward(G)
        for k in a:
            assert torch.equal(a[k], b[k]), k
    finally:
        sim.close()


def test_autograd_rollout_of_two_steps_on_one_context():
    """Two ETacStep.apply calls on one context before backward (a two-step rollout): each
    step's gradient equals that step differentiated on its own, although the second forward
    replaced the context's saved state of the first."""
    sc = I.grad_scene(I.OBJ_SPHERE, seed=1)
    th = I.make_params(2)
    rng = np.random.default_rng(4)
    G1, G2 = (torch.as_tensor(rng.normal(size=(sc.total_nodes, 3)), dtype=torch.float32).cuda()
              for _ in range(2))
    pose0 = torch.as_tensor(sc.obj_pose, dtype=torch.float32).cuda().reshape(-1)
    pose1 = pose0.clone()
    pose1[2] -= 0.3                                   # the second step presses deeper
    sim = X.TactileSim(sc)
    try:
        sim.set_model(th, X.MODE_FULL, X.PREC_FP32, X.ALGO_BATCHED)
        Step = X.make_step_function()
        p = torch.as_tensor(th).cuda().requires_grad_(True)
        q0 = pose0.clone().requires_grad_(True)
        q1 = pose1.clone().requires_grad_(True)
        d0 = Step.apply(sim, p, q0)
        d1 = Step.apply(sim, p, q1)
        ((d0 * G1).sum() + (d1 * G2).sum()).backward()
        single = []
        for pose, G in ((pose0, G1), (pose1, G2)):
            pp = torch.as_tensor(th).cuda().requires_grad_(True)
            qq = pose.clone().requires_grad_(True)
            (Step.apply(sim, pp, qq) * G).sum().backward()
            single.append((pp.grad, qq.grad))
        torch.testing.assert_close(p.grad, single[0][0] + single[1][0], rtol=1e-5, atol=1e-6)
        torch.testing.assert_close(q0.grad, single[0][1], rtol=0, atol=0)
        torch.testing.assert_close(q1.grad, single[1][1], rtol=0, atol=0)
    finally:
        sim.close()
