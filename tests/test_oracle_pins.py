"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics (CPU only).

Each test checks the oracle against something other than itself: closed-form contact
geometry, the dyadic special case of Eq. 1 (golden file), superposition / linearity and
symmetry that Eq. 1 implies, brute force over activation patterns, the m = 0 reading, and an
independent torch float64 restatement (library linear / relu / amax / cdist and autograd).
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_20295_gb300 import inputs as I
from tests import torch_ref as TR

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LN2 = math.log(2.0)


def _theta(seed=0, alpha=None):
    th = I.make_params(seed).astype(np.float64)
    if alpha is not None:
        th[0] = alpha
    return th


def _flat_scene(rows, cols, pitch=1.0, obj=None, pad_pose=(0, 0, 0, 0, 0, 0, 1)):
    objs = {} if obj is None else {0: obj}
    return I.custom_scene([I.flat_pad(rows, cols, pitch)], [0], objs, [pad_pose], 1, 1)


def _load_golden():
    rows = []
    with open(os.path.join(GOLDEN, "single_node_decay.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                dr, dc, fr = line.split()
                rows.append((int(dr), int(dc), float(fr)))
    return rows


# ----------------------------------------------------------------- contact geometry


def test_no_contact_gives_zero():
    """Zero penetration gives zero displacement (m = 0 reading), even with non-zero biases."""
    sc = _flat_scene(8, 8, obj=(I.OBJ_SPHERE, (5, 0, 0), (0, 0, 5.5, 0, 0, 0, 1)))
    out = O.forward(sc, _theta())
    assert out["mask"].sum() == 0
    assert np.all(out["disp"] == 0.0) and np.all(out["pen"] == 0.0)


@pytest.mark.parametrize("R,delta,cx,cy", [(5.0, 1.3, 0.25, -0.4), (12.0, 2.7, -1.1, 0.6)])
def test_sphere_on_flat_pad_closed_form(R, delta, cx, cy):
    """Sphere of radius R, centre (cx, cy, R - delta) over a flat pad in z = 0: a node at
    horizontal distance rho is inside iff rho^2 + (R-delta)^2 < R^2, its penetration is
    R - sqrt(rho^2 + (R-delta)^2), and it moves radially away from the centre by that depth,
    so u_z = -d (R-delta)/(R-d) and u_xy = d (x-cx, y-cy)/(R-d)."""
    sc = _flat_scene(16, 16, obj=(I.OBJ_SPHERE, (R, 0, 0), (cx, cy, R - delta, 0, 0, 0, 1)))
    out = O.forward(sc, _theta(), mode=O.MODE_LINEAR_ONLY)
    # the scene stores float32 inputs; the closed form uses the same stored values
    cx, cy, h = (float(v) for v in sc.obj_pose[:3])
    R = float(sc.obj_dims[0])
    P = sc.types[0].pos.astype(np.float64)
    rho2 = (P[:, 0] - cx) ** 2 + (P[:, 1] - cy) ** 2
    inside = rho2 + h ** 2 < R * R
    np.testing.assert_array_equal(out["mask"].astype(bool), inside)
    d = np.maximum(0.0, R - np.sqrt(rho2 + h ** 2))
    np.testing.assert_allclose(out["pen"], d, atol=1e-12)
    a = inside
    assert a.sum() > 10
    np.testing.assert_allclose(out["disp"][a, 2], -d[a] * h / (R - d[a]), atol=1e-12)
    np.testing.assert_allclose(out["disp"][a, 0], d[a] * (P[a, 0] - cx) / (R - d[a]), atol=1e-12)
    np.testing.assert_allclose(out["disp"][a, 1], d[a] * (P[a, 1] - cy) / (R - d[a]), atol=1e-12)


@pytest.mark.parametrize("R,delta,cx,cy", [(5.0, 1.3, 0.25, -0.4)])
def test_penetration_only_is_the_contact_field(R, delta, cx, cy):
    """Penetration-only mode (no Eq. 1 term, no residual): the same closed-form sphere contact
    displacement on the active nodes and exactly zero on every passive node.  Its reverse mode
    passes dL/dU of active nodes straight to u_hat, and no parameter gets a gradient."""
    sc = _flat_scene(16, 16, obj=(I.OBJ_SPHERE, (R, 0, 0), (cx, cy, R - delta, 0, 0, 0, 1)))
    th = _theta(seed=3)
    out = O.forward(sc, th, mode=O.MODE_PENETRATION_ONLY)
    cx, cy, h = (float(v) for v in sc.obj_pose[:3])
    R = float(sc.obj_dims[0])
    P = sc.types[0].pos.astype(np.float64)
    rho2 = (P[:, 0] - cx) ** 2 + (P[:, 1] - cy) ** 2
    inside = rho2 + h ** 2 < R * R
    np.testing.assert_array_equal(out["mask"].astype(bool), inside)
    d = np.maximum(0.0, R - np.sqrt(rho2 + h ** 2))
    a = inside
    np.testing.assert_allclose(out["disp"][a, 2], -d[a] * h / (R - d[a]), atol=1e-12)
    np.testing.assert_allclose(out["disp"][a, 0], d[a] * (P[a, 0] - cx) / (R - d[a]), atol=1e-12)
    assert np.all(out["disp"][~a] == 0.0)
    G = np.random.default_rng(0).normal(size=(sc.total_nodes, 3))
    g = O.backward(sc, th, G, mode=O.MODE_PENETRATION_ONLY)
    assert np.all(g["params"] == 0.0)
    np.testing.assert_array_equal(g["uhat"][a], G[a])
    assert np.all(g["uhat"][~a] == 0.0)


def test_box_face_flat_patch():
    """A box pressed face-down by delta: a node under its footprint is pushed out through the
    nearest face -- the bottom face (penetration delta, displacement (0, 0, -delta)) unless a
    side face is nearer, in which case it moves sideways by its distance to that face; nodes
    outside the footprint stay passive."""
    delta = 0.8
    sc = _flat_scene(12, 12, obj=(I.OBJ_BOX, (3.0, 2.0, 4.0), (0.25, 0.5, 4.0 - delta, 0, 0, 0, 1)))
    out = O.forward(sc, _theta(), mode=O.MODE_LINEAR_ONLY)
    cz = float(sc.obj_pose[2])
    delta = 4.0 - cz                     # stored float32 height
    P = sc.types[0].pos
    inside = (np.abs(P[:, 0] - 0.25) < 3.0) & (np.abs(P[:, 1] - 0.5) < 2.0)
    np.testing.assert_array_equal(out["mask"].astype(bool), inside)
    dx = 3.0 - np.abs(P[:, 0] - 0.25)
    dy = 2.0 - np.abs(P[:, 1] - 0.5)
    for i in np.nonzero(inside)[0]:
        m = min(dx[i], dy[i], delta)
        if dx[i] == m:
            exp = (m * np.sign(P[i, 0] - 0.25), 0, 0)
        elif dy[i] == m:
            exp = (0, m * np.sign(P[i, 1] - 0.5), 0)
        else:
            exp = (0, 0, -delta)
        assert abs(out["pen"][i] - m) < 1e-12
        np.testing.assert_allclose(out["disp"][i], exp, atol=1e-12)
    assert (out["pen"][inside] == delta).sum() >= 8      # a flat patch at full depth


def test_cylinder_and_capsule_side_closed_form():
    """Cylinder / capsule of radius r lying along the pad's y axis (object z -> world y) at
    centre height r - delta: a node at x inside the radius has penetration
    r - sqrt(x^2 + (r-delta)^2) and moves away from the axis in the x-z plane."""
    r, delta, hl = 6.0, 1.1, 20.0
    q = (math.sin(-math.pi / 4), 0.0, 0.0, math.cos(-math.pi / 4))  # object z -> world y
    for ot in (I.OBJ_CYLINDER, I.OBJ_CAPSULE):
        sc = _flat_scene(10, 10, obj=(ot, (r, hl, 0), (0.375, 0.0, r - delta, *q)))
        # exact stored pose: use the FP64 quaternion so that the axis lies exactly along y
        pose = np.array([0.375, 0.0, float(sc.obj_pose[2]), *q])
        out = O.forward(sc, _theta(), mode=O.MODE_LINEAR_ONLY, obj_pose=pose)
        h = float(sc.obj_pose[2])
        P = sc.types[0].pos.astype(np.float64)
        dist = np.sqrt((P[:, 0] - 0.375) ** 2 + h ** 2)
        d = np.maximum(0, r - dist)
        inside = d > 0
        np.testing.assert_array_equal(out["mask"].astype(bool), inside)
        np.testing.assert_allclose(out["pen"], d, atol=1e-12)
        a = inside
        np.testing.assert_allclose(out["disp"][a, 0], d[a] * (P[a, 0] - 0.375) / dist[a], atol=1e-12)
        np.testing.assert_allclose(out["disp"][a, 1], 0.0, atol=1e-12)
        np.testing.assert_allclose(out["disp"][a, 2], -d[a] * h / dist[a], atol=1e-12)


def _cylinder_cap_case(lib=None):
    """Upright cylinder (axis along the pad normal) pressed cap-down by delta: a node within
    the radius, at distance rho from the axis, is inside with penetration min(r - rho, delta).
    It leaves through the nearer of the side (radially, ties go radial) and the bottom cap
    (straight down by delta).  Returns the oracle's output and the closed form of the mask,
    the penetration and the active nodes' displacement."""
    r, hl, cx, cy = 3.5, 4.0, 0.3, -0.2
    sc = _flat_scene(12, 12, obj=(I.OBJ_CYLINDER, (r, hl, 0), (cx, cy, hl - 0.7, 0, 0, 0, 1)))
    out = O.forward(sc, _theta(), mode=O.MODE_LINEAR_ONLY, lib=lib)
    cx, cy = float(sc.obj_pose[0]), float(sc.obj_pose[1])  # stored float32 position
    delta = hl - float(sc.obj_pose[2])
    P = sc.types[0].pos.astype(np.float64)
    dxy = P[:, :2] - (cx, cy)
    rho = np.hypot(dxy[:, 0], dxy[:, 1])
    inside = rho < r
    pen = np.where(inside, np.minimum(r - rho, delta), 0.0)
    disp = np.zeros_like(P)
    radial = inside & (r - rho <= delta)
    cap = inside & ~radial
    disp[radial, :2] = (r - rho[radial])[:, None] * dxy[radial] / rho[radial][:, None]
    disp[cap, 2] = -delta
    return out, inside, pen, disp


def test_cylinder_cap_flat_patch():
    out, inside, pen, disp = _cylinder_cap_case()
    np.testing.assert_array_equal(out["mask"].astype(bool), inside)
    np.testing.assert_allclose(out["pen"], pen, atol=1e-12)
    np.testing.assert_allclose(out["disp"][inside], disp[inside], atol=1e-12)
    # both exits occur on this patch
    assert (np.abs(disp[inside, 2]) > 0).sum() >= 8 and (np.abs(disp[inside, 0]) > 0).sum() >= 8


def test_pad_pose_frame():
    """Outputs are in the pad frame: rotating and translating both pad and object by the same
    rigid motion leaves every output unchanged."""
    obj = (I.OBJ_CAPSULE, (4.0, 3.0, 0), (0.4, -0.3, 2.9, 0.2, 0.1, -0.3, 0.93))
    sc0 = _flat_scene(8, 8, obj=obj)
    rng = np.random.default_rng(3)
    qm = I.uniform_quat(rng)
    tm = rng.uniform(-20, 20, 3)
    op = np.array(obj[2], np.float64)
    op[3:] /= np.linalg.norm(op[3:])
    qo = I._qmul(qm, op[3:])
    to = I._qrot(qm, op[:3]) + tm
    sc1 = _flat_scene(8, 8, obj=(obj[0], obj[1], (*to, *qo)), pad_pose=(*tm, *qm))
    th = _theta()
    a = O.forward(sc0, th, obj_pose=np.concatenate([op]))
    b = O.forward(sc1, th, obj_pose=np.concatenate([to, qo]),
                  pad_pose=np.concatenate([tm, qm]))
    np.testing.assert_array_equal(a["mask"], b["mask"])
    np.testing.assert_allclose(a["disp"], b["disp"], atol=1e-9)


# ----------------------------------------------------------------- decay propagation (Eq. 1)


def test_single_node_dyadic_golden():
    """Eq. 1 with alpha = ln 2 on a 1 mm grid: a lone active node propagates exactly 2^-d of
    its displacement to a passive node at distance d (golden dyadic values)."""
    rows = cols = 11
    sc = _flat_scene(rows, cols)
    n = rows * cols
    j = 5 * cols + 5
    mask = np.zeros(n, np.uint8)
    mask[j] = 1
    uh = np.zeros((n, 3))
    uh[j] = (0.3, -0.2, -1.0)
    out = O.forward(sc, _theta(alpha=LN2), mode=O.MODE_LINEAR_ONLY,
                    mask_override=mask, uhat_override=uh)
    for dr, dc, frac in _load_golden():
        i = (5 + dr) * cols + (5 + dc)
        np.testing.assert_allclose(out["disp"][i], frac * uh[j], rtol=1e-13, atol=0)
    np.testing.assert_array_equal(out["disp"][j], uh[j])


def test_single_indenter_node_contact():
    """A sphere touching exactly one node (depth below the neighbour threshold) gives that
    node u = (0, 0, -delta) and its 4-neighbours exactly half of it when alpha = ln 2."""
    R, delta = 5.0, 0.0625        # dyadic; neighbours at 1 mm are outside: 1 + (R-d)^2 > R^2
    sc = _flat_scene(9, 9, obj=(I.OBJ_SPHERE, (R, 0, 0), (0.0, 0.0, R - delta, 0, 0, 0, 1)))
    out = O.forward(sc, _theta(alpha=LN2), mode=O.MODE_LINEAR_ONLY)
    j = 4 * 9 + 4
    assert out["mask"].sum() == 1 and out["mask"][j] == 1
    np.testing.assert_allclose(out["disp"][j], [0, 0, -delta], atol=1e-15)
    for i in (j - 1, j + 1, j - 9, j + 9):
        np.testing.assert_allclose(out["disp"][i], [0, 0, -delta / 2], rtol=1e-13, atol=0)
    np.testing.assert_allclose(out["disp"][j + 2], [0, 0, -delta / 4], rtol=1e-13, atol=0)


def test_linear_response_monotone_in_indentation():
    """Eq. 1 alone, a sphere (r = 5 mm) pressed into a flat pad deeper and deeper over the
    configured 0-2 mm range: the contact set only grows, every active node's u_hat points
    further down (|q| shrinks, so R - |q| grows faster than the normal tilts), and Eq. 1
    sums those with positive weights over a growing set.  So a node that stays active, or
    stays passive, moves strictly further down.  (A node that turns active takes its own
    small penetration in place of what its neighbours propagated to it, so no monotonicity
    holds across that switch.)"""
    R, cx, cy = 5.0, 0.25, -0.5
    prev_z, prev_mask, grew = None, None, 0
    for delta in np.linspace(0.125, 2.0, 16):
        sc = _flat_scene(16, 16, obj=(I.OBJ_SPHERE, (R, 0, 0), (cx, cy, R - delta, 0, 0, 0, 1)))
        out = O.forward(sc, _theta(), mode=O.MODE_LINEAR_ONLY)
        z, mask = out["disp"][:, 2], out["mask"].astype(bool)
        assert mask.any()
        if prev_z is not None:
            assert np.all(mask[prev_mask]), delta                    # contact set grows
            same = mask == prev_mask
            grew += int((~same).any())
            assert np.all(z[same] < prev_z[same]), (delta, np.max(z[same] - prev_z[same]))
        prev_z, prev_mask = z, mask
    assert grew >= 8 and prev_mask.sum() > 40     # the sweep crosses many contact sets


def test_monotone_decay_with_distance():
    """For alpha > 0 the propagated magnitude from one active node strictly decreases with
    distance."""
    sc = _flat_scene(9, 9, pitch=0.7)
    n = 81
    j = 40
    mask = np.zeros(n, np.uint8)
    mask[j] = 1
    uh = np.zeros((n, 3))
    uh[j] = (0.1, 0.4, -0.8)
    out = O.forward(sc, _theta(seed=2), mode=O.MODE_LINEAR_ONLY, mask_override=mask, uhat_override=uh)
    P = sc.types[0].pos.astype(np.float64)
    d = np.linalg.norm(P - P[j], axis=1)
    mag = np.linalg.norm(out["disp"], axis=1)
    o = [i for i in np.argsort(d, kind="stable") if i != j]
    for a, b in zip(o[:-1], o[1:]):
        if d[b] > d[a] + 1e-9:
            assert mag[b] < mag[a]


def test_linearity_and_superposition_bruteforce():
    """Brute force on 3x3 and 4x4 pads: for every activation pattern of one and two nodes,
    the linear-only field on passive nodes is the sum of the single-node fields; and the
    field is linear in U_hat for a fixed mask."""
    th = _theta(seed=5)
    rng = np.random.default_rng(0)
    for side in (3, 4):
        sc = _flat_scene(side, side, pitch=1.3)
        n = side * side
        uh = rng.normal(size=(n, 3))
        single = []
        for j in range(n):
            m = np.zeros(n, np.uint8)
            m[j] = 1
            single.append(O.forward(sc, th, O.MODE_LINEAR_ONLY, m, uh)["disp"])
        for j1 in range(n):
            for j2 in range(j1 + 1, n):
                m = np.zeros(n, np.uint8)
                m[[j1, j2]] = 1
                got = O.forward(sc, th, O.MODE_LINEAR_ONLY, m, uh)["disp"]
                pas = m == 0
                np.testing.assert_allclose(got[pas], single[j1][pas] + single[j2][pas],
                                           rtol=1e-12, atol=1e-14)
                np.testing.assert_array_equal(got[~pas], uh[~pas])
        m = (rng.random(n) < 0.4).astype(np.uint8)
        m[0] = 1
        u1, u2 = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
        f = lambda u: O.forward(sc, th, O.MODE_LINEAR_ONLY, m, u)["disp"]
        np.testing.assert_allclose(f(2.5 * u1 - 0.7 * u2), 2.5 * f(u1) - 0.7 * f(u2),
                                   rtol=1e-11, atol=1e-12)


def test_centred_indent_symmetry():
    """A sphere centred on a square flat pad: the contact set and the linear-only field are
    invariant under the pad's 90-degree rotation and mirror (displacements rotate along)."""
    side = 16
    sc = _flat_scene(side, side, obj=(I.OBJ_SPHERE, (9.0, 0, 0), (0, 0, 9.0 - 1.7, 0, 0, 0, 1)))
    out = O.forward(sc, _theta(seed=1), mode=O.MODE_LINEAR_ONLY)
    U = out["disp"].reshape(side, side, 3)      # [row(y), col(x), comp]
    M = out["mask"].reshape(side, side)
    # rotation by +90 deg about z: (x, y) -> (-y, x); node (r, c) -> (c, side-1-r)
    Ur = np.empty_like(U)
    for r in range(side):
        for c in range(side):
            u = U[r, c]
            Ur[c, side - 1 - r] = (-u[1], u[0], u[2])
    np.testing.assert_allclose(Ur, U, atol=1e-12)
    np.testing.assert_array_equal(M, np.rot90(M))
    Um = U[:, ::-1].copy()
    Um[..., 0] *= -1
    np.testing.assert_allclose(Um, U, atol=1e-12)
    assert M.sum() > 0


# ----------------------------------------------------------------- residual network + Eq. 4


def test_zero_weights_give_bias_residual():
    """With every network weight zero except the decoder output bias b, Phi_p = b on every
    passive node; active nodes keep u_hat."""
    th = _theta()
    sl = I.param_slices()
    th[1:] = 0.0
    a, n, _ = sl["bD2"]
    th[a:a + 3] = (0.01, -0.02, 0.03)
    sc = _flat_scene(8, 8, obj=(I.OBJ_SPHERE, (5, 0, 0), (0.25, 0.125, 5 - 1.0, 0, 0, 0, 1)))
    out = O.forward(sc, th, mode=O.MODE_RESIDUAL_ONLY)
    assert out["mask"].sum() > 0
    pas = out["mask"] == 0
    np.testing.assert_allclose(out["disp"][pas], [[0.01, -0.02, 0.03]] * int(pas.sum()), atol=1e-15)


def _small_hand(num_envs=3, seed=11):
    """Hand-like scene on small pads: curved 6x8 fingertips and a flat 8x10 palm."""
    rng = np.random.default_rng(seed)
    types = [I.curved_pad(6, 8, 1.0, 8.0), I.flat_pad(8, 10, 1.0)]
    pt = [0, 0, 0, 0, 0, 1]
    objs, poses = {}, []
    for e in range(num_envs):
        ot, dims = I.random_object(rng)
        q, t = I.uniform_quat(rng), rng.uniform(-20, 20, 3)
        objs[e] = (ot, dims, np.concatenate([t, q]))
        for s_ in range(6):
            poses.append(I.place_pad(rng, types[pt[s_]], ot, dims, t, q, rng.uniform(0, 2), 0.3))
    return I.custom_scene(types, np.tile(pt, num_envs), objs, poses, num_envs, 1)


@pytest.mark.parametrize("mode", [O.MODE_FULL, O.MODE_LINEAR_ONLY, O.MODE_RESIDUAL_ONLY])
def test_forward_matches_torch_restatement(mode):
    """The oracle equals an independent torch float64 restatement (library routines, SDF
    normal by autograd) on small curved and flat pads with every primitive type."""
    th = _theta(seed=4)
    scenes = [_small_hand()] + [I.grad_scene(ot) for ot in
                                (I.OBJ_SPHERE, I.OBJ_BOX, I.OBJ_CYLINDER, I.OBJ_CAPSULE)]
    for sc in scenes:
        out = O.forward(sc, th, mode=mode)
        assert out["mask"].sum() > 0
        ref, _ = TR.step(sc, th, mode=mode)
        np.testing.assert_allclose(out["disp"], ref.detach().numpy(), rtol=1e-10, atol=1e-11)


def test_pool_margin_matches_torch_features():
    """The max-pool margin report equals the top two channel features of the torch
    restatement (library linear / relu, torch.topk) on every pad: the nodes and the relative
    gap; a pad of one node has no second node and an infinite gap."""
    th = _theta(seed=4)
    P = TR.theta_tensors(th)[1]
    for sc in [_small_hand(), I.sphere_press_scene(3, seed=3),
               I.uneven_scene(2, seed=2), I.sphere_press_scene(1, seed=0, rows=1, cols=1)]:
        fw = O.forward(sc, th)
        r = O.pool_margin(sc, th)
        offs = sc.node_offsets
        for p in range(len(offs) - 1):
            t = sc.types[sc.pad_type[p]]
            a, b = offs[p], offs[p + 1]
            X = torch.tensor(np.concatenate(
                [t.pos, t.nrm, fw["disp"][a:b] * fw["mask"][a:b, None]], 1))
            f = torch.relu(torch.nn.functional.linear(
                torch.relu(torch.nn.functional.linear(X, P["WE1"], P["bE1"])), P["WE2"], P["bE2"]))
            if b - a == 1:
                assert np.all(r["top2"][p, :, 1] == -1) and np.all(np.isinf(r["gap"][p]))
                continue
            # stable descending order: equal values keep the lower node first
            order = np.argsort(-f.numpy(), axis=0, kind="stable")[:2].T
            np.testing.assert_array_equal(r["top2"][p], order)
            v = f.numpy()
            top, sec = v[order[:, 0], np.arange(64)], v[order[:, 1], np.arange(64)]
            want = np.where(top > 0, (top - sec) / np.where(top > 0, top, 1), np.inf)
            np.testing.assert_allclose(r["gap"][p], want, rtol=1e-9, atol=1e-15)


def test_decision_margin_matches_torch_restatement():
    """The oracle's report of the reverse mode's decision margins equals the same margins
    computed from an independent torch restatement of the network (library linear / relu /
    amax): per pad, the smallest relative ReLU margin at passive nodes (E1, E2, D1), at the
    active nodes holding a channel maximum (E1, E2), of the global layer, and the max-pool
    gaps with and without an active node among the top two."""
    th = _theta(seed=4)
    P = TR.theta_tensors(th)[1]
    lin = torch.nn.functional.linear
    for sc in [_small_hand(), I.sphere_press_scene(3, seed=3), I.uneven_scene(2, seed=2)]:
        fw = O.forward(sc, th)
        got = O.decision_margin(sc, th)
        offs = sc.node_offsets
        for p in range(len(offs) - 1):
            a, b = offs[p], offs[p + 1]
            m = fw["mask"][a:b] != 0
            if not m.any():
                assert np.all(np.isinf(got[p]))
                continue
            t = sc.types[sc.pad_type[p]]
            X = torch.tensor(np.concatenate([t.pos, t.nrm, fw["disp"][a:b] * m[:, None]], 1))
            a1 = lin(X, P["WE1"], P["bE1"])
            s1 = lin(X.abs(), P["WE1"].abs(), P["bE1"].abs())
            z1 = torch.relu(a1)
            a2 = lin(z1, P["WE2"], P["bE2"])
            s2 = lin(z1, P["WE2"].abs(), P["bE2"].abs())
            f = torch.relu(a2)
            g0, am = f.max(0)
            ag = lin(g0, P["WG1"], P["bG1"])
            sg = lin(g0, P["WG1"].abs(), P["bG1"].abs())
            g = torch.relu(ag)
            cat = torch.cat([f, g.expand(len(f), -1)], 1)
            a3 = lin(cat, P["WD1"], P["bD1"])
            s3 = lin(cat, P["WD1"].abs(), P["bD1"].abs())
            rm = lambda x, sc_: torch.where(sc_ > 0, x.abs() / sc_, torch.full_like(x, np.inf))
            holds = torch.zeros(len(f), dtype=torch.bool)
            holds[am] = True
            mt = torch.tensor(m)
            pas, amx = ~mt, mt & holds
            lo = lambda t_: float(t_.min()) if t_.numel() else np.inf
            want = [min(lo(rm(a1, s1)[pas]), lo(rm(a2, s2)[pas]), lo(rm(a3, s3)[pas])),
                    min(lo(rm(a1, s1)[amx]), lo(rm(a2, s2)[amx])), lo(rm(ag, sg))]
            order = np.argsort(-f.numpy(), axis=0, kind="stable")[:2].T
            v = f.numpy()
            gaps = {3: np.inf, 4: np.inf}
            for c in range(64):
                i1, i2 = order[c]
                if v[i1, c] > 0:
                    k = 3 if (m[i1] or m[i2]) else 4
                    gaps[k] = min(gaps[k], (v[i1, c] - v[i2, c]) / v[i1, c])
            want = [float(w) for w in want] + [gaps[3], gaps[4]]
            np.testing.assert_allclose(got[p], want, rtol=1e-9, atol=1e-15)


# ----------------------------------------------------------------- reverse mode


def _grad_case(ot, seed=0):
    sc = I.grad_scene(ot, seed=seed)
    th = _theta(seed=7)
    rng = np.random.default_rng(seed + 100)
    G = rng.normal(size=(sc.total_nodes, 3))
    return sc, th, G


@pytest.mark.parametrize("ot", [I.OBJ_SPHERE, I.OBJ_BOX, I.OBJ_CYLINDER, I.OBJ_CAPSULE])
def test_backward_matches_torch_autograd(ot):
    """Hand-written reverse mode == torch autograd of the independent restatement, for
    parameters and for object translation / rotation increments."""
    sc, th, G = _grad_case(ot)
    fw = O.forward(sc, th)
    bw = O.backward(sc, th, G)
    U, leaves = TR.step(sc, th, mask=fw["mask"], pose_leaves=True)
    L = (U * torch.tensor(G)).sum()
    gp, gt, gw = torch.autograd.grad(L, [leaves["params"], leaves["dt"], leaves["dw"]])
    np.testing.assert_allclose(bw["params"], gp.numpy(), rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(bw["obj_pose"][:, :3], gt.numpy(), rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(bw["obj_pose"][:, 3:], gw.numpy(), rtol=1e-9, atol=1e-10)


def test_backward_uhat_matches_autograd():
    """Gradient with respect to user-given active displacements (mask fixed)."""
    sc, th, G = _grad_case(I.OBJ_CAPSULE, seed=3)
    fw = O.forward(sc, th)
    uh = fw["disp"] * fw["mask"][:, None]
    bw = O.backward(sc, th, G, mask_override=fw["mask"], uhat_override=uh)
    U, leaves = TR.step(sc, th, mask=fw["mask"], uhat_override=uh)
    (gu,) = torch.autograd.grad((U * torch.tensor(G)).sum(), [leaves["uhat"]])
    gu = gu.numpy() * fw["mask"][:, None]
    np.testing.assert_allclose(bw["uhat"], gu, rtol=1e-9, atol=1e-11)
    # penetration gradient is the projection on the outward normal (u_hat = pen * n)
    bw2 = O.backward(sc, th, G)
    act = fw["mask"] > 0
    nrm = fw["disp"][act] / fw["pen"][act][:, None]
    np.testing.assert_allclose(bw2["pen"][act], (bw2["uhat"][act] * nrm).sum(1), rtol=1e-9, atol=1e-12)


def test_backward_central_differences():
    """FP64 central differences (step 1e-6) of the oracle forward agree with its reverse mode
    for alpha, sampled weights, and every pose component of a capsule contact."""
    sc, th, G = _grad_case(I.OBJ_CAPSULE, seed=1)
    bw = O.backward(sc, th, G)
    h = 1e-6
    L = lambda **kw: float((O.forward(sc, kw.pop("theta", th), **kw)["disp"] * G).sum())
    rng = np.random.default_rng(0)
    idx = [0] + list(rng.choice(np.arange(1, th.size), 40, replace=False))
    for k in idx:
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (L(theta=tp) - L(theta=tm)) / (2 * h)
        assert abs(fd - bw["params"][k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, bw["params"][k])
    op = sc.obj_pose.astype(np.float64)
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
        fd = (L(obj_pose=pose(1)) - L(obj_pose=pose(-1))) / (2 * h)
        assert abs(fd - bw["obj_pose"][0, a]) <= 1e-6 * max(1.0, abs(fd)), (a, fd, bw["obj_pose"][0])


_MUTANTS = {
    # wrong sign of the decay exponent in Eq. 1
    "exp_sign": ("double w = exp(-P->alpha * sqrt(dx * dx + dy * dy + dz * dz));",
                 "double w = exp(P->alpha * sqrt(dx * dx + dy * dy + dz * dz));"),
    # residual term of Eq. 4 dropped
    "drop_residual": ("U[3 * i + a] += acc;", "(void)acc;"),
    # transposed second encoder weight
    "transpose_W2": ("acc += P->W2[c * H + k] * z1[k];", "acc += P->W2[k * H + c] * z1[k];"),
    # displacement pushed into the object instead of onto its surface
    "uhat_sign": ("for (int a = 0; a < 3; ++a) u[a] *= -best;",
                  "for (int a = 0; a < 3; ++a) u[a] *= best;"),
    # wrong concat order of the global feature
    "concat_index": ("acc += P->Wd[c * 2 * H + H + k] * s->g[k];",
                     "acc += P->Wd[c * 2 * H + k] * s->g[k];"),
    # ReLU of the global MLP left out
    "global_relu": ("s->g[c] = relu(acc);", "s->g[c] = acc;"),
    # max-pool over the passive nodes only (the pool covers all n nodes)
    "pool_passive_only": ("if (fv > s->g0[c]) { s->g0[c] = fv; s->amax[c] = i; }",
                          "if (!s->act[i] && fv > s->g0[c]) { s->g0[c] = fv; s->amax[c] = i; }"),
    # squared distance in the decay of Eq. 1
    "squared_distance": ("double w = exp(-P->alpha * sqrt(dx * dx + dy * dy + dz * dz));",
                         "double w = exp(-P->alpha * (dx * dx + dy * dy + dz * dz));"),
    # propagation added to the active nodes too (Eq. 1 applies to passive nodes only)
    "propagate_into_active": ("      if (s->act[i]) continue;\n      const double* pi_",
                              "      const double* pi_"),
    # first encoder layer without its bias
    "e1_bias": ("double acc = P->b1[c];", "double acc = 0.0;"),
}


@pytest.mark.parametrize("name", sorted(_MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    """A copy of the oracle with one planted mistake fails the pins above: the golden Eq. 1
    values, the sphere closed form or the torch restatement."""
    src = open(os.path.join(os.path.dirname(O.__file__), "etac_oracle.c")).read()
    old, new = _MUTANTS[name]
    assert src.count(old) >= 1, name
    p = tmp_path / "mut.c"
    p.write_text(src.replace(old, new))
    lib = O.load_variant(str(p), str(tmp_path / "libmut.so"))
    failures = 0
    # golden single-node decay
    sc = _flat_scene(11, 11)
    mask = np.zeros(121, np.uint8)
    mask[60] = 1
    uh = np.zeros((121, 3))
    uh[60] = (0.3, -0.2, -1.0)
    out = O.forward(sc, _theta(alpha=LN2), O.MODE_LINEAR_ONLY, mask, uh, lib=lib)
    failures += not np.allclose(out["disp"][61], 0.5 * uh[60], rtol=1e-13, atol=0)
    # sphere closed form
    R, delta = 5.0, 1.3
    sc = _flat_scene(16, 16, obj=(I.OBJ_SPHERE, (R, 0, 0), (0.25, -0.4, R - delta, 0, 0, 0, 1)))
    out = O.forward(sc, _theta(), O.MODE_LINEAR_ONLY, lib=lib)
    a = out["mask"] > 0
    failures += not np.allclose(out["disp"][a, 2], -out["pen"][a] * (R - delta) / (R - out["pen"][a]))
    # torch restatement, full model
    sc = _small_hand(2)
    th = _theta(seed=4)
    out = O.forward(sc, th, lib=lib)
    ref, _ = TR.step(sc, th)
    failures += not np.allclose(out["disp"], ref.detach().numpy(), rtol=1e-8, atol=1e-9)
    assert failures > 0, f"planted mistake {name} passed every pin"


# Planted mistakes in the contact step and in the hand-written reverse mode.
_MUTANTS_REV = {
    # every box face pushes along +axis (outward normal sign lost on the negative faces)
    "box_face_sign": ("g[am] = q[am] >= 0 ? 1.0 : -1.0;", "g[am] = 1.0;"),
    # cylinder cap normal always +z: the bottom cap pushes nodes up into the object
    "cylinder_cap_sign": ("    g[2] = sz;\n    return dz;", "    g[2] = 1.0;\n    return dz;"),
    # cylinder side and cap distances swapped when choosing the exit
    "cylinder_exit_choice": ("if (dr >= dz) {", "if (dr <= dz) {"),
    # capsule segment not clamped to its end caps: the capsule becomes an infinite cylinder
    "capsule_clamp": ("double cz = q[2] < -h ? -h : (q[2] > h ? h : q[2]);",
                      "double cz = q[2];"),
    # d w / d alpha = -d w: sign dropped
    "alpha_grad_sign": ("gp[0] += -d * w * dot;", "gp[0] += d * w * dot;"),
    # ReLU gate of the decoder's hidden layer missing in the reverse pass
    "decoder_relu_gate": ("ga3[c] = s.a3[(size_t)i * H + c] > 0 ? gz : 0.0;", "ga3[c] = gz;"),
    # max-pool gradient routed to the first channel's argmax instead of each channel's
    "maxpool_route": ("gf[(size_t)s.amax[c] * H + c] += gg0[c];",
                      "gf[(size_t)s.amax[0] * H + c] += gg0[c];"),
    # curvature (Hessian) term of d(-phi grad phi)/dx with the wrong sign
    "hessian_sign": ("Av[a] += s.phi[i] * Hs[3 * a + b] * vo[b];",
                     "Av[a] -= s.phi[i] * Hs[3 * a + b] * vo[b];"),
    # rotation of the outward normal left out of the torque
    "torque_normal_term": ("gpo[3 + a] += c1[a] - s.phi[i] * c2[a];", "gpo[3 + a] += c1[a];"),
    # u_hat gradient taken through the normal's input column instead of u_hat's
    "uhat_input_column": ("acc += P.W1[c * NIN + 6 + a] * ga1[c];",
                          "acc += P.W1[c * NIN + 3 + a] * ga1[c];"),
    # penetration gradient projected on the object-frame normal, not the pad-frame one
    "pen_frame": ("grad_pen[gi] = npd[0] * gu[3 * i] + npd[1] * gu[3 * i + 1] + npd[2] * gu[3 * i + 2];",
                  "grad_pen[gi] = gobj[0] * gu[3 * i] + gobj[1] * gu[3 * i + 1] + gobj[2] * gu[3 * i + 2];"),
}


def _rev_pin_checks(lib):
    """The contact closed forms and the reverse-mode pins, run against `lib`; yields one
    bool per check (True = the check passed)."""
    # box pressed face-down (centre off the pad's origin so that both x faces are crossed)
    delta = 0.8
    sc = _flat_scene(12, 12, obj=(I.OBJ_BOX, (3.0, 2.0, 4.0), (0.25, 0.5, 4.0 - delta, 0, 0, 0, 1)))
    out = O.forward(sc, _theta(), mode=O.MODE_LINEAR_ONLY, lib=lib)
    P = sc.types[0].pos
    inside = (np.abs(P[:, 0] - 0.25) < 3.0) & (np.abs(P[:, 1] - 0.5) < 2.0)
    side = inside & (3.0 - np.abs(P[:, 0] - 0.25) < 4.0 - float(sc.obj_pose[2]))
    yield bool(np.array_equal(out["mask"].astype(bool), inside)) and bool(
        np.allclose(np.abs(out["disp"][side, 0]) * np.sign(P[side, 0] - 0.25),
                    out["disp"][side, 0], atol=1e-12))
    # capsule lying along y with its caps inside the pad: the caps round off the contact
    r, hl = 3.0, 2.0
    q = (math.sin(-math.pi / 4), 0.0, 0.0, math.cos(-math.pi / 4))
    sc = _flat_scene(14, 14, obj=(I.OBJ_CAPSULE, (r, hl, 0), (0.0, 0.0, r - 1.0, *q)))
    pose = np.array([0.0, 0.0, float(sc.obj_pose[2]), *q])
    out = O.forward(sc, _theta(), mode=O.MODE_LINEAR_ONLY, obj_pose=pose, lib=lib)
    Pd = sc.types[0].pos.astype(np.float64)
    cy = np.clip(Pd[:, 1], -hl, hl)
    dist = np.sqrt(Pd[:, 0] ** 2 + (Pd[:, 1] - cy) ** 2 + pose[2] ** 2)
    yield bool(np.allclose(out["pen"], np.maximum(0, r - dist), atol=1e-12))
    # upright cylinder pressed cap-down: side and cap exits
    out, inside, pen, disp = _cylinder_cap_case(lib)
    yield (bool(np.array_equal(out["mask"].astype(bool), inside))
           and bool(np.allclose(out["pen"], pen, atol=1e-12))
           and bool(np.allclose(out["disp"][inside], disp[inside], atol=1e-12)))
    # reverse mode vs torch autograd of the restatement, every primitive
    for ot in (I.OBJ_SPHERE, I.OBJ_BOX, I.OBJ_CYLINDER, I.OBJ_CAPSULE):
        sc, th, G = _grad_case(ot)
        fw = O.forward(sc, th, lib=lib)
        bw = O.backward(sc, th, G, lib=lib)
        U, leaves = TR.step(sc, th, mask=fw["mask"], pose_leaves=True)
        gp, gt, gw = torch.autograd.grad((U * torch.tensor(G)).sum(),
                                         [leaves["params"], leaves["dt"], leaves["dw"]])
        yield (np.allclose(bw["params"], gp.numpy(), rtol=1e-9, atol=1e-10)
               and np.allclose(bw["obj_pose"][:, :3], gt.numpy(), rtol=1e-9, atol=1e-10)
               and np.allclose(bw["obj_pose"][:, 3:], gw.numpy(), rtol=1e-9, atol=1e-10))
    # u_hat gradient (mask fixed) vs autograd; penetration gradient = its normal projection
    sc, th, G = _grad_case(I.OBJ_CAPSULE, seed=3)
    fw = O.forward(sc, th, lib=lib)
    uh = fw["disp"] * fw["mask"][:, None]
    bw = O.backward(sc, th, G, mask_override=fw["mask"], uhat_override=uh, lib=lib)
    U, leaves = TR.step(sc, th, mask=fw["mask"], uhat_override=uh)
    (gu,) = torch.autograd.grad((U * torch.tensor(G)).sum(), [leaves["uhat"]])
    yield bool(np.allclose(bw["uhat"], gu.numpy() * fw["mask"][:, None], rtol=1e-9, atol=1e-11))
    bw2 = O.backward(sc, th, G, lib=lib)
    act = fw["mask"] > 0
    nrm = fw["disp"][act] / fw["pen"][act][:, None]
    yield bool(np.allclose(bw2["pen"][act], (bw2["uhat"][act] * nrm).sum(1), rtol=1e-9, atol=1e-12))


def test_reverse_pin_checks_pass_on_the_oracle():
    assert all(_rev_pin_checks(None))


@pytest.mark.parametrize("name", sorted(_MUTANTS_REV))
def test_planted_reverse_or_contact_mistake_is_caught(name, tmp_path):
    """A copy of the oracle with one planted mistake in its contact step or its reverse mode
    fails at least one of the box, capsule-cap, cylinder-cap, autograd or
    penetration-projection pins."""
    src = open(os.path.join(os.path.dirname(O.__file__), "etac_oracle.c")).read()
    old, new = _MUTANTS_REV[name]
    assert src.count(old) == 1, name
    p = tmp_path / "mut.c"
    p.write_text(src.replace(old, new))
    lib = O.load_variant(str(p), str(tmp_path / "libmut.so"))
    assert not all(_rev_pin_checks(lib)), f"planted mistake {name} passed every pin"


def test_results_do_not_depend_on_the_thread_count():
    """The oracle parallelises over pads only: the forward and the per-node and pose gradients
    are bitwise the same on 1 and 4 threads; the parameter gradient, summed per thread before
    the threads are combined, agrees to FP64 rounding."""
    sc = I.uneven_scene(6, seed=3)
    th = _theta(seed=1)
    G = np.random.default_rng(0).normal(size=(sc.total_nodes, 3))
    try:
        f1, f4 = O.forward(sc, th, nthreads=1), O.forward(sc, th, nthreads=4)
        b1, b4 = O.backward(sc, th, G, nthreads=1), O.backward(sc, th, G, nthreads=4)
    finally:
        O.forward(_flat_scene(2, 2), th, nthreads=len(os.sched_getaffinity(0)))
    for k in f1:
        np.testing.assert_array_equal(f1[k], f4[k])
    for k in ("obj_pose", "uhat", "pen"):
        np.testing.assert_array_equal(b1[k], b4[k])
    np.testing.assert_allclose(b1["params"], b4["params"], rtol=1e-10,
                               atol=1e-12 * np.abs(b1["params"]).max())
