"""Pins of the oracle's triangle-mesh contact (object meshes of Sec. III-A "Overview"): the
signed distance to a closed mesh, its gradient and Hessian, and the contact step and
reverse mode driven by it.  Each check rests on something other than the oracle's own
formula: closed-form shapes, dense sampling of the surface, ray casting, the inscribed-
polytope bound of a tessellated sphere, and finite differences.  CPU only."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2604_20295_gb300 import inputs as I

MESHES = {
    "box": lambda: I.box_mesh(3.0, 2.0, 4.0),
    "icosphere": lambda: I.icosphere(5.0, 2),
    "torus": lambda: I.torus_mesh(10.0, 3.0, 48, 24),
    "rock": lambda: I.rock_mesh(3, 6.0, subdiv=2, amp=0.25),
}


def _mesh_scene(mesh, pose=(0, 0, 0, 0, 0, 0, 1), pad=None):
    pad = pad or I.flat_pad(4, 4, 1.0)
    return I.custom_scene([pad], [0], {0: (I.OBJ_MESH, (0, 0, 0), pose)},
                          [(0, 0, 0, 0, 0, 0, 1)], 1, 1, meshes=[mesh])


def _query(mesh, q, lib=None):
    return O.mesh_sdf(_mesh_scene(mesh), 0, q, lib=lib)


def _edge_counts(m):
    e = {}
    for a, b, c in m.tris:
        for u, v in ((a, b), (b, c), (c, a)):
            e[(int(u), int(v))] = e.get((int(u), int(v)), 0) + 1
    return e


@pytest.mark.parametrize("name", sorted(MESHES))
def test_generated_meshes_are_closed_and_outward(name):
    """Every directed edge appears once and its reverse once (closed, consistently wound);
    the signed volume is positive (counter-clockwise seen from outside)."""
    m = MESHES[name]()
    e = _edge_counts(m)
    assert all(v == 1 for v in e.values())
    assert all((b, a) in e for a, b in e)
    V = m.verts.astype(np.float64)
    T = m.tris
    vol = np.einsum("ij,ij->i", V[T[:, 0]], np.cross(V[T[:, 1]], V[T[:, 2]])).sum() / 6
    assert vol > 0


def _sampled_distance(m, q, k):
    """Unsigned distance from each q to a dense barycentric sampling of every triangle, and
    the sampling bound (longest edge / k): the exact distance d satisfies
    d <= sampled <= d + bound."""
    V = m.verts.astype(np.float64)[m.tris]                    # [T,3,3]
    i, j = np.meshgrid(np.arange(k + 1), np.arange(k + 1), indexing="ij")
    keep = (i + j) <= k
    u, v = (i[keep] / k), (j[keep] / k)
    S = (V[:, 0][:, None] + u[None, :, None] * (V[:, 1] - V[:, 0])[:, None] +
         v[None, :, None] * (V[:, 2] - V[:, 0])[:, None]).reshape(-1, 3)
    d = np.full(len(q), np.inf)
    for c in range(0, len(S), 20000):
        blk = S[c:c + 20000]
        d = np.minimum(d, np.sqrt(((q[:, None, :] - blk[None]) ** 2).sum(-1)).min(1))
    edges = np.linalg.norm(V - np.roll(V, 1, axis=1), axis=2).max()
    return d, edges / k


@pytest.mark.parametrize("name", ["rock", "torus", "box"])
def test_distance_matches_dense_surface_sampling(name):
    m = MESHES[name]()
    if name == "rock":
        m = I.rock_mesh(3, 6.0, subdiv=1, amp=0.25)
    rng = np.random.default_rng(4)
    V = m.verts.astype(np.float64)
    lo, hi = V.min(0) - 2.0, V.max(0) + 2.0
    q = rng.uniform(lo, hi, size=(150, 3))
    got = np.abs(_query(m, q)["phi"])
    ds, bound = _sampled_distance(m, q, 40)
    assert np.all(got <= ds + 1e-12)
    assert np.all(ds - got <= bound + 1e-12)


def _ray_hit(m, d):
    """Distance along unit direction d from the origin to the surface of a mesh that is
    star-shaped about the origin (Moller-Trumbore against every triangle)."""
    V = m.verts.astype(np.float64)[m.tris]
    e1, e2 = V[:, 1] - V[:, 0], V[:, 2] - V[:, 0]
    pv = np.cross(d, e2)
    det = (e1 * pv).sum(1)
    tv = -V[:, 0]
    u = (tv * pv).sum(1) / det
    qv = np.cross(tv, e1)
    v = (qv @ d) / det
    t = (e2 * qv).sum(1) / det
    ok = (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 0)
    return t[ok].min()


def test_sign_by_ray_casting_and_closed_forms():
    """Inside iff phi < 0: for the box by its half-extents, for the star-shaped rock by a ray
    from its centre, for the torus by the ideal torus where the point is clear of the
    tessellation error."""
    rng = np.random.default_rng(9)
    box = MESHES["box"]()
    q = rng.uniform(-5, 5, size=(400, 3))
    inside = np.all(np.abs(q) < (3.0, 2.0, 4.0), axis=1)
    assert np.array_equal(_query(box, q)["phi"] < 0, inside)

    rock = MESHES["rock"]()
    dirs = rng.normal(size=(120, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    hit = np.array([_ray_hit(rock, d) for d in dirs])
    radii = hit * rng.uniform(0.3, 1.7, size=len(hit))
    keep = np.abs(radii - hit) > 1e-6
    q = (dirs * radii[:, None])[keep]
    assert np.array_equal(_query(rock, q)["phi"] < 0, (radii < hit)[keep])

    tor = MESHES["torus"]()
    q = rng.uniform((-15, -15, -5), (15, 15, 5), size=(600, 3))
    ideal = np.sqrt((np.hypot(q[:, 0], q[:, 1]) - 10.0) ** 2 + q[:, 2] ** 2) - 3.0
    # chordal deviation of the tessellation: the sagittas of the two angular steps
    dev = 13.0 * (1 - math.cos(math.pi / 48)) + 3.0 * (1 - math.cos(math.pi / 24))
    clear = np.abs(ideal) > 4 * dev
    res = _query(tor, q[clear])["phi"]
    assert np.array_equal(res < 0, ideal[clear] < 0)
    assert np.all(np.abs(res - ideal[clear]) < 1.2 * dev)
    c = _query(tor, np.array([[0.0, 0.0, 0.0], [10.0, 0.0, 0.0]]))["phi"]
    assert c[0] > 0 and c[1] < 0                                 # the hole / the tube


def test_face_point_gradient_is_the_face_normal():
    """Above a box face at height t: phi = t, gradient = the face normal, Hessian zero;
    below it (inside, nearest that face): phi = -t, same gradient.  The first two points
    project onto the diagonal that splits the +z face into two triangles, where the face
    (not the shared edge) holds the nearest point."""
    box = MESHES["box"]()
    q = np.array([[0.3, 0.2, 4.0 + 0.7], [0.3, 0.2, 4.0 - 0.5], [3.0 + 0.4, -0.1, 0.5]])
    r = _query(box, q)
    np.testing.assert_allclose(r["phi"], [0.7, -0.5, 0.4], atol=1e-12)
    np.testing.assert_allclose(r["grad"], [[0, 0, 1], [0, 0, 1], [1, 0, 0]], atol=1e-12)
    assert np.all(r["hess"] == 0)


def test_edge_and_vertex_distances_closed_form():
    """Outside a box beyond an edge the distance is to that edge line, beyond a corner to
    the corner; the Hessian is the projector off the gradient (and off the edge) / d."""
    box = MESHES["box"]()
    q = np.array([[3.0 + 0.6, 2.0 + 0.8, 1.0],      # beyond the (+x, +y) edge, along z
                  [3.0 + 0.3, 2.0 + 0.4, 4.0 + 1.2]])  # beyond the (+, +, +) corner
    r = _query(box, q)
    np.testing.assert_allclose(r["phi"], [1.0, 1.3], atol=1e-12)
    np.testing.assert_allclose(r["grad"][0], [0.6, 0.8, 0.0], atol=1e-12)
    np.testing.assert_allclose(r["grad"][1], np.array([0.3, 0.4, 1.2]) / 1.3, atol=1e-12)
    g0 = np.array([0.6, 0.8, 0.0])
    np.testing.assert_allclose(r["hess"][0], (np.eye(3) - np.outer(g0, g0) -
                                              np.diag([0, 0, 1.0])) / 1.0, atol=1e-12)
    g1 = r["grad"][1]
    np.testing.assert_allclose(r["hess"][1], (np.eye(3) - np.outer(g1, g1)) / 1.3, atol=1e-12)


@pytest.mark.parametrize("name", ["box", "rock", "torus"])
def test_gradient_and_hessian_match_finite_differences(name):
    m = MESHES[name]()
    rng = np.random.default_rng(12)
    V = m.verts.astype(np.float64)
    q = rng.uniform(V.min(0) - 1.5, V.max(0) + 1.5, size=(80, 3))
    q = q[np.abs(_query(m, q)["phi"]) > 0.05]                  # Hessian ~ 1/distance
    r = _query(m, q)
    h = 1e-5
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        rp, rm = _query(m, q + e), _query(m, q - e)
        fd_g = (rp["phi"] - rm["phi"]) / (2 * h)
        fd_H = (rp["grad"] - rm["grad"]) / (2 * h)
        np.testing.assert_allclose(r["grad"][:, a], fd_g, atol=1e-7)
        tol = 1e-4 / np.abs(r["phi"])[:, None]
        assert np.all(np.abs(r["hess"][:, :, a] - fd_H) <= tol), (name, a)
    feats = {int(np.count_nonzero(np.abs(np.linalg.eigvalsh(H)) > 1e-9)) for H in r["hess"]}
    print(name, "Hessian ranks seen", sorted(feats))
    assert np.all(np.abs(np.linalg.norm(r["grad"], axis=1) - 1.0) < 1e-12)


def test_box_mesh_contact_equals_the_box_closed_form():
    """A box mesh pressed face-down reproduces the analytic box-face press exactly: the
    footprint is the active set, depth delta on the flat patch, sideways push where a side
    face is nearer."""
    delta = 0.8
    pose = (0.25, 0.5, 4.0 - delta, 0, 0, 0, 1)
    sc = _mesh_scene(MESHES["box"](), pose, I.flat_pad(12, 12, 1.0))
    out = O.forward(sc, I.make_params(0).astype(np.float64), mode=O.MODE_LINEAR_ONLY)
    delta = 4.0 - float(sc.obj_pose[2])
    P = sc.types[0].pos
    inside = (np.abs(P[:, 0] - 0.25) < 3.0) & (np.abs(P[:, 1] - 0.5) < 2.0)
    np.testing.assert_array_equal(out["mask"].astype(bool), inside)
    dx = 3.0 - np.abs(P[:, 0] - 0.25)
    dy = 2.0 - np.abs(P[:, 1] - 0.5)
    for i in np.nonzero(inside)[0]:
        mn = min(dx[i], dy[i], delta)
        if dx[i] == mn:
            exp = (mn * np.sign(P[i, 0] - 0.25), 0, 0)
        elif dy[i] == mn:
            exp = (0, mn * np.sign(P[i, 1] - 0.5), 0)
        else:
            exp = (0, 0, -delta)
        assert abs(out["pen"][i] - mn) < 1e-12
        np.testing.assert_allclose(out["disp"][i], exp, atol=1e-12)


@pytest.mark.parametrize("subdiv", [2, 3])
def test_icosphere_press_within_the_inscribed_polytope_bound(subdiv):
    """An icosphere inscribed in the sphere of radius R: its active set is a subset of the
    sphere's and, on it, 0 <= pen_sphere - pen_mesh <= R - r_in (r_in = the smallest distance
    from the centre to a face plane)."""
    R = 5.0
    m = I.icosphere(R, subdiv)
    V = m.verts.astype(np.float64)[m.tris]
    n = np.cross(V[:, 1] - V[:, 0], V[:, 2] - V[:, 0])
    r_in = np.min(np.abs((n * V[:, 0]).sum(1)) / np.linalg.norm(n, axis=1))
    pose = (0.25, -0.4, R - 1.3, 0, 0, 0, 1)
    th = I.make_params(0).astype(np.float64)
    pad = I.flat_pad(16, 16, 1.0)
    fm = O.forward(_mesh_scene(m, pose, pad), th, mode=O.MODE_LINEAR_ONLY)
    fs = O.forward(I.custom_scene([pad], [0], {0: (I.OBJ_SPHERE, (R, 0, 0), pose)},
                                  [(0, 0, 0, 0, 0, 0, 1)], 1, 1), th, mode=O.MODE_LINEAR_ONLY)
    am, asp = fm["mask"] > 0, fs["mask"] > 0
    assert am.sum() > 10 and np.all(asp[am])
    gap = fs["pen"][am] - fm["pen"][am]
    assert np.all(gap >= -1e-12) and np.all(gap <= (R - r_in) + 1e-12)


def test_mesh_contact_backward_central_differences():
    """Reverse mode through a mesh contact (a tilted rock, nodes inside concave regions):
    object pose and parameter gradients equal FP64 central differences of the forward."""
    rock = I.rock_mesh(5, 6.0, subdiv=2, amp=0.3)
    q = I._qmul(I._axis_angle([1.0, 0.3, 0.0], 0.35), I._axis_angle([0, 0, 1.0], 0.7))
    q = q / np.linalg.norm(q)
    lowest = min(I._qrot(q, v)[2] for v in rock.verts.astype(np.float64))
    pose = np.array([0.3, -0.2, -lowest - 1.1, *q])
    sc = _mesh_scene(rock, pose, I.flat_pad(8, 8, 1.0))
    pose = np.concatenate([sc.obj_pose[:3].astype(np.float64), q])
    th = I.make_params(7).astype(np.float64)
    fw = O.forward(sc, th, obj_pose=pose)
    assert fw["mask"].sum() >= 4
    G = np.random.default_rng(2).normal(size=(sc.total_nodes, 3))
    bw = O.backward(sc, th, G, obj_pose=pose)
    L = lambda **kw: float((O.forward(sc, kw.pop("theta", th), **kw)["disp"] * G).sum())
    h = 1e-6
    for a in range(6):
        def moved(sgn):
            o = pose.copy()
            if a < 3:
                o[a] += sgn * h
            else:
                ax = np.zeros(3)
                ax[a - 3] = 1.0
                o[3:] = I._qmul(I._axis_angle(ax, sgn * h), o[3:])
            return o
        fd = (L(obj_pose=moved(1)) - L(obj_pose=moved(-1))) / (2 * h)
        assert abs(fd - bw["obj_pose"][0, a]) <= 1e-6 * max(1.0, abs(fd)), (a, fd, bw["obj_pose"][0])
    for k in (0, 5, 700, 17000):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (L(theta=tp, obj_pose=pose) - L(theta=tm, obj_pose=pose)) / (2 * h)
        assert abs(fd - bw["params"][k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, bw["params"][k])


_MESH_MUTANTS = {
    # solid angle missing its factor 2: the winding number inside is 1/2, never above it
    "solid_angle_half": ("return 2.0 * atan2(num, den);", "return atan2(num, den);"),
    # one barycentric weight left out of the inside-the-face test
    "barycentric_check": ("if (wa >= -1e-12 && wb >= -1e-12 && wc >= -1e-12) {",
                          "if (wa >= -1e-12 && wb >= -1e-12) {"),
    # segment parameter not clamped at the far end
    "segment_clamp": ("t = t < 0 ? 0 : (t > 1 ? 1 : t);", "t = t < 0 ? 0 : t;"),
    # edge Hessian without the projector off the edge direction
    "edge_hessian": ("(bf == 1 ? be[a] * be[b] : 0.0)", "0.0"),
    # gradient pointing inward
    "gradient_sign": ("g[a] = sgn * (q[a] - bc[a]) / d;", "g[a] = (q[a] - bc[a]) / d;"),
}


def _mesh_pin_checks(lib):
    """The sign, sampling, closed-form and finite-difference pins above, against `lib`."""
    rng = np.random.default_rng(21)
    box = MESHES["box"]()
    q = rng.uniform(-5, 5, size=(200, 3))
    r = _query(box, q, lib)
    yield bool(np.array_equal(r["phi"] < 0, np.all(np.abs(q) < (3.0, 2.0, 4.0), axis=1)))
    rock = I.rock_mesh(3, 6.0, subdiv=1, amp=0.25)
    V = rock.verts.astype(np.float64)
    q = rng.uniform(V.min(0) - 2.0, V.max(0) + 2.0, size=(60, 3))
    got = np.abs(_query(rock, q, lib)["phi"])
    ds, bound = _sampled_distance(rock, q, 30)
    yield bool(np.all(got <= ds + 1e-12) and np.all(ds - got <= bound + 1e-12))
    qe = np.array([[3.6, 2.8, 1.0], [3.3, 2.4, 5.2]])
    r = _query(box, qe, lib)
    g0 = np.array([0.6, 0.8, 0.0])
    yield bool(np.allclose(r["hess"][0], np.eye(3) - np.outer(g0, g0) - np.diag([0, 0, 1.0]),
                           atol=1e-12))
    qf = np.array([[0.3, 0.2, 3.5], [3.4, -0.1, 0.5]])
    yield bool(np.allclose(_query(box, qf, lib)["grad"], [[0, 0, 1], [1, 0, 0]], atol=1e-12))


def test_mesh_pin_checks_pass_on_the_oracle():
    assert all(_mesh_pin_checks(None))


@pytest.mark.parametrize("name", sorted(_MESH_MUTANTS))
def test_planted_mesh_mistake_is_caught(name, tmp_path):
    src = open(os.path.join(os.path.dirname(O.__file__), "etac_oracle.c")).read()
    old, new = _MESH_MUTANTS[name]
    assert src.count(old) == 1, name
    p = tmp_path / "mut.c"
    p.write_text(src.replace(old, new))
    lib = O.load_variant(str(p), str(tmp_path / "libmut.so"))
    assert not all(_mesh_pin_checks(lib)), f"planted mistake {name} passed every mesh pin"
