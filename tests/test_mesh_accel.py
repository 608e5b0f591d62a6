"""The host-side acceleration structure for triangle-mesh contact (etac_mesh_accel_build,
CPU only): mesh validation, the grid's cover of the bounding box, the cell classification
and candidate lists against the FP64 oracle's exact signed distance, and the pseudo-normals
against closed forms and against the oracle's winding-number sign."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2604_20295_gb300 import build as B
from paper_2604_20295_gb300 import etac as X
from paper_2604_20295_gb300 import inputs as I

MESHES = {
    "box": lambda: I.box_mesh(3.0, 2.0, 4.0),
    "rock": lambda: I.rock_mesh(3, 6.0, subdiv=2, amp=0.25),
    "torus": lambda: I.torus_mesh(10.0, 3.0, 48, 24),
    "icosphere": lambda: I.icosphere(15.0, 3),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    X.lib()


def _oracle_sdf(mesh, q):
    sc = I.custom_scene([I.flat_pad(2, 2, 1.0)], [0], {}, [(0, 0, 0, 0, 0, 0, 1)], 1, 1,
                        meshes=[mesh])
    return O.mesh_sdf(sc, 0, q)


def _cell_of(acc, q):
    """Cell index of each point (float32 arithmetic, as a query reads the grid), -1 outside."""
    rel = (q.astype(np.float32) - acc["origin"]) / np.float32(acc["cell"])
    ijk = np.floor(rel).astype(np.int64)
    dims = np.array(acc["dims"])
    ok = np.all((ijk >= 0) & (ijk < dims), axis=1)
    idx = (ijk[:, 2] * dims[1] + ijk[:, 1]) * dims[0] + ijk[:, 0]
    return np.where(ok, idx, -1)


def _samples(mesh, n, seed, pad=1.0):
    rng = np.random.default_rng(seed)
    V = mesh.verts.astype(np.float64)
    return rng.uniform(V.min(0) - pad, V.max(0) + pad, size=(n, 3))


@pytest.mark.parametrize("case", ["open", "flipped", "index", "degenerate", "grid", "few"])
def test_invalid_meshes_are_rejected(case):
    m = I.rock_mesh(1, 5.0, subdiv=1)
    v, t, grid = m.verts.copy(), m.tris.copy(), 0
    if case == "open":
        t = t[1:]
    elif case == "flipped":
        t[3] = t[3][::-1]
    elif case == "index":
        t[5, 1] = len(v)
    elif case == "degenerate":
        v = np.vstack([v, v[0], v[0] + 1.0])
        t = np.vstack([t, [[0, len(v) - 2, len(v) - 1]]])   # repeats a position: zero area
    elif case == "grid":
        grid = 513
    else:
        v, t = v[:3], t[:1]
    with pytest.raises(X.EtacError) as e:
        X.mesh_accel(v, t, grid)
    assert e.value.status == X.ERR_INVALID_ARG
    assert X.lib().etac_last_error(None)
    assert X.lib().etac_mesh_accel_build(None, None) == X.ERR_INVALID_ARG


def test_build_is_deterministic_and_covers_the_bounding_box():
    m = MESHES["rock"]()
    a, b = X.mesh_accel(m.verts, m.tris, 24), X.mesh_accel(m.verts, m.tris, 24)
    for k in ("cell_start", "cell_kind", "cand", "tri", "pseudo"):
        assert np.array_equal(a[k], b[k]), k
    V = m.verts
    np.testing.assert_array_equal(a["origin"], V.min(0))
    far = a["origin"].astype(np.float64) + np.array(a["dims"]) * a["cell"]
    assert np.all(far > V.max(0))
    assert max(a["dims"]) in (24, 25)
    assert np.all(_cell_of(a, V.astype(np.float64)) >= 0)        # every vertex is in a cell
    assert a["cell_start"][0] == 0 and np.all(np.diff(a["cell_start"]) >= 0)
    for c in range(0, len(a["cell_kind"]), 97):                  # ascending, in range
        s = a["cand"][a["cell_start"][c]:a["cell_start"][c + 1]]
        assert np.all(np.diff(s) > 0) and np.all((s >= 0) & (s < len(m.tris)))
    assert np.all(np.diff(a["cell_start"])[a["cell_kind"] == X.CELL_OUTSIDE] == 0)


@pytest.mark.parametrize("name", sorted(MESHES))
def test_cell_kinds_and_candidates_against_the_oracle(name):
    """OUTSIDE cells hold only outside points and INSIDE cells only inside points; in every
    other cell the listed triangles hold the nearest surface point (the distance over the
    listed triangles equals the distance over the whole mesh, bit for bit)."""
    m = MESHES[name]()
    acc = X.mesh_accel(m.verts, m.tris, 20)
    q = _samples(m, 500, seed=7)
    ref = _oracle_sdf(m, q)
    cell = _cell_of(acc, q)
    out_grid = cell < 0
    assert np.all(ref["phi"][out_grid] > 0)                      # outside the box: outside
    kind = np.where(out_grid, -1, acc["cell_kind"][np.maximum(cell, 0)].astype(np.int64))
    assert np.all(ref["phi"][kind == X.CELL_OUTSIDE] > 0)
    assert np.all(ref["phi"][kind == X.CELL_INSIDE] < 0)
    assert (kind == X.CELL_SURFACE).sum() > 20
    listed = np.nonzero((kind == X.CELL_INSIDE) | (kind == X.CELL_SURFACE))[0]
    for i in listed[:120]:
        c = cell[i]
        sub = acc["cand"][acc["cell_start"][c]:acc["cell_start"][c + 1]]
        part = I.Mesh("part", m.verts, m.tris[sub])
        d_sub = abs(_oracle_sdf(part, q[i:i + 1])["phi"][0])
        assert d_sub == abs(ref["phi"][i]), (name, i, d_sub, ref["phi"][i])


def _nearest_feature(V, tris, c, tol):
    """(triangle, feature) holding the surface point c: feature -1 face, 0..2 edges ab, bc,
    ca, 3..5 vertices a, b, c (the order of the pseudo-normal array)."""
    for t, (ia, ib, ic) in enumerate(tris):
        a, b, cc = V[ia], V[ib], V[ic]
        n = np.cross(b - a, cc - a)
        if abs(np.dot(c - a, n)) > tol * np.linalg.norm(n):
            continue
        M = np.stack([b - a, cc - a], 1)
        uv = np.linalg.lstsq(M, c - a, rcond=None)[0]
        w = np.array([1 - uv.sum(), uv[0], uv[1]])
        if np.any(w < -1e-7):
            continue
        for k in range(3):
            if w[k] > 1 - 1e-7:
                return t, 3 + k
        zero = np.abs(w) < 1e-7
        if zero.sum() == 1:
            k = int(np.nonzero(zero)[0][0])        # weight of the vertex opposite the edge
            return t, {0: 1, 1: 2, 2: 0}[k]
        return t, -1
    raise AssertionError("surface point on no triangle")


@pytest.mark.parametrize("name", ["rock", "torus", "box"])
def test_pseudo_normal_sign_matches_the_winding_number(name):
    """At the nearest feature F of a point q (found from the oracle's nearest point
    c = q - phi * grad), (q - c) . n_F < 0 exactly when the oracle's winding number puts q
    inside (the pseudo-normal theorem for closed meshes)."""
    m = MESHES[name]()
    acc = X.mesh_accel(m.verts, m.tris, 16)
    V = m.verts.astype(np.float64)
    q = _samples(m, 160, seed=3, pad=0.5)
    ref = _oracle_sdf(m, q)
    q, phi, g = q[np.abs(ref["phi"]) > 1e-3], ref["phi"][np.abs(ref["phi"]) > 1e-3], \
        ref["grad"][np.abs(ref["phi"]) > 1e-3]
    kinds = set()
    for qi, ph, gi in zip(q, phi, g):
        c = qi - ph * gi
        t, f = _nearest_feature(V, m.tris, c, 1e-7)
        n = acc["tri"][t, 3, :3] if f < 0 else acc["pseudo"][t, f, :3]
        kinds.add("face" if f < 0 else ("edge" if f < 3 else "vertex"))
        assert (np.dot(qi - c, n.astype(np.float64)) < 0) == (ph < 0), (name, qi, f)
    assert "face" in kinds and len(kinds) >= 2, kinds


def test_box_normals_closed_form():
    """Box: face normals are the axes; a box edge's pseudo-normal bisects its two faces; a
    corner's is (+-1, +-1, +-1)/sqrt(3); the diagonal splitting a face has that face's
    normal; the vertex records are the input vertices exactly."""
    m = MESHES["box"]()
    acc = X.mesh_accel(m.verts, m.tris, 8)
    np.testing.assert_array_equal(acc["tri"][:, :3, :3], m.verts[m.tris])
    assert np.all(acc["tri"][:, :, 3] == 0) and np.all(acc["pseudo"][:, :, 3] == 0)
    V = m.verts.astype(np.float64)
    h = np.array([3.0, 2.0, 4.0])
    for t, tri in enumerate(m.tris):
        fn = acc["tri"][t, 3, :3]
        axis = np.argmax(np.abs(fn))
        assert np.isclose(abs(fn[axis]), 1.0, atol=1e-7)
        assert np.isclose(np.sign(fn[axis]) * h[axis], V[tri[0], axis])
        for e in range(3):
            a, b = V[tri[e]], V[tri[(e + 1) % 3]]
            mid = 0.5 * (a + b)
            on = np.isclose(np.abs(mid), h)            # which box faces hold the edge
            exp = np.where(on, np.sign(mid), 0.0)
            np.testing.assert_allclose(acc["pseudo"][t, e, :3], exp / np.linalg.norm(exp),
                                       atol=1e-7)
        for k in range(3):
            np.testing.assert_allclose(acc["pseudo"][t, 3 + k, :3],
                                       np.sign(V[tri[k]]) / math.sqrt(3.0), atol=1e-7)


def test_varied_and_corrupted_meshes_seeded_fuzz():
    """Seeded variations of the generated meshes at many grid sizes build, and keep the
    structure's invariants (monotone cell starts, every candidate a valid triangle); the same
    meshes with a flipped triangle, a NaN vertex, an index moved out of range or triangles
    removed are rejected with ETAC_ERR_INVALID_ARG, never built."""
    rng = np.random.default_rng(11)
    gens = [lambda: I.box_mesh(*rng.uniform(0.5, 20, 3)),
            lambda: I.icosphere(float(rng.uniform(1, 30)), int(rng.integers(0, 3))),
            lambda: I.torus_mesh(float(rng.uniform(5, 15)), float(rng.uniform(1, 4)),
                                 int(rng.integers(6, 30)), int(rng.integers(4, 16))),
            lambda: I.rock_mesh(int(rng.integers(100)), float(rng.uniform(3, 20)),
                                subdiv=int(rng.integers(0, 3)), amp=float(rng.uniform(0, 0.5)))]
    for it in range(120):
        m = gens[it % len(gens)]()
        v, t = m.verts.copy(), m.tris.copy()
        corrupt = it % 5
        if corrupt == 1:
            k = rng.integers(len(t))
            t[k] = t[k][::-1]
        elif corrupt == 2:
            v[rng.integers(len(v)), rng.integers(3)] = np.nan
        elif corrupt == 3:
            t[rng.integers(len(t)), rng.integers(3)] = len(v) + int(rng.integers(0, 3))
        elif corrupt == 4:
            t = t[: len(t) - int(rng.integers(1, 3))]
        grid = int(rng.choice([0, 1, 2, 3, 7, 16, 33, 64]))
        if corrupt:
            with pytest.raises(X.EtacError) as e:
                X.mesh_accel(v, t, grid)
            assert e.value.status == X.ERR_INVALID_ARG, (it, corrupt)
            continue
        acc = X.mesh_accel(v, t, grid)
        cs = acc["cell_start"]
        assert cs[0] == 0 and cs[-1] == len(acc["cand"]) and np.all(np.diff(cs) >= 0), it
        assert len(cs) == np.prod(acc["dims"]) + 1
        assert acc["cand"].size == 0 or (acc["cand"].min() >= 0
                                         and acc["cand"].max() < acc["num_tris"]), it
        assert acc["num_tris"] == len(t)
