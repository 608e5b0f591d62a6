"""GPU signed-distance query against closed triangle meshes (etac_mesh_sdf_query) against the
FP64 oracle's exact mesh SDF: sign exact away from the surface, distance within the FP32
bound, gradient, outside cells, non-finite points, a large ragged batch, repeatability."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_20295_gb300 import build as B
from paper_2604_20295_gb300 import etac as X
from paper_2604_20295_gb300 import inputs as I

pytestmark = pytest.mark.gpu

MESHES = {
    "box": lambda: I.box_mesh(3.0, 2.0, 4.0),
    "rock": lambda: I.rock_mesh(3, 6.0, subdiv=2, amp=0.25),
    "torus": lambda: I.torus_mesh(10.0, 3.0, 48, 24),
    "icosphere": lambda: I.icosphere(15.0, 3),
}

# FP32 distance error: the point, vertex and nearest-point coordinates (|x| <= 25 mm) carry
# a relative rounding of 2^-24 through about ten dependent operations, ~2e-5 mm; signs are
# compared only where the oracle's |phi| exceeds 5x that.
DIST_TOL = 2e-5
SIGN_BAND = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    X.lib()


def _oracle(mesh, q):
    sc = I.custom_scene([I.flat_pad(2, 2, 1.0)], [0], {}, [(0, 0, 0, 0, 0, 0, 1)], 1, 1,
                        meshes=[mesh])
    return O.mesh_sdf(sc, 0, q)


def _gpu(mesh, q, grid=0):
    s = X.MeshSDF(mesh.verts, mesh.tris, grid)
    try:
        qt = torch.as_tensor(np.ascontiguousarray(q, np.float32)).cuda()
        phi, grad = s.query(qt)
        torch.cuda.synchronize()
        return phi.cpu().numpy().astype(np.float64), grad.cpu().numpy().astype(np.float64)
    finally:
        s.close()


@pytest.mark.parametrize("name", sorted(MESHES))
def test_query_matches_the_oracle(name):
    m = MESHES[name]()
    rng = np.random.default_rng(5)
    V = m.verts.astype(np.float64)
    q = rng.uniform(V.min(0) - 1.0, V.max(0) + 1.0, size=(4000, 3)).astype(np.float32)
    q64 = q.astype(np.float64)
    ref = _oracle(m, q64)
    phi, grad = _gpu(m, q)
    inf = np.isinf(phi)
    assert np.all(phi[inf] > 0) and np.all(ref["phi"][inf] > 0)      # skipped: outside only
    assert np.all(grad[inf] == 0)
    fin = ~inf
    assert fin.sum() > 500
    clear = fin & (np.abs(ref["phi"]) > SIGN_BAND)
    np.testing.assert_array_equal(phi[clear] < 0, ref["phi"][clear] < 0)
    np.testing.assert_allclose(phi[fin], ref["phi"][fin], atol=DIST_TOL, rtol=0)
    far = fin & (np.abs(ref["phi"]) > 1e-2)
    np.testing.assert_allclose(grad[far], ref["grad"][far], atol=5e-3, rtol=0)


def test_edge_cases_empty_nonfinite_and_vertices():
    m = MESHES["rock"]()
    s = X.MeshSDF(m.verts, m.tris)
    try:
        X.etac_mesh_sdf_query(s.handle, 0, 0, 0)                     # n = 0: nothing to do
        q = np.array([[np.nan, 0, 0], [np.inf, 1, 1], [0, 0, 0], [1e6, 0, 0]], np.float32)
        q = np.vstack([q, m.verts[:8]])                               # vertices: phi = 0
        phi, grad = s.query(torch.as_tensor(q).cuda())
        phi = phi.cpu().numpy()
        assert np.isinf(phi[0]) and np.isinf(phi[1]) and np.isinf(phi[3])
        ref = _oracle(m, q[2:3].astype(np.float64))["phi"][0]
        assert phi[2] < 0 and abs(phi[2] - ref) < DIST_TOL             # the centre: inside
        assert np.all(np.abs(phi[4:]) < DIST_TOL)
        with pytest.raises(X.EtacError):
            X.etac_mesh_sdf_query(s.handle, -1, 0, 0)
        with pytest.raises(X.EtacError):
            X.etac_mesh_sdf_query(s.handle, 4, 0, 0)
    finally:
        s.close()


def test_large_ragged_batch_and_repeatability():
    """2,000,003 points (not a multiple of the block size, more than one grid-stride pass):
    a sample against the oracle, and two runs bit-identical."""
    m = I.icosphere(15.0, 3)
    rng = np.random.default_rng(8)
    n = 2_000_003
    q = rng.uniform(-16.5, 16.5, size=(n, 3)).astype(np.float32)
    s = X.MeshSDF(m.verts, m.tris)
    try:
        qt = torch.as_tensor(q).cuda()
        p1, g1 = s.query(qt)
        p2, g2 = s.query(qt)
        torch.cuda.synchronize()
        assert torch.equal(p1, p2) and torch.equal(g1, g2)
        phi = p1.cpu().numpy().astype(np.float64)
    finally:
        s.close()
    idx = np.concatenate([rng.choice(n, 3000, replace=False), np.arange(n - 40, n)])
    ref = _oracle(m, q[idx].astype(np.float64))["phi"]
    got = phi[idx]
    fin = ~np.isinf(got)
    assert np.all(ref[~fin] > 0)
    np.testing.assert_allclose(got[fin], ref[fin], atol=DIST_TOL, rtol=0)
