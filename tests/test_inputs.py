"""The seeded synthetic workloads have the shapes and contact statistics the workloads call
for (CPU only; contact measured with the FP64 oracle on a sample of environments)."""
import numpy as np
import pytest

import oracle as O
from paper_2604_20295_gb300 import inputs as I


def test_hand_scene_layout():
    """4,096 envs x (5 curved 16x32 fingertips + one flat 32x64 palm) = 18,874,368 nodes."""
    sc = I.hand_scene(4096, seed=2)
    assert sc.num_envs == 4096 and sc.pads_per_env == 6 and sc.max_objects == 1
    assert sc.total_nodes == 18874368
    assert [len(t.pos) for t in sc.types] == [512, 2048]
    tip = sc.types[0].pos
    # 16 nodes around an arc of radius 8 mm at 1 mm pitch (1/8 rad apart), 32 along the axis
    rho = np.hypot(tip[:, 0], tip[:, 2] + 8.0)
    np.testing.assert_allclose(rho, 8.0, atol=1e-5)
    assert np.ptp(tip[:, 1]) == 31.0
    palm = sc.types[1].pos
    assert np.all(palm[:, 2] == 0.0) and np.ptp(palm[:, 0]) == 63.0 and np.ptp(palm[:, 1]) == 31.0
    assert set(np.unique(sc.obj_type)) <= {I.OBJ_SPHERE, I.OBJ_BOX, I.OBJ_CYLINDER, I.OBJ_CAPSULE}


def test_hand_scene_is_seeded():
    a, b, c = I.hand_scene(8, seed=5), I.hand_scene(8, seed=5), I.hand_scene(8, seed=6)
    assert np.array_equal(a.obj_pose, b.obj_pose) and np.array_equal(a.pad_pose, b.pad_pose)
    assert not np.array_equal(a.obj_pose, c.obj_pose)


def test_hand_scene_contact_fraction():
    """Every pad touches its object; the contacted share of a pad's nodes averages about 0.2 and
    stays within 0-40 % (the workload's contact range) for most pads (the generator does not
    cap it: a large box face can cover a fingertip)."""
    sc = I.hand_scene(4096, seed=2).subset(np.arange(0, 4096, 128))   # 32 envs
    out = O.forward(sc, I.make_params(0))
    offs = sc.node_offsets
    frac = np.add.reduceat(out["mask"].astype(np.float64), offs[:-1]) / np.diff(offs)
    assert np.all(frac > 0)
    assert 0.1 < frac.mean() < 0.3
    assert np.mean(frac <= 0.4) > 0.85


def test_sphere_press_steps_follow_the_recipe():
    """Single 16x16 flat pad at 1 mm pitch; sphere r = 5 mm centred over the pad with
    penetration depth in [0, 2] mm (centre height 5 - depth)."""
    sc = I.sphere_press_scene(100, seed=0)
    assert sc.num_envs == 100 and sc.total_nodes == 100 * 256
    dims, pose = sc.obj_dims.reshape(-1, 3), sc.obj_pose.reshape(-1, 7)
    assert np.all(sc.obj_type == I.OBJ_SPHERE) and np.all(dims[:, 0] == 5.0)
    xy, z = pose[:, :2], pose[:, 2]
    assert np.all(np.abs(xy) <= 7.5) and np.all((z >= 3.0) & (z <= 5.0))


def test_uneven_scene_types():
    """6 flat pads per env with 8x8 .. 64x64 nodes at 0.5-2 mm pitch (16 shared types), 1-3
    primitives per env."""
    sc = I.uneven_scene(64, seed=5)
    sizes = sorted({len(t.pos) for t in sc.types})
    assert sizes == [64, 256, 1024, 4096] and len(sc.types) <= 16
    nobj = (sc.obj_type.reshape(sc.num_envs, sc.max_objects) != I.OBJ_NONE).sum(axis=1)
    assert nobj.min() >= 1 and nobj.max() <= 3


@pytest.mark.parametrize("make", [lambda: I.hand_scene(12, seed=2),
                                  lambda: I.uneven_scene(10, seed=4)])
def test_subset_matches_slices_of_the_full_scene(make):
    """A subset of environments (used to sample the oracle against a full-size GPU run) has
    the same nodes, in the same order, as the matching slices of the full scene: the oracle's
    output on the subset equals the full output at those environments' node ranges."""
    sc = make()
    th = I.make_params(0)
    envs = np.array([0, 3, 7, 9])
    full = O.forward(sc, th)
    sub = O.forward(sc.subset(envs), th)
    P = sc.pads_per_env
    offs = sc.node_offsets
    idx = np.concatenate([np.arange(offs[e * P], offs[e * P + P]) for e in envs])
    np.testing.assert_array_equal(sub["disp"], full["disp"][idx])
    np.testing.assert_array_equal(sub["mask"], full["mask"][idx])
    assert sc.subset(envs).total_nodes == len(idx)
