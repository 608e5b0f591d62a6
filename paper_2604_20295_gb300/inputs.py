"""Seeded synthetic inputs for the ETac tactile step (pads, rigid primitives, poses, params).

This module builds scenes only: grid node positions and normals of elastomer pads, rigid
primitive shapes, world poses that bring each pad into contact with its object, and the
propagation-model parameters.  It holds none of the method's arithmetic (no signed
distance, no penetration, no propagation, no network); both the CUDA path and the FP64
oracle consume the arrays it returns.  Every array is float32 / int32, laid out exactly as
the C ABI expects (see ``include/etac.h``).

Workloads follow the evaluation setting of the paper: primitive indenters pressed into a
flat and a curved elastomer (Sec. IV-A, depths of a few millimetres) and a many-environment
batch (Sec. IV-B, 4,096 environments).  The FEM indentation data of Sec. IV-A is not
available; these seeded scenes stand in for it.

Conventions: millimetres; quaternions are (x, y, z, w); a pose is t(3) followed by q(4);
nodes of a pad are row-major; pads are env-major, pad-minor.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# object type codes (the C ABI uses the same numbers; OBJ_MESH objects name a closed
# triangle mesh of the scene by index in obj_dims[0])
OBJ_NONE, OBJ_SPHERE, OBJ_BOX, OBJ_CYLINDER, OBJ_CAPSULE, OBJ_MESH = 0, 1, 2, 3, 4, 5

# parameter layout of the propagation model: alpha, then (W, b) for E1, E2, G1, D1, D2
HIDDEN = 64
LAYERS = (("E1", HIDDEN, 9), ("E2", HIDDEN, HIDDEN), ("G1", HIDDEN, HIDDEN),
          ("D1", HIDDEN, 2 * HIDDEN), ("D2", 3, HIDDEN))


def param_count() -> int:
    return 1 + sum(o * i + o for _, o, i in LAYERS)


def param_slices() -> dict:
    """Offsets of every tensor inside the flat parameter vector."""
    out, off = {"alpha": (0, 1, ())}, 1
    for name, o, i in LAYERS:
        out["W" + name] = (off, o * i, (o, i))
        off += o * i
        out["b" + name] = (off, o, (o,))
        off += o
    return out


def unpack_params(theta: np.ndarray) -> dict:
    return {k: np.asarray(theta[a:a + n]).reshape(s) if s else float(theta[a])
            for k, (a, n, s) in param_slices().items()}


def make_params(seed: int, d2_scale: float = 0.1) -> np.ndarray:
    """Model parameters from PCG64(seed).

    alpha ~ U[0.5, 1.5) 1/mm; each layer's W and b ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in));
    the output layer D2 is scaled by ``d2_scale`` so that the residual correction is of the
    same order as the propagated displacement.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = np.empty(param_count(), np.float64)
    theta[0] = 0.5 + rng.random()
    off = 1
    for name, o, i in LAYERS:
        bound = 1.0 / math.sqrt(i)
        scale = d2_scale if name == "D2" else 1.0
        theta[off:off + o * i] = scale * rng.uniform(-bound, bound, o * i)
        off += o * i
        theta[off:off + o] = scale * rng.uniform(-bound, bound, o)
        off += o
    return theta.astype(np.float32)



# parameter layout of the real-to-sim taxel regressor (appendix "Modeling Real Sensors"):
# a per-node encoder with a residual layer, an attention MLP of widths [256, 128, 1] with
# tanh, softmax pooling over the pad's nodes, and a head to the sensor's eight taxels; each
# layer is W (row-major, out x in) followed by b
REG_TAXELS = 8
REG_LAYERS = (("R1", 64, 9), ("R2", 128, 64), ("R3", 256, 128), ("R4", 256, 256),
              ("A1", 128, 256), ("A2", 1, 128), ("H1", 128, 256), ("H2", REG_TAXELS, 128))


def regressor_param_count() -> int:
    return sum(o * i + o for _, o, i in REG_LAYERS)


def regressor_param_slices() -> dict:
    out, off = {}, 0
    for name, o, i in REG_LAYERS:
        out["W" + name] = (off, o * i, (o, i))
        off += o * i
        out["b" + name] = (off, o, (o,))
        off += o
    return out


def make_regressor_params(seed: int) -> np.ndarray:
    """Regressor parameters from PCG64(seed): W, b ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = np.empty(regressor_param_count(), np.float64)
    off = 0
    for _, o, i in REG_LAYERS:
        bound = 1.0 / math.sqrt(i)
        theta[off:off + o * i + o] = rng.uniform(-bound, bound, o * i + o)
        off += o * i + o
    return theta.astype(np.float32)

# ----------------------------------------------------------------------------- pads


@dataclasses.dataclass
class PadType:
    """One elastomer pad geometry: a rows x cols grid of surface nodes (row-major)."""
    name: str
    rows: int
    cols: int
    pitch: float
    radius: float            # 0 for a flat pad; otherwise curvature radius of the arc (rows)
    pos: np.ndarray          # [n,3] float32, pad frame
    nrm: np.ndarray          # [n,3] float32, unit outward normals

    @property
    def n(self) -> int:
        return self.rows * self.cols


def flat_pad(rows: int, cols: int, pitch: float) -> PadType:
    """Flat grid centred at the origin in the z = 0 plane, normal +z."""
    r, c = np.meshgrid(np.arange(rows), np.arange(cols), indexing="ij")
    x = (c - (cols - 1) / 2.0) * pitch
    y = (r - (rows - 1) / 2.0) * pitch
    pos = np.stack([x, y, np.zeros_like(x)], -1).reshape(-1, 3)
    nrm = np.zeros_like(pos)
    nrm[:, 2] = 1.0
    return PadType(f"flat{rows}x{cols}@{pitch:g}", rows, cols, pitch, 0.0,
                   pos.astype(np.float32), nrm.astype(np.float32))


def curved_pad(rows: int, cols: int, pitch: float, radius: float) -> PadType:
    """Cylindrical fingertip pad: rows run around an arc of the given radius (arc pitch =
    ``pitch``), cols run along the cylinder axis (y).  The apex node region sits at z = 0
    with normal +z; p = (R sin t, y, R cos t - R), n = (sin t, 0, cos t)."""
    r, c = np.meshgrid(np.arange(rows), np.arange(cols), indexing="ij")
    theta = (r - (rows - 1) / 2.0) * (pitch / radius)
    y = (c - (cols - 1) / 2.0) * pitch
    pos = np.stack([radius * np.sin(theta), y, radius * np.cos(theta) - radius], -1)
    nrm = np.stack([np.sin(theta), np.zeros_like(theta), np.cos(theta)], -1)
    return PadType(f"curved{rows}x{cols}@{pitch:g}r{radius:g}", rows, cols, pitch, radius,
                   pos.reshape(-1, 3).astype(np.float32), nrm.reshape(-1, 3).astype(np.float32))


# ----------------------------------------------------------------------------- meshes


@dataclasses.dataclass
class Mesh:
    """A closed triangle mesh in its object frame (mm): triangles wind counter-clockwise
    seen from outside, so (v1 - v0) x (v2 - v0) points out of the solid."""
    name: str
    verts: np.ndarray        # [V,3] float32
    tris: np.ndarray         # [T,3] int32

    @property
    def soup(self) -> np.ndarray:
        """[T,3,3] float32 vertex coordinates of each triangle."""
        return np.ascontiguousarray(self.verts[self.tris], np.float32)


def box_mesh(hx: float, hy: float, hz: float) -> Mesh:
    """Axis-aligned box of half-extents (hx, hy, hz): 8 vertices, 2 triangles per face."""
    v = np.array([[sx * hx, sy * hy, sz * hz] for sz in (-1, 1) for sy in (-1, 1)
                  for sx in (-1, 1)], np.float32)           # index = 4*(z>0) + 2*(y>0) + (x>0)
    quads = [(0, 2, 3, 1), (4, 5, 7, 6),                    # -z, +z
             (0, 1, 5, 4), (2, 6, 7, 3),                    # -y, +y
             (0, 4, 6, 2), (1, 3, 7, 5)]                    # -x, +x
    t = [(a, b, c) for a, b, c, d in quads] + [(a, c, d) for a, b, c, d in quads]
    return Mesh(f"box{hx:g}x{hy:g}x{hz:g}", v, np.array(t, np.int32))


def icosphere(radius: float, subdiv: int) -> Mesh:
    """Icosahedron subdivided ``subdiv`` times (each triangle into four), vertices pushed
    onto the sphere of the given radius; 20 * 4**subdiv triangles."""
    g = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, g, 0), (1, g, 0), (-1, -g, 0), (1, -g, 0), (0, -1, g), (0, 1, g), (0, -1, -g),
         (0, 1, -g), (g, 0, -1), (g, 0, 1), (-g, 0, -1), (-g, 0, 1)]
    v = [np.array(p, np.float64) / np.linalg.norm(p) for p in v]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
         (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
         (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        mid = {}

        def m(a, b):
            k = (min(a, b), max(a, b))
            if k not in mid:
                p = v[a] + v[b]
                v.append(p / np.linalg.norm(p))
                mid[k] = len(v) - 1
            return mid[k]
        f = [t for a, b, c in f for t in ((a, m(a, b), m(c, a)), (b, m(b, c), m(a, b)),
                                           (c, m(c, a), m(b, c)), (m(a, b), m(b, c), m(c, a)))]
    return Mesh(f"icosphere{radius:g}s{subdiv}", (radius * np.array(v)).astype(np.float32),
                np.array(f, np.int32))


def torus_mesh(R: float, r: float, nu: int, nv: int) -> Mesh:
    """Torus about the z axis (tube radius r at distance R), nu x nv vertex grid; a solid
    with a hole, for inside/outside tests that a convex shape cannot make."""
    u = 2 * math.pi * np.arange(nu) / nu
    w = 2 * math.pi * np.arange(nv) / nv
    U, W = np.meshgrid(u, w, indexing="ij")
    v = np.stack([(R + r * np.cos(W)) * np.cos(U), (R + r * np.cos(W)) * np.sin(U),
                  r * np.sin(W)], -1).reshape(-1, 3)
    idx = lambda i, j: (i % nu) * nv + (j % nv)
    t = []
    for i in range(nu):
        for j in range(nv):
            a, b, c, d = idx(i, j), idx(i + 1, j), idx(i + 1, j + 1), idx(i, j + 1)
            t += [(a, b, c), (a, c, d)]
    return Mesh(f"torus{R:g}r{r:g}", v.astype(np.float32), np.array(t, np.int32))


def rock_mesh(seed: int, radius: float, subdiv: int = 3, amp: float = 0.2) -> Mesh:
    """Seeded star-shaped 'rock': an icosphere whose vertex radii are scaled by
    1 + amp * (a smooth random function of direction, |.| <= 1), so the surface stays
    closed and free of self-intersection for amp < 1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    base = icosphere(1.0, subdiv)
    d = base.verts.astype(np.float64)
    k = rng.normal(size=(6, 3))
    ph = rng.uniform(0, 2 * math.pi, 6)
    bump = np.mean(np.cos(d @ k.T * 1.5 + ph), axis=1)
    v = d * (radius * (1.0 + amp * bump))[:, None]
    return Mesh(f"rock{seed}r{radius:g}", v.astype(np.float32), base.tris.copy())


# ----------------------------------------------------------------------------- scenes


@dataclasses.dataclass
class Scene:
    """A batch of environments: pads (instances of pad types) and rigid primitives."""
    types: list              # list[PadType]
    num_envs: int
    pads_per_env: int
    max_objects: int
    pad_type: np.ndarray     # [E*P] int32
    obj_type: np.ndarray     # [E*K] int32 (OBJ_*)
    obj_dims: np.ndarray     # [E*K*3] float32
    obj_pose: np.ndarray     # [E*K*7] float32 world pose t(3) q(4, xyzw)
    pad_pose: np.ndarray     # [E*P*7] float32 world pose
    name: str = ""
    meshes: list = dataclasses.field(default_factory=list)   # list[Mesh], for OBJ_MESH

    @property
    def type_num_nodes(self) -> np.ndarray:
        return np.array([t.n for t in self.types], np.int32)

    @property
    def type_pos(self) -> np.ndarray:
        return np.ascontiguousarray(np.concatenate([t.pos for t in self.types]), np.float32)

    @property
    def type_nrm(self) -> np.ndarray:
        return np.ascontiguousarray(np.concatenate([t.nrm for t in self.types]), np.float32)

    @property
    def pad_nodes(self) -> np.ndarray:
        return self.type_num_nodes[self.pad_type]

    @property
    def node_offsets(self) -> np.ndarray:
        """CSR offsets of each pad instance's nodes in the flat node arrays, [E*P+1]."""
        return np.concatenate([[0], np.cumsum(self.pad_nodes, dtype=np.int64)])

    @property
    def total_nodes(self) -> int:
        return int(self.pad_nodes.sum())

    def subset(self, envs) -> "Scene":
        """The scene restricted to the given environment indices (same pad types)."""
        envs = np.asarray(envs, np.int64)
        P, K = self.pads_per_env, self.max_objects
        pi = (envs[:, None] * P + np.arange(P)[None]).reshape(-1)
        ki = (envs[:, None] * K + np.arange(K)[None]).reshape(-1)
        return Scene(self.types, len(envs), P, K, self.pad_type[pi].copy(),
                     self.obj_type[ki].copy(),
                     self.obj_dims.reshape(-1, 3)[ki].reshape(-1).copy(),
                     self.obj_pose.reshape(-1, 7)[ki].reshape(-1).copy(),
                     self.pad_pose.reshape(-1, 7)[pi].reshape(-1).copy(), self.name,
                     list(self.meshes))


# --- small rigid-motion helpers used only to place pads (scene construction)


def _qmul(a, b):
    ax, ay, az, aw = a
    bx, by, bz, bw = b
    return np.array([aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw,
                     aw * bw - ax * bx - ay * by - az * bz])


def _qrot(q, v):
    """Rotate vector v by unit quaternion q (q v q*)."""
    u, w = np.asarray(q[:3]), q[3]
    v = np.asarray(v, np.float64)
    return v + 2.0 * np.cross(u, np.cross(u, v) + w * v)


def _axis_angle(axis, ang):
    axis = np.asarray(axis, np.float64)
    axis = axis / np.linalg.norm(axis)
    return np.concatenate([axis * math.sin(ang / 2), [math.cos(ang / 2)]])


def _q_from_to(a, b):
    """Shortest-arc rotation taking unit vector a onto unit vector b."""
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    d = float(a @ b)
    if d < -1.0 + 1e-12:
        perp = np.cross(a, [1.0, 0, 0])
        if np.linalg.norm(perp) < 1e-6:
            perp = np.cross(a, [0, 1.0, 0])
        return _axis_angle(perp, math.pi)
    q = np.concatenate([np.cross(a, b), [1.0 + d]])
    return q / np.linalg.norm(q)


def uniform_quat(rng) -> np.ndarray:
    """Uniformly distributed rotation (Shoemake 1992, subgroup algorithm), (x, y, z, w)."""
    u1, u2, u3 = rng.random(3)
    a, b = math.sqrt(1 - u1), math.sqrt(u1)
    return np.array([a * math.sin(2 * math.pi * u2), a * math.cos(2 * math.pi * u2),
                     b * math.sin(2 * math.pi * u3), b * math.cos(2 * math.pi * u3)])


def _support(rng, otype: int, dims, mesh=None) -> tuple:
    """A surface point of the primitive (or mesh) and its outward unit normal, object frame,
    sampled with probability proportional to area."""
    if otype == OBJ_MESH:
        V = mesh.verts.astype(np.float64)[mesh.tris]
        n = np.cross(V[:, 1] - V[:, 0], V[:, 2] - V[:, 0])
        area = np.linalg.norm(n, axis=1)
        t = int(rng.choice(len(area), p=area / area.sum()))
        u, v = rng.random(2)
        if u + v > 1:
            u, v = 1 - u, 1 - v
        return V[t, 0] + u * (V[t, 1] - V[t, 0]) + v * (V[t, 2] - V[t, 0]), n[t] / area[t]
    if otype == OBJ_SPHERE:
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        return dims[0] * u, u
    if otype == OBJ_BOX:
        h = np.asarray(dims[:3], np.float64)
        areas = np.array([h[1] * h[2], h[0] * h[2], h[0] * h[1]])
        ax = int(rng.choice(3, p=areas / areas.sum()))
        sgn = 1.0 if rng.random() < 0.5 else -1.0
        s = rng.uniform(-h, h)
        s[ax] = sgn * h[ax]
        nrm = np.zeros(3)
        nrm[ax] = sgn
        return s, nrm
    r, hl = float(dims[0]), float(dims[1])
    if otype == OBJ_CYLINDER:
        side, cap = 2 * math.pi * r * 2 * hl, 2 * math.pi * r * r
        if rng.random() < side / (side + cap):
            t = rng.uniform(0, 2 * math.pi)
            nrm = np.array([math.cos(t), math.sin(t), 0.0])
            return np.array([r * nrm[0], r * nrm[1], rng.uniform(-hl, hl)]), nrm
        sgn = 1.0 if rng.random() < 0.5 else -1.0
        rad, t = r * math.sqrt(rng.random()), rng.uniform(0, 2 * math.pi)
        return np.array([rad * math.cos(t), rad * math.sin(t), sgn * hl]), np.array([0, 0, sgn])
    if otype == OBJ_CAPSULE:
        side, caps = 2 * math.pi * r * 2 * hl, 4 * math.pi * r * r
        if rng.random() < side / (side + caps):
            t = rng.uniform(0, 2 * math.pi)
            nrm = np.array([math.cos(t), math.sin(t), 0.0])
            return np.array([r * nrm[0], r * nrm[1], rng.uniform(-hl, hl)]), nrm
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        c = np.array([0.0, 0.0, hl if u[2] >= 0 else -hl])
        return c + r * u, u
    raise ValueError(otype)


def random_object(rng) -> tuple:
    """Primitive indenter of Sec. IV-A/B sizes: sphere r~U[10,30]; box edges ~U[20,60];
    cylinder / capsule r~U[10,30], half-length ~U[10,30] (mm)."""
    otype = int(rng.integers(1, 5))
    if otype == OBJ_SPHERE:
        dims = np.array([rng.uniform(10, 30), 0, 0])
    elif otype == OBJ_BOX:
        dims = rng.uniform(20, 60, 3) / 2.0
    else:
        dims = np.array([rng.uniform(10, 30), rng.uniform(10, 30), 0])
    return otype, dims


def place_pad(rng, ptype: PadType, otype: int, dims, obj_t, obj_q, depth: float,
              max_tilt: float, mesh=None) -> np.ndarray:
    """World pose of a pad whose randomly chosen node sits ``depth`` mm inside the object
    below a random surface point, pad normal opposing the surface normal, random spin about
    the normal and a random tilt (<= max_tilt rad) about an axis through that node."""
    s, ns = _support(rng, otype, dims, mesh)
    i0 = int(rng.integers(ptype.n))
    p0, n0 = ptype.pos[i0].astype(np.float64), ptype.nrm[i0].astype(np.float64)
    q_align = _q_from_to(n0, -ns)
    q_spin = _axis_angle(-ns, rng.uniform(0, 2 * math.pi))
    perp = np.cross(ns, rng.normal(size=3))
    q_tilt = _axis_angle(perp, rng.uniform(0, max_tilt))
    q_rel = _qmul(q_tilt, _qmul(q_spin, q_align))
    q_pad = _qmul(obj_q, q_rel)
    q_pad /= np.linalg.norm(q_pad)
    x_target = _qrot(obj_q, s - depth * ns) + obj_t
    t_pad = x_target - _qrot(q_pad, p0)
    return np.concatenate([t_pad, q_pad])


def _pack(types, E, P, K, pad_type, objs, pad_poses, name, meshes=()):
    obj_type = np.zeros(E * K, np.int32)
    obj_dims = np.zeros(E * K * 3, np.float32)
    obj_pose = np.zeros(E * K * 7, np.float32)
    obj_pose[6::7] = 1.0
    for idx, (ot, dims, pose) in objs.items():
        obj_type[idx] = ot
        obj_dims[idx * 3: idx * 3 + 3] = dims
        obj_pose[idx * 7: idx * 7 + 7] = pose
    return Scene(types, E, P, K, np.asarray(pad_type, np.int32), obj_type, obj_dims,
                 obj_pose, np.asarray(pad_poses, np.float32).reshape(-1), name, list(meshes))


def sphere_press_scene(steps: int, seed: int, rows: int = 16, cols: int = 16,
                       pitch: float = 1.0, radius: float = 5.0, max_depth: float = 2.0,
                       name: str = "flat16x16-sphere") -> Scene:
    """Flat pad at the origin (identity pose) pressed by a sphere of the given radius whose
    centre lies uniformly over the pad and whose depth is U[0, max_depth]; one step per
    environment (the model is quasi-static, so steps are independent problems)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pt = flat_pad(rows, cols, pitch)
    hx, hy = (cols - 1) / 2.0 * pitch, (rows - 1) / 2.0 * pitch
    objs, pads = {}, []
    for e in range(steps):
        cx, cy = rng.uniform(-hx, hx), rng.uniform(-hy, hy)
        depth = rng.uniform(0.0, max_depth)
        objs[e] = (OBJ_SPHERE, (radius, 0, 0), (cx, cy, radius - depth, 0, 0, 0, 1))
        pads.append([0, 0, 0, 0, 0, 0, 1])
    return _pack([pt], steps, 1, 1, np.zeros(steps, np.int32), objs, pads, name)


def hand_scene(num_envs: int, seed: int, max_depth: float = 3.0, max_tilt: float = 0.35,
               name: str = "hand-5tip-1palm") -> Scene:
    """Per environment: 5 curved fingertip pads (16x32, 1 mm pitch, radius 8 mm) and one
    flat palm pad (32x64, 1 mm pitch), all touching one seeded primitive (sphere, box,
    cylinder or capsule) with a uniformly random world pose near the hand."""
    rng = np.random.Generator(np.random.PCG64(seed))
    tip, palm = curved_pad(16, 32, 1.0, 8.0), flat_pad(32, 64, 1.0)
    types = [tip, palm]
    P = 6
    pad_type = np.tile(np.array([0, 0, 0, 0, 0, 1], np.int32), num_envs)
    objs, pads = {}, []
    for e in range(num_envs):
        ot, dims = random_object(rng)
        q = uniform_quat(rng)
        t = rng.uniform(-40.0, 40.0, 3)
        objs[e] = (ot, dims, np.concatenate([t, q]))
        for s in range(P):
            pads.append(place_pad(rng, types[pad_type[s]], ot, dims, t, q,
                                  rng.uniform(0.0, max_depth), max_tilt))
    return _pack(types, num_envs, P, 1, pad_type, objs, pads, name)


def uneven_scene(num_envs: int, seed: int, max_depth: float = 3.0, max_tilt: float = 0.35,
                 name: str = "uneven-6pad-1to3obj") -> Scene:
    """Per environment: 6 flat pads whose resolution is drawn from {8x8, 16x16, 32x32, 64x64}
    and pitch from {0.5, 1.0, 1.5, 2.0} mm (16 shared pad types), and 1-3 seeded primitives;
    each pad touches one of the env's primitives."""
    rng = np.random.Generator(np.random.PCG64(seed))
    res, pitches = (8, 16, 32, 64), (0.5, 1.0, 1.5, 2.0)
    types = [flat_pad(r, r, p) for r in res for p in pitches]
    P, K = 6, 3
    pad_type = np.empty(num_envs * P, np.int32)
    objs, pads = {}, []
    for e in range(num_envs):
        nobj = int(rng.integers(1, 4))
        placed = []
        for k in range(nobj):
            ot, dims = random_object(rng)
            q = uniform_quat(rng)
            t = rng.uniform(-40.0, 40.0, 3)
            objs[e * K + k] = (ot, dims, np.concatenate([t, q]))
            placed.append((ot, dims, t, q))
        for s in range(P):
            ti = int(rng.integers(len(res))) * len(pitches) + int(rng.integers(len(pitches)))
            pad_type[e * P + s] = ti
            ot, dims, t, q = placed[int(rng.integers(nobj))]
            pads.append(place_pad(rng, types[ti], ot, dims, t, q,
                                  rng.uniform(0.0, max_depth), max_tilt))
    return _pack(types, num_envs, P, K, pad_type, objs, pads, name)


def uneven_continuous_scene(num_envs: int, seed: int, max_depth: float = 3.0,
                            max_tilt: float = 0.35, name: str = "uneven-continuous-pitch") -> Scene:
    """``uneven_scene`` with a continuous pitch: every pad instance draws its resolution from
    {8x8, 16x16, 32x32, 64x64} and its own pitch from U[0.5, 2.0] mm, so every pad is its own
    type (no two share geometry: per-type Omega tables cannot be reused), with 1-3 seeded
    primitives per env, each pad touching one of them."""
    rng = np.random.Generator(np.random.PCG64(seed))
    res = (8, 16, 32, 64)
    P, K = 6, 3
    types, objs, pads = [], {}, []
    for e in range(num_envs):
        nobj = int(rng.integers(1, 4))
        placed = []
        for k in range(nobj):
            ot, dims = random_object(rng)
            q = uniform_quat(rng)
            t = rng.uniform(-40.0, 40.0, 3)
            objs[e * K + k] = (ot, dims, np.concatenate([t, q]))
            placed.append((ot, dims, t, q))
        for s in range(P):
            r = res[int(rng.integers(len(res)))]
            ty = flat_pad(r, r, float(rng.uniform(0.5, 2.0)))
            types.append(ty)
            ot, dims, t, q = placed[int(rng.integers(nobj))]
            pads.append(place_pad(rng, ty, ot, dims, t, q, rng.uniform(0.0, max_depth), max_tilt))
    pad_type = np.arange(num_envs * P, dtype=np.int32)
    return _pack(types, num_envs, P, K, pad_type, objs, pads, name)


def mesh_scene(num_envs: int, seed: int, num_meshes: int = 4, max_depth: float = 3.0,
               max_tilt: float = 0.35, name: str = "hand-mesh") -> Scene:
    """The hand layout of ``hand_scene`` (5 curved 16x32 fingertips + a flat 32x64 palm per
    env) pressed into seeded rock meshes (1,280 triangles, radius U[10, 30] mm) instead of
    primitives: ``num_meshes`` shared meshes, one per env chosen uniformly, uniform rotation,
    t ~ U[-40, 40]^3, pads placed as in ``hand_scene`` with depth U[0, max_depth]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    meshes = [rock_mesh(seed * 1000 + i, float(rng.uniform(10, 30)), subdiv=3)
              for i in range(num_meshes)]
    types = [curved_pad(16, 32, 1.0, 8.0), flat_pad(32, 64, 1.0)]
    P, K = 6, 1
    pad_type = np.tile(np.array([0, 0, 0, 0, 0, 1], np.int32), num_envs)
    objs, pads = {}, []
    for e in range(num_envs):
        mi = int(rng.integers(num_meshes))
        q = uniform_quat(rng)
        t = rng.uniform(-40, 40, 3)
        objs[e] = (OBJ_MESH, (mi, 0, 0), (*t, *q))
        for k in range(P):
            pads.append(place_pad(rng, types[pad_type[e * P + k]], OBJ_MESH, None, t, q,
                                  rng.uniform(0.0, max_depth), max_tilt, meshes[mi]))
    return _pack(types, num_envs, P, K, pad_type, objs, pads, name, meshes)


def custom_scene(types, pad_type, objects, pad_poses, num_envs: int, max_objects: int,
                 name: str = "custom", meshes=()) -> Scene:
    """Scene from explicit parts: ``objects`` maps a flat object slot (env * K + k) to
    (type, dims[3], pose[7]); ``pad_poses`` lists one world pose per pad instance; an
    OBJ_MESH object's dims[0] indexes ``meshes``."""
    P = len(pad_type) // num_envs
    return _pack(list(types), num_envs, P, max_objects, pad_type, objects, pad_poses, name,
                 meshes)


def grad_scene(otype: int = OBJ_CAPSULE, rows: int = 8, cols: int = 8, pitch: float = 1.0,
               depth: float = 1.2, seed: int = 0) -> Scene:
    """One environment, one flat 8x8 pad at the origin and one primitive pressed into it
    off-centre with a seeded tilt, so that every pose component carries a gradient.  The
    primitive's local z axis is laid roughly along the pad (capsule / cylinder side down)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pt = flat_pad(rows, cols, pitch)
    if otype == OBJ_SPHERE:
        dims, reach = (5.0, 0, 0), 5.0
    elif otype == OBJ_BOX:
        dims, reach = (2.0, 1.5, 6.0), 1.5
    else:
        dims, reach = (4.0, 3.0, 0), 4.0
    q = _qmul(_axis_angle(rng.normal(size=3), 0.15), _axis_angle([1.0, 0, 0], math.pi / 2))
    q = _qmul(_axis_angle([0, 0, 1.0], 0.4), q)
    off = rng.uniform(-0.6, 0.6, 2)
    objs = {0: (otype, dims, (off[0], off[1], reach - depth, *q))}
    return _pack([pt], 1, 1, 1, np.zeros(1, np.int32), objs, [[0, 0, 0, 0, 0, 0, 1]],
                 f"grad-flat{rows}x{cols}-obj{otype}")
