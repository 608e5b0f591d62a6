"""FP64 CPU oracle of the ETac tactile step -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It shares no code with the CUDA library: the C source in this folder
restates the method of ETac Sec. III-A (SDF contact, Eq. 1 decay propagation, the PointNet
residual network, Eq. 4) literally in double precision, and this module only marshals
numpy arrays into it through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "etac_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

MODE_FULL, MODE_LINEAR_ONLY, MODE_RESIDUAL_ONLY, MODE_PENETRATION_ONLY = 0, 1, 2, 3
OBJ_MESH = 5


def build(force: bool = False, src: str = _SRC, lib: str = _LIB) -> str:
    """Compile the oracle with gcc (-O2, OpenMP over pads) if missing or stale."""
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= os.path.getmtime(src)):
        return lib
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
    os.replace(tmp, lib)
    return lib


class _Scene(ctypes.Structure):
    _fields_ = [("num_types", ctypes.c_int), ("type_n", ctypes.c_void_p),
                ("type_pos", ctypes.c_void_p), ("type_nrm", ctypes.c_void_p),
                ("num_envs", ctypes.c_int), ("pads_per_env", ctypes.c_int),
                ("max_objects", ctypes.c_int), ("pad_type", ctypes.c_void_p),
                ("obj_type", ctypes.c_void_p), ("obj_dims", ctypes.c_void_p),
                ("obj_pose", ctypes.c_void_p), ("pad_pose", ctypes.c_void_p),
                ("num_meshes", ctypes.c_int), ("mesh_tri_off", ctypes.c_void_p),
                ("mesh_tri", ctypes.c_void_p)]


def _open(path):
    lib = ctypes.CDLL(path)
    lib.orc_param_count.restype = ctypes.c_size_t
    lib.orc_forward.restype = ctypes.c_int
    lib.orc_backward.restype = ctypes.c_int
    return lib


def _load(lib=None):
    global _lib
    if lib is not None:
        return lib
    if _lib is None:
        _lib = _open(build())
    return _lib


def load_variant(src: str, lib: str):
    """Compile and open another copy of the oracle source (used by tests that plant a
    mistake in a copy of the oracle to show that the pins catch it)."""
    return _open(build(force=True, src=src, lib=lib))


def param_count() -> int:
    return int(_load().orc_param_count())


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


class _Marshalled:
    """Keeps the double-precision copies of a scene alive while the C call runs."""

    def __init__(self, scene, obj_pose=None, pad_pose=None):
        f64 = lambda a: np.ascontiguousarray(a, np.float64)
        i32 = lambda a: np.ascontiguousarray(a, np.int32)
        self.arrs = dict(
            type_n=i32(scene.type_num_nodes), type_pos=f64(scene.type_pos),
            type_nrm=f64(scene.type_nrm), pad_type=i32(scene.pad_type),
            obj_type=i32(scene.obj_type), obj_dims=f64(scene.obj_dims),
            obj_pose=f64(scene.obj_pose if obj_pose is None else obj_pose),
            pad_pose=f64(scene.pad_pose if pad_pose is None else pad_pose))
        meshes = list(getattr(scene, "meshes", []))
        a = self.arrs
        a["mesh_tri_off"] = i32(np.concatenate([[0], np.cumsum([len(m.tris) for m in meshes],
                                                               dtype=np.int64)]))
        a["mesh_tri"] = (f64(np.concatenate([m.soup for m in meshes])) if meshes
                         else np.zeros((1, 3, 3)))
        self.s = _Scene(len(scene.types), _ptr(a["type_n"]), _ptr(a["type_pos"]),
                        _ptr(a["type_nrm"]), scene.num_envs, scene.pads_per_env,
                        scene.max_objects, _ptr(a["pad_type"]), _ptr(a["obj_type"]),
                        _ptr(a["obj_dims"]), _ptr(a["obj_pose"]), _ptr(a["pad_pose"]),
                        len(meshes), _ptr(a["mesh_tri_off"]), _ptr(a["mesh_tri"]))


def forward(scene, theta, mode: int = MODE_FULL, mask_override=None, uhat_override=None,
            obj_pose=None, pad_pose=None, nthreads: int = 0, lib=None) -> dict:
    """Displacement of every node (pad frame, mm) plus contact outputs, all FP64.

    ``obj_pose`` / ``pad_pose`` (float64) replace the scene's float32 poses, which lets a
    finite-difference check perturb them by less than a float32 ulp.  ``mask_override``
    (uint8 [N]) and ``uhat_override`` (float64 [N,3]) replace the contact result."""
    lib = _load(lib)
    m = _Marshalled(scene, obj_pose, pad_pose)
    N = scene.total_nodes
    th = np.ascontiguousarray(theta, np.float64)
    mo = None if mask_override is None else np.ascontiguousarray(mask_override, np.uint8)
    uo = None if uhat_override is None else np.ascontiguousarray(uhat_override, np.float64)
    out = dict(disp=np.zeros((N, 3)), mask=np.zeros(N, np.uint8), phi=np.zeros(N),
               pen=np.zeros(N), active_count=np.zeros(scene.num_envs * scene.pads_per_env,
                                                      np.int32))
    rc = lib.orc_forward(ctypes.byref(m.s), _ptr(th), int(mode), _ptr(mo), _ptr(uo),
                         _ptr(out["disp"]), _ptr(out["mask"]), _ptr(out["phi"]),
                         _ptr(out["pen"]), _ptr(out["active_count"]), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"orc_forward failed ({rc})")
    return out


def pool_margin(scene, theta, mask_override=None, uhat_override=None, nthreads: int = 0,
                lib=None) -> dict:
    """Margin of every pad's max-pool choice per channel (FP64): top2 [pads, 64, 2] = the
    nodes holding the largest and second-largest feature (ties to the lower index, -1 when
    none), gap [pads, 64] = (f_top1 - f_top2) / f_top1 (inf when f_top1 <= 0)."""
    lib = _load(lib)
    m = _Marshalled(scene)
    th = np.ascontiguousarray(theta, np.float64)
    mo = None if mask_override is None else np.ascontiguousarray(mask_override, np.uint8)
    uo = None if uhat_override is None else np.ascontiguousarray(uhat_override, np.float64)
    npads = scene.num_envs * scene.pads_per_env
    out = dict(top2=np.zeros((npads, 64, 2), np.int32), gap=np.zeros((npads, 64)))
    lib.orc_pool_margin.restype = ctypes.c_int
    rc = lib.orc_pool_margin(ctypes.byref(m.s), _ptr(th), _ptr(mo), _ptr(uo), _ptr(out["top2"]),
                             _ptr(out["gap"]), ctypes.c_int(nthreads))
    if rc != 0:
        raise RuntimeError(f"orc_pool_margin failed ({rc})")
    return out


MARGIN_KINDS = ("relu_passive", "relu_active_max", "relu_global", "pool_active", "pool_passive")


def decision_margin(scene, theta, mask_override=None, uhat_override=None, nthreads: int = 0,
                    lib=None) -> np.ndarray:
    """[pads, 5] smallest relative margin of each kind of discrete decision the reverse mode
    of the residual network takes on each pad (see MARGIN_KINDS and orc_decision_margin):
    ReLU margins |a| / (|b| + sum |w x|), max-pool gaps (f1 - f2) / f1; inf where none."""
    lib = _load(lib)
    m = _Marshalled(scene)
    th = np.ascontiguousarray(theta, np.float64)
    mo = None if mask_override is None else np.ascontiguousarray(mask_override, np.uint8)
    uo = None if uhat_override is None else np.ascontiguousarray(uhat_override, np.float64)
    out = np.zeros((scene.num_envs * scene.pads_per_env, 5))
    lib.orc_decision_margin.restype = ctypes.c_int
    rc = lib.orc_decision_margin(ctypes.byref(m.s), _ptr(th), _ptr(mo), _ptr(uo), _ptr(out),
                                 ctypes.c_int(nthreads))
    if rc != 0:
        raise RuntimeError(f"orc_decision_margin failed ({rc})")
    return out


def regressor_param_count(lib=None) -> int:
    lib = _load(lib)
    lib.orc_regressor_param_count.restype = ctypes.c_size_t
    return int(lib.orc_regressor_param_count())


def regress(scene, disp, rparams, nthreads: int = 0, lib=None) -> dict:
    """Real-to-sim taxel regressor on every pad: taxels [pads, 8] from the displacement field
    disp [N, 3] (pad frame) and the pads' geometry; attn [N] = each node's softmax weight
    within its pad (FP64)."""
    lib = _load(lib)
    m = _Marshalled(scene)
    N = scene.total_nodes
    d = np.ascontiguousarray(disp, np.float64).reshape(N, 3)
    rp = np.ascontiguousarray(rparams, np.float64)
    if rp.size != regressor_param_count(lib):
        raise ValueError(f"regressor parameters: {rp.size} values, want {regressor_param_count(lib)}")
    npads = scene.num_envs * scene.pads_per_env
    out = dict(taxels=np.zeros((npads, 8)), attn=np.zeros(N))
    rc = lib.orc_regress(ctypes.byref(m.s), _ptr(d), _ptr(rp), _ptr(out["taxels"]),
                         _ptr(out["attn"]), ctypes.c_int(nthreads))
    if rc != 0:
        raise RuntimeError(f"orc_regress failed ({rc})")
    return out


def mesh_sdf(scene, mesh: int, q, lib=None) -> dict:
    """Signed distance (negative inside), outward gradient and Hessian of one of the scene's
    meshes at object-frame points q [n,3] (FP64)."""
    lib = _load(lib)
    m = _Marshalled(scene)
    q = np.ascontiguousarray(q, np.float64).reshape(-1, 3)
    n = len(q)
    out = dict(phi=np.zeros(n), grad=np.zeros((n, 3)), hess=np.zeros((n, 3, 3)))
    rc = lib.orc_mesh_sdf(ctypes.byref(m.s), ctypes.c_int(mesh), ctypes.c_long(n), _ptr(q),
                          _ptr(out["phi"]), _ptr(out["grad"]), _ptr(out["hess"]))
    if rc != 0:
        raise ValueError(f"orc_mesh_sdf failed ({rc})")
    return out


def backward(scene, theta, grad_disp, mode: int = MODE_FULL, mask_override=None,
             uhat_override=None, obj_pose=None, pad_pose=None, nthreads: int = 0,
             lib=None) -> dict:
    """Hand-written reverse mode: gradients of sum(grad_disp * disp) (all FP64)."""
    lib = _load(lib)
    m = _Marshalled(scene, obj_pose, pad_pose)
    N = scene.total_nodes
    th = np.ascontiguousarray(theta, np.float64)
    gd = np.ascontiguousarray(grad_disp, np.float64).reshape(N, 3)
    mo = None if mask_override is None else np.ascontiguousarray(mask_override, np.uint8)
    uo = None if uhat_override is None else np.ascontiguousarray(uhat_override, np.float64)
    out = dict(obj_pose=np.zeros((scene.num_envs * scene.max_objects, 6)),
               uhat=np.zeros((N, 3)), pen=np.zeros(N), params=np.zeros(th.size))
    rc = lib.orc_backward(ctypes.byref(m.s), _ptr(th), int(mode), _ptr(mo), _ptr(uo),
                          _ptr(gd), _ptr(out["obj_pose"]), _ptr(out["uhat"]), _ptr(out["pen"]),
                          _ptr(out["params"]), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"orc_backward failed ({rc})")
    return out
