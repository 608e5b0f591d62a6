"""ctypes binding of libetac (``include/etac.h``).

The ``etac_*`` functions carry the C names and only marshal arguments: integers are device
or host addresses, structures mirror the C ones, every GPU step runs in the library's CUDA
kernels.  ``TactileSim`` is a convenience owner of a context plus the torch tensors that
hold its inputs and outputs (torch is used for device memory and streams only).  There is no
CPU fallback: if the library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

ETAC_OK = 0
ERR_INVALID_ARG = 1
STATUS_NAMES = {0: "ETAC_OK", 1: "ETAC_ERR_INVALID_ARG", 2: "ETAC_ERR_STATE", 3: "ETAC_ERR_CUDA",
                4: "ETAC_ERR_OOM", 5: "ETAC_ERR_TIMEOUT", 6: "ETAC_ERR_NONFINITE",
                7: "ETAC_ERR_UNSUPPORTED", 8: "ETAC_ERR_BOUNDS"}
MODE_FULL, MODE_LINEAR_ONLY, MODE_RESIDUAL_ONLY, MODE_PENETRATION_ONLY = 0, 1, 2, 3
PREC_FP32, PREC_BF16 = 0, 1
OMEGA_AUTO, OMEGA_TABLE, OMEGA_ON_THE_FLY = 0, 1, 2
ALGO_PLAIN, ALGO_BATCHED = 0, 1
HIDDEN = 64

EXPORTS = ("etac_param_count", "etac_total_nodes", "etac_create_pads", "etac_set_model",
           "etac_step_forward", "etac_step_backward", "etac_last_step", "etac_poll_status",
           "etac_forward_f64",
           "etac_last_error", "etac_destroy", "etac_step_forward_noalloc",
           "etac_enable_timing", "etac_kernel_times", "etac_pose_grad_to_quat",
           "etac_autotune", "etac_set_tuning", "etac_test_withhold_load", "etac_mesh_accel_build",
           "etac_mesh_accel_get_view", "etac_mesh_accel_destroy", "etac_mesh_gpu_create",
           "etac_mesh_sdf_query", "etac_mesh_gpu_destroy", "etac_regress", "etac_set_meshes")
TAXELS = 8
REGRESSOR_PARAMS = 174729
CELL_OUTSIDE, CELL_INSIDE, CELL_SURFACE = 0, 1, 2
TUNE_MAX = 8

_vp = ctypes.c_void_p


class etac_pads_desc(ctypes.Structure):
    _fields_ = [("num_types", ctypes.c_int32), ("type_num_nodes", _vp), ("type_pos", _vp),
                ("type_nrm", _vp), ("num_envs", ctypes.c_int32), ("pads_per_env", ctypes.c_int32),
                ("pad_type", _vp), ("max_objects", ctypes.c_int32)]


class etac_model_desc(ctypes.Structure):
    _fields_ = [("hidden", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("algo", ctypes.c_int32)]


class etac_step_in(ctypes.Structure):
    _fields_ = [("obj_type", _vp), ("obj_dims", _vp), ("obj_pose", _vp), ("pad_pose", _vp),
                ("active_disp_in", _vp), ("active_mask_in", _vp)]


class etac_tuning(ctypes.Structure):
    _fields_ = [("gemm_inst_per_tile", ctypes.c_int32), ("gemm_tile_order", ctypes.c_int32),
                ("bwd_node_range", ctypes.c_int32), ("num_fwd", ctypes.c_int32),
                ("fwd_cand", (ctypes.c_int32 * 2) * 8), ("fwd_ms", ctypes.c_float * 8),
                ("num_bwd", ctypes.c_int32), ("bwd_cand", ctypes.c_int32 * 8),
                ("bwd_ms", ctypes.c_float * 8), ("front_ctas_per_sm", ctypes.c_int32),
                ("num_front", ctypes.c_int32), ("front_cand", ctypes.c_int32 * 8),
                ("front_ms", ctypes.c_float * 8), ("omega_source", ctypes.c_int32),
                ("omega_ms", ctypes.c_float * 2)]


class etac_step_out(ctypes.Structure):
    _fields_ = [("disp", _vp), ("active_mask", _vp), ("penetration", _vp),
                ("active_count", _vp)]


class etac_noalloc_pads(ctypes.Structure):
    _fields_ = [("num_types", ctypes.c_int32), ("type_num_nodes", _vp), ("type_off", _vp),
                ("type_pos", _vp), ("type_nrm", _vp), ("num_envs", ctypes.c_int32),
                ("pads_per_env", ctypes.c_int32), ("max_objects", ctypes.c_int32),
                ("pad_type", _vp), ("pad_off", _vp)]


class etac_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int32),
                ("total_ms", ctypes.c_float)]


class etac_mesh_desc(ctypes.Structure):
    _fields_ = [("num_verts", ctypes.c_int32), ("num_tris", ctypes.c_int32),
                ("verts", _vp), ("tris", _vp), ("grid", ctypes.c_int32)]


class etac_mesh_accel_view(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_float * 3), ("cell", ctypes.c_float),
                ("dims", ctypes.c_int32 * 3), ("num_tris", ctypes.c_int32),
                ("num_cand", ctypes.c_int64), ("cell_start", _vp), ("cell_kind", _vp),
                ("cand", _vp), ("tri", _vp), ("pseudo", _vp)]


class EtacError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib():
    """The loaded libetac.so (raises if it has not been built).  ``ETAC_LIBRARY`` may name
    another build of the same sources (a variant from ``build.build(variant=...)``)."""
    global _lib
    if _lib is None:
        path = os.environ.get("ETAC_LIBRARY") or _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2604_20295_gb300.build.build()"
                               " (CUDA toolkit required); there is no CPU fallback")
        L = ctypes.CDLL(path)
        L.etac_param_count.restype = ctypes.c_size_t
        L.etac_param_count.argtypes = [_vp]
        L.etac_total_nodes.restype = ctypes.c_int64
        L.etac_total_nodes.argtypes = [_vp]
        L.etac_create_pads.restype = ctypes.c_int
        L.etac_create_pads.argtypes = [ctypes.POINTER(_vp), _vp, _vp]
        L.etac_set_model.restype = ctypes.c_int
        L.etac_set_model.argtypes = [_vp, _vp, _vp, _vp]
        L.etac_step_forward.restype = ctypes.c_int
        L.etac_step_forward.argtypes = [_vp, _vp, _vp, _vp]
        L.etac_step_backward.restype = ctypes.c_int
        L.etac_step_backward.argtypes = [_vp, ctypes.c_uint64] + [_vp] * 6
        L.etac_test_withhold_load.restype = ctypes.c_int
        L.etac_test_withhold_load.argtypes = [_vp, ctypes.c_int32, ctypes.c_uint64]
        L.etac_last_step.restype = ctypes.c_int
        L.etac_last_step.argtypes = [_vp, ctypes.POINTER(ctypes.c_uint64)]
        L.etac_poll_status.restype = ctypes.c_int
        L.etac_poll_status.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32), _vp]
        L.etac_forward_f64.restype = ctypes.c_int
        L.etac_forward_f64.argtypes = [_vp] * 9
        L.etac_last_error.restype = ctypes.c_char_p
        L.etac_last_error.argtypes = [_vp]
        L.etac_destroy.restype = None
        L.etac_destroy.argtypes = [_vp]
        L.etac_enable_timing.restype = ctypes.c_int
        L.etac_enable_timing.argtypes = [_vp, ctypes.c_int32]
        L.etac_kernel_times.restype = ctypes.c_int
        L.etac_kernel_times.argtypes = [_vp, _vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
        L.etac_autotune.restype = ctypes.c_int
        L.etac_autotune.argtypes = [_vp, ctypes.POINTER(etac_step_in), ctypes.POINTER(etac_step_out),
                                    _vp, ctypes.POINTER(etac_tuning), _vp]
        L.etac_set_tuning.restype = ctypes.c_int
        L.etac_set_tuning.argtypes = [_vp, ctypes.POINTER(etac_tuning), _vp]
        L.etac_pose_grad_to_quat.restype = ctypes.c_int
        L.etac_pose_grad_to_quat.argtypes = [_vp, _vp, _vp, ctypes.c_int64, _vp]
        L.etac_step_forward_noalloc.restype = ctypes.c_int
        L.etac_step_forward_noalloc.argtypes = [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp]
        L.etac_mesh_accel_build.restype = ctypes.c_int
        L.etac_mesh_accel_build.argtypes = [ctypes.POINTER(_vp), _vp]
        L.etac_mesh_accel_get_view.restype = ctypes.c_int
        L.etac_mesh_accel_get_view.argtypes = [_vp, ctypes.POINTER(etac_mesh_accel_view)]
        L.etac_mesh_accel_destroy.restype = None
        L.etac_mesh_accel_destroy.argtypes = [_vp]
        L.etac_mesh_gpu_create.restype = ctypes.c_int
        L.etac_mesh_gpu_create.argtypes = [ctypes.POINTER(_vp), _vp, _vp]
        L.etac_mesh_sdf_query.restype = ctypes.c_int
        L.etac_mesh_sdf_query.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp]
        L.etac_mesh_gpu_destroy.restype = None
        L.etac_mesh_gpu_destroy.argtypes = [_vp]
        L.etac_regress.restype = ctypes.c_int
        L.etac_regress.argtypes = [_vp] * 5 + [ctypes.c_int32, _vp]
        L.etac_set_meshes.restype = ctypes.c_int
        L.etac_set_meshes.argtypes = [_vp, _vp, ctypes.c_int32, _vp]
        _lib = L
    return _lib


def _check(ctx, status, what):
    if status != ETAC_OK:
        msg = lib().etac_last_error(ctx)
        raise EtacError(status, f"{what}: {msg.decode() if msg else ''}")


# ------------------------------------------------------------------ C entry points


def etac_param_count(desc: etac_model_desc) -> int:
    return int(lib().etac_param_count(ctypes.addressof(desc)))


def etac_total_nodes(desc: etac_pads_desc) -> int:
    return int(lib().etac_total_nodes(ctypes.addressof(desc)))


def etac_create_pads(desc: etac_pads_desc, stream: int = 0) -> int:
    out = _vp()
    _check(None, lib().etac_create_pads(ctypes.byref(out), ctypes.addressof(desc), stream),
           "etac_create_pads")
    return out.value


def etac_mesh_accel_build(desc: etac_mesh_desc) -> int:
    out = _vp()
    _check(None, lib().etac_mesh_accel_build(ctypes.byref(out), ctypes.addressof(desc)),
           "etac_mesh_accel_build")
    return out.value


def etac_mesh_accel_get_view(accel: int) -> etac_mesh_accel_view:
    v = etac_mesh_accel_view()
    _check(None, lib().etac_mesh_accel_get_view(accel, ctypes.byref(v)), "etac_mesh_accel_get_view")
    return v


def etac_mesh_accel_destroy(accel: int) -> None:
    lib().etac_mesh_accel_destroy(accel)


def mesh_accel(verts, tris, grid: int = 0) -> dict:
    """Builds the host acceleration structure of a closed triangle mesh (verts [V,3] float32,
    tris [T,3] int32) and returns copies of its arrays as numpy (host only, no GPU)."""
    v = np.ascontiguousarray(verts, np.float32)
    t = np.ascontiguousarray(tris, np.int32)
    h = etac_mesh_accel_build(etac_mesh_desc(len(v), len(t), v.ctypes.data, t.ctypes.data, grid))
    try:
        w = etac_mesh_accel_get_view(h)
        C = int(w.dims[0]) * int(w.dims[1]) * int(w.dims[2])
        T = int(w.num_tris)

        def arr(ptr, ctype, n, dtype):
            if n == 0:
                return np.zeros(0, dtype)
            return np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ctype)), (n,)).astype(dtype)
        return dict(origin=np.array(w.origin[:], np.float32), cell=float(w.cell),
                    dims=tuple(int(d) for d in w.dims), num_tris=T,
                    cell_start=arr(w.cell_start, ctypes.c_int32, C + 1, np.int32),
                    cell_kind=arr(w.cell_kind, ctypes.c_uint8, C, np.uint8),
                    cand=arr(w.cand, ctypes.c_int32, int(w.num_cand), np.int32),
                    tri=arr(w.tri, ctypes.c_float, 16 * T, np.float32).reshape(T, 4, 4),
                    pseudo=arr(w.pseudo, ctypes.c_float, 24 * T, np.float32).reshape(T, 6, 4))
    finally:
        etac_mesh_accel_destroy(h)


def etac_regress(ctx: int, disp: int, rparams: int, taxels: int, attn: int = 0,
                 precision: int = PREC_BF16, stream: int = 0) -> None:
    _check(ctx, lib().etac_regress(ctx, disp, rparams, taxels, attn or None, precision, stream),
           "etac_regress")


def etac_mesh_gpu_create(accel: int, stream: int = 0) -> int:
    out = _vp()
    _check(None, lib().etac_mesh_gpu_create(ctypes.byref(out), accel, stream), "etac_mesh_gpu_create")
    return out.value


def etac_mesh_sdf_query(mesh: int, n: int, q: int, phi: int, grad: int = 0, stream: int = 0) -> None:
    _check(None, lib().etac_mesh_sdf_query(mesh, n, q, phi, grad or None, stream),
           "etac_mesh_sdf_query")


def etac_set_meshes(ctx: int, meshes, stream: int = 0) -> None:
    """Meshes (device mesh handles) of the context's ETAC_OBJ_MESH objects, by index."""
    arr = (_vp * max(len(meshes), 1))(*[int(m) for m in meshes])
    _check(ctx, lib().etac_set_meshes(ctx, arr if len(meshes) else None, len(meshes), stream),
           "etac_set_meshes")


def etac_mesh_gpu_destroy(mesh: int) -> None:
    lib().etac_mesh_gpu_destroy(mesh)


class MeshSDF:
    """A closed triangle mesh resident on the GPU for signed-distance queries (builds the
    host acceleration structure, copies it to the device, frees the host copy)."""

    def __init__(self, verts, tris, grid: int = 0, stream: int = 0):
        v = np.ascontiguousarray(verts, np.float32)
        t = np.ascontiguousarray(tris, np.int32)
        acc = etac_mesh_accel_build(etac_mesh_desc(len(v), len(t), v.ctypes.data, t.ctypes.data, grid))
        try:
            self.handle = etac_mesh_gpu_create(acc, stream)
        finally:
            etac_mesh_accel_destroy(acc)

    def query(self, q, stream=None):
        """phi [n] and grad [n,3] (float32 CUDA tensors) at object-frame points q [n,3]
        (a float32 CUDA tensor); +inf where a point is outside without a computed distance."""
        import torch
        if not (q.is_cuda and q.dtype == torch.float32 and q.is_contiguous() and q.shape[-1] == 3):
            raise ValueError("q must be a contiguous float32 CUDA tensor of shape [n, 3]")
        n = q.numel() // 3
        phi = torch.empty(n, dtype=torch.float32, device=q.device)
        grad = torch.empty(n, 3, dtype=torch.float32, device=q.device)
        st = torch.cuda.current_stream().cuda_stream if stream is None else stream
        etac_mesh_sdf_query(self.handle, n, q.data_ptr(), phi.data_ptr(), grad.data_ptr(), st)
        return phi, grad

    def close(self):
        if getattr(self, "handle", None):
            etac_mesh_gpu_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def etac_set_model(ctx: int, desc: etac_model_desc, params: int, stream: int = 0) -> None:
    _check(ctx, lib().etac_set_model(ctx, ctypes.addressof(desc), params, stream), "etac_set_model")


def etac_step_forward(ctx: int, sin: etac_step_in, sout: etac_step_out, stream: int = 0) -> None:
    _check(ctx, lib().etac_step_forward(ctx, ctypes.addressof(sin), ctypes.addressof(sout), stream),
           "etac_step_forward")


def etac_test_withhold_load(ctx: int, tile: int, wait_limit_ns: int = 0) -> None:
    """Failure-path tests only: see include/etac.h."""
    _check(ctx, lib().etac_test_withhold_load(ctx, tile, wait_limit_ns), "etac_test_withhold_load")


def etac_last_step(ctx: int) -> int:
    v = ctypes.c_uint64(0)
    _check(ctx, lib().etac_last_step(ctx, ctypes.byref(v)), "etac_last_step")
    return int(v.value)


def etac_step_backward(ctx: int, grad_disp: int, grad_obj_pose: int = 0, grad_uhat: int = 0,
                       grad_penetration: int = 0, grad_params: int = 0, stream: int = 0,
                       step_id: int = 0) -> None:
    _check(ctx, lib().etac_step_backward(ctx, step_id, grad_disp, grad_obj_pose or None,
                                         grad_uhat or None, grad_penetration or None,
                                         grad_params or None, stream),
           "etac_step_backward")


def etac_poll_status(ctx: int, stream: int = 0) -> int:
    v = ctypes.c_int32(0)
    _check(ctx, lib().etac_poll_status(ctx, ctypes.byref(v), stream), "etac_poll_status")
    return int(v.value)


def etac_forward_f64(ctx: int, desc: etac_model_desc, obj_type: int, obj_dims: int,
                     obj_pose: int, pad_pose: int, params: int, disp: int, stream: int = 0) -> None:
    _check(ctx, lib().etac_forward_f64(ctx, ctypes.addressof(desc), obj_type, obj_dims, obj_pose,
                                       pad_pose, params, disp, stream), "etac_forward_f64")


def etac_last_error(ctx: int = 0) -> str:
    m = lib().etac_last_error(ctx or None)
    return m.decode() if m else ""


def etac_destroy(ctx: int) -> None:
    if ctx:
        lib().etac_destroy(ctx)


def etac_enable_timing(ctx: int, enable: bool = True) -> None:
    _check(ctx, lib().etac_enable_timing(ctx, int(bool(enable))), "etac_enable_timing")


def etac_autotune(ctx: int, step_in, step_out, grad_disp: int = 0, stream: int = 0) -> etac_tuning:
    r = etac_tuning()
    _check(ctx, lib().etac_autotune(ctx, ctypes.byref(step_in), ctypes.byref(step_out),
                                    grad_disp or None, ctypes.byref(r), stream), "etac_autotune")
    return r


def etac_set_tuning(ctx: int, tuning: etac_tuning, stream: int = 0) -> None:
    _check(ctx, lib().etac_set_tuning(ctx, ctypes.byref(tuning), stream), "etac_set_tuning")


def tuning_dict(t: etac_tuning) -> dict:
    return {"gemm_inst_per_tile": t.gemm_inst_per_tile, "gemm_tile_order": t.gemm_tile_order,
            "bwd_node_range": t.bwd_node_range,
            "fwd": [(t.fwd_cand[k][0], t.fwd_cand[k][1], round(t.fwd_ms[k], 4)) for k in range(t.num_fwd)],
            "bwd": [(t.bwd_cand[k], round(t.bwd_ms[k], 4)) for k in range(t.num_bwd)],
            "front_ctas_per_sm": t.front_ctas_per_sm,
            "front": [(t.front_cand[k], round(t.front_ms[k], 4)) for k in range(t.num_front)],
            "omega_source": t.omega_source,
            "omega_ms": [round(t.omega_ms[0], 4), round(t.omega_ms[1], 4)]}


def etac_kernel_times(ctx: int) -> dict:
    """{kernel name: (launches, summed ms)} since timing was enabled or last read."""
    buf = (etac_kernel_time * 32)()
    n = ctypes.c_int32(0)
    _check(ctx, lib().etac_kernel_times(ctx, ctypes.addressof(buf), 32, ctypes.byref(n)),
           "etac_kernel_times")
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms))
            for i in range(n.value)}


def etac_pose_grad_to_quat(poses: int, twist_grad: int, pose_grad: int, count: int,
                           stream: int = 0) -> None:
    _check(None, lib().etac_pose_grad_to_quat(poses, twist_grad, pose_grad, count, stream),
           "etac_pose_grad_to_quat")


def etac_step_forward_noalloc(pads: etac_noalloc_pads, mode: int, params: int,
                              sin: etac_step_in, sout: etac_step_out, device_status: int = 0,
                              stream: int = 0) -> None:
    """Batched FP32 forward that allocates nothing (scratch in a static device array);
    ``device_status`` is an optional device int32 that receives the step's status word."""
    _check(None, lib().etac_step_forward_noalloc(ctypes.addressof(pads), mode, params,
                                                 ctypes.addressof(sin), ctypes.addressof(sout),
                                                 device_status or None, stream),
           "etac_step_forward_noalloc")


# ------------------------------------------------------------------ convenience owner


def _device_f32(t, device, numel: int, what: str):
    """``t`` (tensor or array) as a contiguous float32 tensor on ``device`` holding exactly
    ``numel`` values; the library reads that many floats from the pointer it is given, so a
    host tensor or a short buffer is rejected here instead of reaching a kernel."""
    import torch
    t = torch.as_tensor(t).to(device=device, dtype=torch.float32).contiguous()
    if t.numel() != numel:
        raise EtacError(ERR_INVALID_ARG, f"{what} has {t.numel()} values, expected {numel}")
    return t


class TactileSim:
    """Owns an etac context for one batch of pads (a ``Scene`` from ``inputs``) together with
    device tensors for its inputs and outputs.  ``step()`` runs one forward on the current
    torch stream; inputs can be replaced in place between steps (e.g. under a CUDA graph)."""

    def __init__(self, scene, device="cuda"):
        import torch
        self.torch = torch
        self.scene = scene
        self.device = torch.device(device)
        self._host = dict(type_n=np.ascontiguousarray(scene.type_num_nodes, np.int32),
                          type_pos=np.ascontiguousarray(scene.type_pos, np.float32),
                          type_nrm=np.ascontiguousarray(scene.type_nrm, np.float32),
                          pad_type=np.ascontiguousarray(scene.pad_type, np.int32))
        h = self._host
        self.pads_desc = etac_pads_desc(len(scene.types), h["type_n"].ctypes.data,
                                        h["type_pos"].ctypes.data, h["type_nrm"].ctypes.data,
                                        scene.num_envs, scene.pads_per_env,
                                        h["pad_type"].ctypes.data, scene.max_objects)
        self.N = etac_total_nodes(self.pads_desc)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        self.ctx = etac_create_pads(self.pads_desc, stream)
        E, P, K = scene.num_envs, scene.pads_per_env, scene.max_objects
        f32, i32, dev = torch.float32, torch.int32, self.device
        self.obj_type = torch.as_tensor(scene.obj_type, dtype=i32).to(dev)
        self.obj_dims = torch.as_tensor(scene.obj_dims, dtype=f32).to(dev)
        self.obj_pose = torch.as_tensor(scene.obj_pose, dtype=f32).to(dev)
        self.pad_pose = torch.as_tensor(scene.pad_pose, dtype=f32).to(dev)
        self.disp = torch.zeros(self.N, 3, dtype=f32, device=dev)
        self.mask = torch.zeros(self.N, dtype=torch.uint8, device=dev)
        self.pen = torch.zeros(self.N, dtype=f32, device=dev)
        self.count = torch.zeros(E * P, dtype=i32, device=dev)
        self.model = None

    def set_model(self, params, mode=MODE_FULL, precision=PREC_FP32, algo=ALGO_PLAIN):
        torch = self.torch
        model = etac_model_desc(HIDDEN, mode, precision, algo)
        self.params = _device_f32(params, self.device, etac_param_count(model), "params")
        self.model = model
        etac_set_model(self.ctx, self.model, self.params.data_ptr(),
                       torch.cuda.current_stream(self.device).cuda_stream)

    def set_meshes(self, meshes=None):
        """Builds device meshes for the scene's meshes (``scene.meshes``, or the given list of
        ``MeshSDF``) and hands them to the context for OBJ_MESH objects; they stay owned by
        this object."""
        if meshes is None:
            meshes = [MeshSDF(m.verts, m.tris) for m in self.scene.meshes]
        self._meshes = list(meshes)
        etac_set_meshes(self.ctx, [m.handle for m in self._meshes],
                        self.torch.cuda.current_stream(self.device).cuda_stream)

    def step_in(self, given=None) -> etac_step_in:
        """Step inputs; ``given`` = (u_hat [N, 3] float32, mask [N] uint8) device tensors
        selects mode B (the caller's contact result; objects are not read)."""
        if given is None:
            return etac_step_in(self.obj_type.data_ptr(), self.obj_dims.data_ptr(),
                                self.obj_pose.data_ptr(), self.pad_pose.data_ptr())
        u, m = given
        return etac_step_in(None, None, None, None, u.data_ptr(), m.data_ptr())

    def step_out(self, want_mask=True, want_pen=True, want_count=True, disp=None) -> etac_step_out:
        d = self.disp if disp is None else disp
        return etac_step_out(d.data_ptr(), self.mask.data_ptr() if want_mask else None,
                             self.pen.data_ptr() if want_pen else None,
                             self.count.data_ptr() if want_count else None)

    def regress(self, rparams, disp=None, want_attn=True, precision=None):
        """Real-to-sim taxel regressor on every pad: taxels [E*P, 8] (and each node's softmax
        weight [N]) from a displacement field (default: the last step's) and the regressor's
        flat FP32 parameters (a device tensor or array of REGRESSOR_PARAMS values).
        ``precision``: PREC_BF16 (default; the per-node layers on the tensor cores) or
        PREC_FP32 (all layers in FP32 on the CUDA cores)."""
        torch = self.torch
        rp = torch.as_tensor(np.asarray(rparams, np.float32) if not torch.is_tensor(rparams)
                             else rparams, dtype=torch.float32).to(self.device).contiguous()
        if rp.numel() != REGRESSOR_PARAMS:
            raise ValueError(f"regressor parameters: {rp.numel()} values, want {REGRESSOR_PARAMS}")
        d = self.disp if disp is None else disp
        if not (d.is_cuda and d.dtype == torch.float32 and d.is_contiguous() and d.numel() == 3 * self.N):
            raise ValueError("disp must be a contiguous float32 CUDA tensor of shape [N, 3]")
        npads = self.scene.num_envs * self.scene.pads_per_env
        taxels = torch.empty(npads, TAXELS, dtype=torch.float32, device=self.device)
        attn = torch.empty(self.N, dtype=torch.float32, device=self.device) if want_attn else None
        etac_regress(self.ctx, d.data_ptr(), rp.data_ptr(), taxels.data_ptr(),
                     attn.data_ptr() if want_attn else 0,
                     PREC_BF16 if precision is None else precision,
                     torch.cuda.current_stream(self.device).cuda_stream)
        return taxels, attn

    def step(self, want_mask=True, want_pen=True, want_count=True, disp=None, uhat_in=None,
             mask_in=None):
        """One forward step on the current stream.  ``disp`` (a contiguous float32 [N, 3]
        device tensor) receives the displacement instead of ``self.disp``, e.g. to alternate
        output buffers while an earlier step's result is copied to the host.  ``uhat_in``
        ([N, 3] float32) and ``mask_in`` ([N] uint8), both device tensors, select mode B: the
        contact result comes from the caller (kept referenced here until the next step, since
        the reverse mode reads them again)."""
        if disp is not None and (disp.shape != self.disp.shape or disp.dtype != self.disp.dtype
                                 or not disp.is_contiguous() or disp.device != self.disp.device):
            raise EtacError(ERR_INVALID_ARG, f"disp must be a contiguous float32 "
                            f"{tuple(self.disp.shape)} tensor on {self.disp.device}")
        given = None
        if uhat_in is not None or mask_in is not None:
            torch = self.torch
            if uhat_in is None or mask_in is None:
                raise EtacError(ERR_INVALID_ARG, "uhat_in and mask_in go together")
            u = _device_f32(uhat_in, self.device, 3 * self.N, "uhat_in")
            m = torch.as_tensor(mask_in).to(device=self.device, dtype=torch.uint8).contiguous()
            if m.numel() != self.N:
                raise EtacError(ERR_INVALID_ARG, f"mask_in has {m.numel()} values, expected {self.N}")
            given = (u, m)
        self._given = given
        etac_step_forward(self.ctx, self.step_in(given),
                          self.step_out(want_mask, want_pen, want_count, disp),
                          self.torch.cuda.current_stream(self.device).cuda_stream)
        return self.disp if disp is None else disp

    def last_step(self) -> int:
        """Id of the last forward step on this context (etac_last_step)."""
        return etac_last_step(self.ctx)

    def backward(self, grad_disp, want=("params", "obj_pose", "uhat", "pen"), step_id=0):
        """Reverse mode of a step for dL/d(disp) = grad_disp [N,3] (device tensor): the step
        ``step_id`` (from ``last_step()``; the library refuses one that is no longer the
        last), or the last step when 0.  Returns a dict with any of: params [P], obj_pose
        [E*K, 6] (dL/dt, dL/d omega), uhat [N, 3], pen [N]."""
        torch = self.torch
        g = _device_f32(grad_disp, self.device, 3 * self.N, "grad_disp")
        out = {}
        f32 = dict(dtype=torch.float32, device=self.device)
        sc = self.scene
        if "params" in want:
            out["params"] = torch.empty(self.params.numel(), **f32)
        if "obj_pose" in want:
            out["obj_pose"] = torch.empty(sc.num_envs * sc.max_objects, 6, **f32)
        if "uhat" in want:
            out["uhat"] = torch.empty(self.N, 3, **f32)
        if "pen" in want:
            out["pen"] = torch.empty(self.N, **f32)
        ptr = lambda k: out[k].data_ptr() if k in out else 0
        etac_step_backward(self.ctx, g.data_ptr(), ptr("obj_pose"), ptr("uhat"), ptr("pen"),
                           ptr("params"), torch.cuda.current_stream(self.device).cuda_stream,
                           step_id)
        self._grad_keepalive = g
        return out

    def tuning_key(self, with_reverse: bool) -> str:
        """What a tuning choice depends on: the GPU (name, SM count), the pad-type histogram
        (node count and instances of each type), objects per env and the model's mode,
        precision and algorithm."""
        props = self.torch.cuda.get_device_properties(self.device)
        sc = self.scene
        inst = np.bincount(np.asarray(sc.pad_type), minlength=len(sc.types))
        hist = ",".join(f"{int(n)}x{int(k)}" for n, k in zip(sc.type_num_nodes, inst))
        m = self.model
        return (f"{props.name}|sms={props.multi_processor_count}|types={hist}|K={sc.max_objects}|"
                f"mode={m.mode}|prec={m.precision}|algo={m.algo}|reverse={int(with_reverse)}")

    def autotune(self, grad_disp=None, cache=None) -> dict:
        """Times the tile / block shape candidates on this scene's step (and, given an upstream
        gradient, the reverse mode's node ranges) and keeps the fastest.  ``cache`` (a JSON
        file path) stores each choice under ``tuning_key``; a later call with the same key
        applies the stored choice without timing (the result then has "cached": True)."""
        import json
        key = self.tuning_key(grad_disp is not None)
        table = {}
        if cache is not None and os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
            if key in table:
                d = table[key]
                self.set_tuning(d["gemm_inst_per_tile"], d["gemm_tile_order"], d["bwd_node_range"],
                                d.get("front_ctas_per_sm", 0), d.get("omega_source", 0))
                return dict(d, cached=True)
        g = None if grad_disp is None else _device_f32(grad_disp, self.device, 3 * self.N,
                                                       "grad_disp")
        t = etac_autotune(self.ctx, self.step_in(), self.step_out(),
                          0 if g is None else g.data_ptr(),
                          self.torch.cuda.current_stream(self.device).cuda_stream)
        d = tuning_dict(t)
        if cache is not None:
            table[key] = d
            tmp = f"{cache}.tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1)
            os.replace(tmp, cache)
        return dict(d, cached=False)

    def set_tuning(self, inst_per_tile=64, tile_order=0, bwd_node_range=0, front_ctas_per_sm=0,
                   omega_source=0):
        """Applies tile / block shapes (see etac_tuning in etac.h); ``omega_source`` is one of
        OMEGA_AUTO, OMEGA_TABLE, OMEGA_ON_THE_FLY (batched FP32 only)."""
        t = etac_tuning()
        t.gemm_inst_per_tile, t.gemm_tile_order, t.bwd_node_range = inst_per_tile, tile_order, bwd_node_range
        t.front_ctas_per_sm = front_ctas_per_sm
        t.omega_source = omega_source
        etac_set_tuning(self.ctx, t, self.torch.cuda.current_stream(self.device).cuda_stream)

    def poll_status(self) -> int:
        return etac_poll_status(self.ctx, self.torch.cuda.current_stream(self.device).cuda_stream)

    def close(self):
        if getattr(self, "ctx", 0):
            etac_destroy(self.ctx)
            self.ctx = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# (algo, precision, relative tolerance) exercised by the smoke check
SMOKE_CONFIGS = ((ALGO_PLAIN, PREC_FP32, 1e-5), (ALGO_BATCHED, PREC_FP32, 1e-5),
                 (ALGO_BATCHED, PREC_BF16, 2e-2))


def make_step_function():
    """torch.autograd.Function over one tactile step: (params, obj_pose) -> displacement.

    ``ETacStep.apply(sim, params, obj_pose)`` copies params and poses into ``sim`` (the
    model is re-set when params change), runs the forward and returns a copy of the
    displacement; backward returns dL/dparams and dL/d(obj_pose) in the 7-float pose layout.
    The context keeps the saved state of its last forward only, so each apply records the
    step id the library gave it; when a later apply on the same ``sim`` has replaced that
    state (a multi-step rollout), backward first re-runs this step's forward from its saved
    params and pose, then differentiates it under its new id.  All arithmetic runs in the
    library's kernels."""
    import torch

    def _run(sim, p, pose):
        if getattr(sim, "params", None) is None or not torch.equal(sim.params, p):
            m = sim.model
            sim.set_model(p, m.mode, m.precision, m.algo)
        sim.obj_pose.copy_(pose)
        disp = sim.step().clone()
        return disp, sim.last_step()

    class ETacStep(torch.autograd.Function):
        @staticmethod
        def forward(ctx, sim, params, obj_pose):
            p = params.detach().to(device=sim.device, dtype=torch.float32).contiguous()
            pose = obj_pose.detach().reshape(-1).to(device=sim.device, dtype=torch.float32)
            disp, sid = _run(sim, p, pose)
            ctx.sim, ctx.step_id = sim, sid
            ctx.params, ctx.pose = p.clone(), pose.clone()
            return disp

        @staticmethod
        def backward(ctx, grad_disp):
            sim, sid = ctx.sim, ctx.step_id
            if sim.last_step() != sid:
                _, sid = _run(sim, ctx.params, ctx.pose)
            g = sim.backward(grad_disp, want=("params", "obj_pose"), step_id=sid)
            pose7 = torch.empty(sim.obj_pose.numel(), dtype=torch.float32, device=sim.device)
            etac_pose_grad_to_quat(sim.obj_pose.data_ptr(), g["obj_pose"].data_ptr(),
                                   pose7.data_ptr(), sim.obj_pose.numel() // 7,
                                   torch.cuda.current_stream(sim.device).cuda_stream)
            return None, g["params"], pose7.reshape(-1)

    return ETacStep
