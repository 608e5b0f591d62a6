"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/etac.h declares; host-side argument checks work without a GPU (CPU only)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2604_20295_gb300 import build as B
from paper_2604_20295_gb300 import etac as X
from paper_2604_20295_gb300 import inputs as I

HEADER = os.path.join(B.ROOT, "include", "etac.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(etac_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return X.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(X.EXPORTS)


def test_param_count_matches_layout(lib):
    d = X.etac_model_desc(64, 0, 0, 0)
    assert X.etac_param_count(d) == I.param_count() == 17412
    assert X.etac_param_count(X.etac_model_desc(32, 0, 0, 0)) == 0


def test_total_nodes_and_validation(lib):
    sc = I.hand_scene(2, seed=0)
    tn = np.ascontiguousarray(sc.type_num_nodes, np.int32)
    pt = np.ascontiguousarray(sc.pad_type, np.int32)
    pos = np.ascontiguousarray(sc.type_pos)
    d = X.etac_pads_desc(2, tn.ctypes.data, pos.ctypes.data, pos.ctypes.data, 2, 6,
                         pt.ctypes.data, 1)
    assert X.etac_total_nodes(d) == sc.total_nodes == 2 * (5 * 512 + 2048)
    bad = np.array([0, 0, 0, 0, 0, 7] * 2, np.int32)
    d.pad_type = bad.ctypes.data
    assert X.etac_total_nodes(d) == 0
    # create rejects a bad description on the host, before touching any GPU
    with pytest.raises(X.EtacError) as e:
        X.etac_create_pads(d)
    assert e.value.status == 1
    assert X.lib().etac_create_pads(None, None, None) == 1
    d.pad_type = pt.ctypes.data
    d.max_objects = 99
    with pytest.raises(X.EtacError) as e:
        X.etac_create_pads(d)
    assert e.value.status == 1 and "max_objects" in X.etac_last_error(0)


def test_null_context_calls_fail_cleanly(lib):
    m = X.etac_model_desc(64, 0, 0, 0)
    assert lib.etac_set_model(None, ctypes.addressof(m), None, None) == 1
    assert lib.etac_step_forward(None, None, None, None) == 1
    assert lib.etac_step_backward(None, 0, None, None, None, None, None, None) == 1
    lib.etac_destroy(None)


def _header_enums():
    """name -> value of every `ETAC_NAME = value` in the header's enums."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\bETAC_([A-Z0-9_]+)\s*=\s*(\d+)", src)}


def test_binding_constants_match_the_header():
    """The binding's mode, precision, algorithm, object and status numbers are the header's,
    and the oracle numbers the modes the same way."""
    import oracle as O

    e = _header_enums()
    for name in ("MODE_FULL", "MODE_LINEAR_ONLY", "MODE_RESIDUAL_ONLY", "MODE_PENETRATION_ONLY",
                 "PREC_FP32", "PREC_BF16", "ALGO_PLAIN", "ALGO_BATCHED", "OMEGA_AUTO",
                 "OMEGA_TABLE", "OMEGA_ON_THE_FLY"):
        assert getattr(X, name) == e[name], name
    for name in ("MODE_FULL", "MODE_LINEAR_ONLY", "MODE_RESIDUAL_ONLY", "MODE_PENETRATION_ONLY"):
        assert getattr(O, name) == e[name], name
    for name in ("OBJ_NONE", "OBJ_SPHERE", "OBJ_BOX", "OBJ_CYLINDER", "OBJ_CAPSULE"):
        assert getattr(I, name) == e[name], name
    for code, label in X.STATUS_NAMES.items():
        assert e[label[len("ETAC_"):]] == code, label
    assert X.ERR_INVALID_ARG == e["ERR_INVALID_ARG"]
    for name in ("CELL_OUTSIDE", "CELL_INSIDE", "CELL_SURFACE"):
        assert getattr(X, name) == e[name], name
    defs = {m.group(1): int(m.group(2)) for m in
            re.finditer(r"#define ETAC_([A-Z0-9_]+)\s+(\d+)\b", open(HEADER).read())}
    assert X.TAXELS == defs["TAXELS"] == I.REG_TAXELS
    assert X.REGRESSOR_PARAMS == defs["REGRESSOR_PARAMS"] == I.regressor_param_count()
    assert O.regressor_param_count() == I.regressor_param_count()


def _noalloc_scratch_bytes(type_nodes, num_pads):
    """Bytes of static scratch that the no-allocation step needs, restated from the limit
    the header gives: 896 B per pad-type node, 4 B per same-type node pair and 4 B per pad
    instance, each array starting on a 256-byte boundary (plus the queue counter, the status
    word, the invalid-input word, the Omega offsets and the per-type extents)."""
    up = lambda b: (b + 255) // 256 * 256
    T, tn = len(type_nodes), sum(type_nodes)
    nn2 = sum(n * n for n in type_nodes)
    return (up(4) + up(4) + up(4) + up(8 * (T + 1)) + up(4 * T) + up(4 * num_pads)
            + 3 * up(4 * 64 * tn) + up(2 * 64 * tn) + up(4 * nn2))


def test_noalloc_host_checks_need_no_gpu(lib):
    """etac_step_forward_noalloc rejects bad arguments and batches beyond its static scratch
    on the host, before any CUDA call: every case here fails before the library would read a
    device pointer, so the placeholder addresses below are never dereferenced."""
    fake = np.zeros(16, np.int64)            # stands in for device pointers
    ptr = fake.ctypes.data
    sin = X.etac_step_in(ptr, ptr, ptr, ptr)
    sout = X.etac_step_out(ptr, None, None, None)

    def call(tn, mode=0, envs=1, ppe=1, K=1):
        tn = np.ascontiguousarray(tn, np.int32)
        pads = X.etac_noalloc_pads(len(tn), tn.ctypes.data, ptr, ptr, ptr, envs, ppe, K, ptr,
                                   ptr)
        with pytest.raises(X.EtacError) as e:
            X.etac_step_forward_noalloc(pads, mode, ptr, sin, sout, 0)
        assert e.value.status == X.ERR_INVALID_ARG
        return str(e.value)

    assert lib.etac_step_forward_noalloc(None, 0, None, None, None, None, None) == X.ERR_INVALID_ARG
    assert "NULL" in X.etac_last_error(0)
    assert "unknown mode" in call([256], mode=4)
    assert "bad sizes" in call([256], K=9)
    assert "pad type size" in call([256, 0])
    assert "pad type size" in call([4097])
    # past the 32 MiB scratch: the message gives the bytes needed, as the header's limit says
    for tn, pads in (([4096] * 16, 1), ([4096], 1), ([2048] * 2, 4), ([256], 9_000_000)):
        need = _noalloc_scratch_bytes(tn, pads)
        assert need > 32 << 20
        msg = call(tn, envs=pads)
        assert f"need {need} bytes of scratch" in msg, msg
        assert f"holds {32 << 20} bytes" in msg


def test_create_rejects_empty_and_oversized_descriptions(lib):
    """Empty batches (no environments, no pads per env, no pad types), pad types of 0 or
    more than ETAC_MAX_PAD_NODES nodes and non-finite geometry are rejected on the host with
    ETAC_ERR_INVALID_ARG and a message, before any GPU work."""
    def attempt(tn, envs=1, ppe=1, T=None, pos=None, K=1):
        tn = np.ascontiguousarray(tn, np.int32)
        n = max(int(tn.sum()), 1)
        pos = np.zeros((n, 3), np.float32) if pos is None else pos
        nrm = np.tile(np.float32([0, 0, 1]), (n, 1))
        pt = np.zeros(max(envs * ppe, 1), np.int32)
        d = X.etac_pads_desc(len(tn) if T is None else T, tn.ctypes.data, pos.ctypes.data,
                             nrm.ctypes.data, envs, ppe, pt.ctypes.data, K)
        with pytest.raises(X.EtacError) as e:
            X.etac_create_pads(d)
        assert e.value.status == X.ERR_INVALID_ARG
        return X.etac_last_error(0)

    assert ">= 1" in attempt([16], envs=0)
    assert ">= 1" in attempt([16], ppe=0)
    assert "num_types" in attempt([16], T=0)
    assert "0 nodes" in attempt([0])
    assert "4097 nodes" in attempt([4097])
    bad = np.zeros((16, 3), np.float32)
    bad[5, 1] = np.nan
    assert "non-finite" in attempt([16], pos=bad)
    assert "max_objects" in attempt([16], K=0)


def test_binding_converts_and_sizes_device_buffers():
    """The binding hands the library float32 buffers of exactly the size it reads: arrays and
    other dtypes are converted, and a buffer of the wrong size is refused before any call."""
    import torch

    cpu = torch.device("cpu")
    t = X._device_f32(np.arange(6, dtype=np.float64).reshape(2, 3), cpu, 6, "x")
    assert t.dtype == torch.float32 and t.is_contiguous() and t.tolist() == [[0, 1, 2], [3, 4, 5]]
    nc = torch.arange(12, dtype=torch.float32).reshape(3, 4)[:, :3]
    assert not nc.is_contiguous()
    c = X._device_f32(nc, cpu, 9, "x")
    assert c.is_contiguous() and torch.equal(c, nc)
    with pytest.raises(X.EtacError) as e:
        X._device_f32(torch.zeros(17411), cpu, 17412, "params")
    assert e.value.status == X.ERR_INVALID_ARG and "17411 values, expected 17412" in str(e.value)


_STRUCTS = ("etac_pads_desc", "etac_model_desc", "etac_step_in", "etac_step_out", "etac_tuning",
            "etac_kernel_time", "etac_mesh_desc", "etac_mesh_accel_view", "etac_noalloc_pads")


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every struct the binding passes by address has the header's size and field offsets:
    a C program built against include/etac.h prints sizeof / offsetof, compared with ctypes."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "etac.h"', "int main(void) {"]
    for s in _STRUCTS:
        ct = getattr(X, s)
        lines.append(f'  printf("{s} size %zu\\n", sizeof({s}));')
        for f, _ in ct._fields_:
            lines.append(f'  printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c11", "-I" + os.path.dirname(HEADER), str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n"):
        if line:
            s, f, v = line.split()
            got[(s, f)] = int(v)
    for s in _STRUCTS:
        ct = getattr(X, s)
        assert got[(s, "size")] == ctypes.sizeof(ct), s
        for f, _ in ct._fields_:
            assert got[(s, f)] == getattr(ct, f).offset, (s, f)
    assert sorted(set(re.findall(r"\}\s*(etac_[a-z_]+)\s*;", open(HEADER).read())) - {"etac_status"}) \
        == sorted(_STRUCTS)


def test_binding_prototypes_match_the_header(lib):
    """Each declared function has argument types set in the binding, as many as the header's
    prototype takes, and a C int result where the header returns etac_status."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    protos = re.findall(r"\b(etac_status|size_t|int64_t|void|const char\*)\s+(etac_[a-z0-9_]+)"
                        r"\s*\(([^)]*)\)\s*;", src)
    assert sorted(p[1] for p in protos) == _declared()
    for ret, name, args in protos:
        fn = getattr(lib, name)
        n = 0 if args.strip() in ("", "void") else args.count(",") + 1
        assert fn.argtypes is not None and len(fn.argtypes) == n, name
        if ret == "etac_status":
            assert fn.restype is ctypes.c_int, name


def test_library_exports_only_declared_entry_points(lib):
    """The C-linkage etac_* symbols the library exports are exactly the header's entry points
    (read from the library's dynamic symbol table with nm)."""
    import shutil
    import subprocess

    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm is not installed")
    out = subprocess.run([nm, "-D", "--defined-only", B.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = sorted({f[2] for f in (l.split() for l in out.splitlines())
                       if len(f) == 3 and f[1] == "T" and f[2].startswith("etac_")})
    assert exported == _declared()
