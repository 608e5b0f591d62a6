"""Runs CPU test files with the oracle and the host mesh structure swapped for sanitizer
builds (argv: oracle .so, mesh .so, then pytest arguments).  Started by
tests/test_sanitizers.py in a child process whose LD_PRELOAD holds the sanitizer runtime."""
import ctypes
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import pytest  # noqa: E402

import oracle as O  # noqa: E402
from paper_2604_20295_gb300 import etac as X  # noqa: E402


def main(oracle_so, mesh_so, *pytest_args):
    O._lib = O._open(oracle_so)
    L = ctypes.CDLL(mesh_so)
    vp = ctypes.c_void_p
    L.etac_mesh_accel_build.restype = ctypes.c_int
    L.etac_mesh_accel_build.argtypes = [ctypes.POINTER(vp), vp]
    L.etac_mesh_accel_get_view.restype = ctypes.c_int
    L.etac_mesh_accel_get_view.argtypes = [vp, ctypes.POINTER(X.etac_mesh_accel_view)]
    L.etac_mesh_accel_destroy.restype = None
    L.etac_mesh_accel_destroy.argtypes = [vp]
    L.etac_last_error.restype = ctypes.c_char_p
    L.etac_last_error.argtypes = [vp]
    X._lib = L
    X.lib = lambda: L
    maps = open("/proc/self/maps").read()
    assert os.path.basename(oracle_so) in maps and os.path.basename(mesh_so) in maps
    return pytest.main(list(pytest_args))


if __name__ == "__main__":
    sys.exit(main(*sys.argv[1:]))
