"""Runs CPU test files with sanitizer builds swapped in for the compiled code they load.

    python tests/sanitizer_run.py [--oracle SO] [--mesh SO] [--etac SO] -- <pytest args>

--oracle replaces the FP64 oracle library, --mesh a build of the host mesh structure alone,
--etac a host-sanitized build of the whole libetac.  Started by tests/test_sanitizers.py in
a child process whose LD_PRELOAD holds the sanitizer runtime.  Test infrastructure only."""
import ctypes
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import pytest  # noqa: E402

import oracle as O  # noqa: E402
from paper_2604_20295_gb300 import build as B  # noqa: E402
from paper_2604_20295_gb300 import etac as X  # noqa: E402


def _use_mesh_only(path):
    L = ctypes.CDLL(path)
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
    B.build = lambda *a, **k: path     # nothing is compiled under the sanitizer runtime


def _use_etac(path):
    B.LIB = path
    B.build = lambda *a, **k: path     # the tests' build() calls keep this library
    X._lib = None
    X.lib()


def main(argv):
    sep = argv.index("--")
    opts, pytest_args = argv[:sep], argv[sep + 1:]
    libs = dict(zip(opts[0::2], opts[1::2]))
    if "--oracle" in libs:
        O._lib = O._open(libs["--oracle"])
    if "--mesh" in libs:
        _use_mesh_only(libs["--mesh"])
    if "--etac" in libs:
        _use_etac(libs["--etac"])
    maps = open("/proc/self/maps").read()
    assert all(os.path.basename(p) in maps for p in libs.values()), "sanitizer build not loaded"
    return pytest.main(pytest_args)


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
