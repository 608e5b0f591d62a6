"""Memory and undefined-behaviour checks of the host C/C++ code (CPU only): the FP64 oracle
and the host-built mesh acceleration structure are compiled with gcc's address and
undefined-behaviour sanitizers, and the oracle pins and mesh-structure tests run against
those builds in a child process.  An out-of-bounds access, a use after free or an undefined
operation aborts the child (a planted off-by-one read in the oracle's first layer was caught
this way)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))
FLAGS = ["-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
         "-fno-omit-frame-pointer", "-fPIC", "-shared"]


def _runtime():
    try:
        p = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True,
                           text=True, check=True).stdout.strip()
    except (OSError, subprocess.CalledProcessError):
        return None
    return p if os.path.isabs(p) and os.path.exists(p) else None


@pytest.mark.slow
def test_oracle_and_mesh_structure_are_clean_under_sanitizers(tmp_path):
    asan = _runtime()
    if asan is None:
        pytest.skip("gcc's address-sanitizer runtime is not installed")
    ora = str(tmp_path / "liboracle_san.so")
    mesh = str(tmp_path / "libmesh_san.so")
    subprocess.check_call(["gcc", *FLAGS, "-fopenmp", "-o", ora,
                           os.path.join(ROOT, "oracle", "etac_oracle.c"), "-lm"])
    subprocess.check_call(["g++", *FLAGS, "-std=c++17", "-pthread",
                           "-I" + os.path.join(ROOT, "include"), "-o", mesh,
                           os.path.join(ROOT, "paper_2604_20295_gb300", "csrc", "mesh_accel.cpp"),
                           os.path.join(HERE, "sanitizer_stub.cpp")])
    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1")
    files = [os.path.join(HERE, f) for f in ("test_oracle_pins.py", "test_oracle_mesh.py",
                                              "test_oracle_regressor.py", "test_mesh_accel.py")]
    r = subprocess.run([sys.executable, os.path.join(HERE, "sanitizer_run.py"), ora, mesh,
                        "-x", "-q", "-s", "-p", "no:cacheprovider", "-k", "not planted", *files],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    out = r.stdout + r.stderr
    assert r.returncode == 0, out[-4000:]
    assert "AddressSanitizer" not in out and "runtime error" not in out, out[-4000:]
    assert " passed" in out
