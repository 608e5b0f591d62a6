"""Memory and undefined-behaviour checks of the host C/C++ code (CPU only), with gcc's address
and undefined-behaviour sanitizers:

- the FP64 oracle and the host-built mesh acceleration structure, under the oracle pins and
  the mesh-structure tests;
- the whole libetac with its host code sanitized (device code unchanged), under the ABI and
  mesh-structure tests: argument validation, error paths and the host-side builders.

The tests run in a child process (tests/sanitizer_run.py) whose LD_PRELOAD holds the
sanitizer runtime.  An out-of-bounds access, a use after free or an undefined operation
aborts the child: a planted off-by-one read in the oracle's first layer was caught this way,
and so was a read of a freed context in an error message of etac_create_pads."""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))
SAN = ["-fsanitize=address", "-fsanitize=undefined", "-fno-sanitize-recover=undefined",
       "-fno-omit-frame-pointer", "-g"]   # one option each: nvcc -Xcompiler splits at commas


def _runtime():
    try:
        p = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True,
                           text=True, check=True).stdout.strip()
    except (OSError, subprocess.CalledProcessError):
        return None
    return p if os.path.isabs(p) and os.path.exists(p) else None


def _run(libs, files):
    asan = _runtime()
    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1")
    opts = [a for k, v in libs.items() for a in (k, v)]
    r = subprocess.run([sys.executable, os.path.join(HERE, "sanitizer_run.py"), *opts, "--",
                        "-x", "-q", "-s", "-p", "no:cacheprovider", "-k", "not planted",
                        *[os.path.join(HERE, f) for f in files]],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    out = r.stdout + r.stderr
    assert r.returncode == 0, out[-4000:]
    assert "AddressSanitizer" not in out and "runtime error" not in out, out[-4000:]
    assert " passed" in out


@pytest.fixture(scope="module")
def runtime():
    if _runtime() is None:
        pytest.skip("gcc's address-sanitizer runtime is not installed")


@pytest.mark.slow
def test_oracle_and_mesh_structure_are_clean_under_sanitizers(runtime, tmp_path):
    ora = str(tmp_path / "liboracle_san.so")
    mesh = str(tmp_path / "libmesh_san.so")
    base = ["-O1", *SAN, "-fPIC", "-shared"]
    subprocess.check_call(["gcc", *base, "-fopenmp", "-o", ora,
                           os.path.join(ROOT, "oracle", "etac_oracle.c"), "-lm"])
    subprocess.check_call(["g++", *base, "-std=c++17", "-pthread",
                           "-I" + os.path.join(ROOT, "include"), "-o", mesh,
                           os.path.join(ROOT, "paper_2604_20295_gb300", "csrc", "mesh_accel.cpp"),
                           os.path.join(HERE, "sanitizer_stub.cpp")])
    _run({"--oracle": ora, "--mesh": mesh},
         ["test_oracle_pins.py", "test_oracle_mesh.py", "test_oracle_regressor.py",
          "test_mesh_accel.py"])


@pytest.mark.slow
def test_library_host_code_is_clean_under_sanitizers(runtime, tmp_path):
    from paper_2604_20295_gb300 import build as B
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc is not installed")
    host = ["-Xcompiler", ",".join(SAN)]

    def compile_one(src):
        obj = str(tmp_path / (os.path.basename(src) + ".o"))
        subprocess.check_call([nvcc, *B.ARCH, *B.NVCC_FLAGS, *host, "-c", src, "-o", obj],
                              stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        return obj

    srcs = B.sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    lib = str(tmp_path / "libetac_san.so")
    subprocess.check_call([nvcc, *B.ARCH, "-shared", "-o", lib, *objs, *host])
    assert len(glob.glob(str(tmp_path / "*.o"))) == len(srcs)
    _run({"--etac": lib}, ["test_abi.py", "test_mesh_accel.py"])
