"""The exact contact decision (contact_refine) built as an out-of-line call in every kernel
must give the inlined library's results: the reverse-mode parity tests against the oracle (all
scenes and modes, entry by entry) and the forward parity tests run again, in a child process,
on the ``outline_refine`` build of the same sources."""
import os
import subprocess
import sys

import pytest

from paper_2604_20295_gb300 import build as B

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_outlined_contact_refine_passes_the_parity_tests():
    lib = B.build(variant="outline_refine")
    env = dict(os.environ, ETAC_LIBRARY=lib)
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
           "tests/test_gpu_backward.py", "tests/test_gpu_forward.py",
           "-k", "matches_oracle or sampled_envs or uneven_pads"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout, tail
