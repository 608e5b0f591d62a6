"""The ETAC_BOUNDS build (index checks that latch ETAC_ERR_BOUNDS and skip the access instead of
faulting) on valid inputs: no check fires and every output equals the regular build's, bit for
bit.  Both libraries run the same child script (tests/bounds_run.py) in their own process:
every forward algorithm and precision in every mode, mode B, mesh objects, the reverse mode and
the regressor.  No test plants a bad index on the GPU: an out-of-range access is what the build
exists to catch, and only valid inputs are run here."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2604_20295_gb300 import build as B

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(lib, path):
    env = dict(os.environ, ETAC_LIBRARY=lib,
               PYTHONPATH=os.pathsep.join([ROOT] + [p for p in [os.environ.get("PYTHONPATH")] if p]))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_run.py"), path],
                       cwd=ROOT, env=env, capture_output=True, text=True)
    assert r.returncode == 0, (r.stdout + r.stderr)[-3000:]
    return dict(np.load(path))


def test_bounds_build_fires_no_check_and_changes_no_output(tmp_path):
    regular = _run(B.build(), str(tmp_path / "regular.npz"))
    checked = _run(B.build(variant="bounds"), str(tmp_path / "bounds.npz"))
    assert regular.keys() == checked.keys()
    statuses = [k for k in checked if k.endswith(":status")]
    assert len(statuses) >= 20
    for k in statuses:
        assert int(checked[k]) == 0, f"{k}: device status {int(checked[k])}"
        assert int(regular[k]) == 0, k
    for k, v in regular.items():
        np.testing.assert_array_equal(checked[k], v, err_msg=k)
