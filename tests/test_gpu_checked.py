"""The bounds-checked build (compute-sanitizer's stand-in on this pool): every
index the kernels compute stays in range over render, residual, adjustment,
backward, the reconstruction loop with its variants, the hull, batches and
the server.  Runs tests/checked_workload.py in a child process with
FR_LIBRARY_VARIANT=checked and requires an all-zero check word."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_checked_build_records_no_out_of_range_index():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    here = os.path.dirname(os.path.abspath(__file__))
    env = dict(os.environ, FR_LIBRARY_VARIANT="checked")
    r = subprocess.run([sys.executable, os.path.join(here, "checked_workload.py")], capture_output=True, text=True,
                       env=env, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    print(out)
    assert out["checks_enabled"] == 1
    assert all(w == 0 for w in out["words"].values()), out
