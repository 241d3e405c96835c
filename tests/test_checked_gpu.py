"""The bounds-checked build (-DSPH_CHECK; built as libsph_gb300_check.so and
loaded with SPH_CHECKED=1): every neighbour range and mask-walk index is
tested against its buffer and a violation sets SPH_STATUS_BOUNDS.  Run over
every model's step, the adjoint, the batched form, the sampling operator and
the neighbour counts (checked_workloads.py) in a child process, it reports
no violation and reproduces the normal build's results bit for bit."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_08259_gb300 import build as B
    B.build()
    B.build(check=True)
    from paper_1710_08259_gb300 import sph
    return sph


def test_checked_build_finds_no_violation_and_matches(S, tmp_path):
    sys.path.insert(0, HERE)
    import checked_workloads as W
    ref = W.run()
    path = str(tmp_path / "checked.npz")
    env = dict(os.environ, SPH_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_workloads.py"), path], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    got = np.load(path)
    assert sorted(got.files) == sorted(ref)
    for k in ref:
        if k.endswith("/status"):
            assert int(got[k][0]) == 0 and int(ref[k][0]) == 0, (k, int(got[k][0]), int(ref[k][0]))
        else:
            np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
