"""The debug build of the library (-DLRU_DEBUG): the same kernels with
device-side checks of work-item indices (a failed check records a sticky
error and skips the work, never traps) and guard zones after every region of
a handle's allocation that lru_check_device_error verifies.  Small chains run
through it in a child process against the oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_chains_match_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_05255_gb300 import _build
    _build.build(debug=True)
    env = dict(os.environ, LRUGB_DEBUG="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "debug_chain.py")], capture_output=True,
                         text=True, timeout=900, env=env, cwd=ROOT)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "debug chains ok" in out.stdout and "debug" in out.stdout
