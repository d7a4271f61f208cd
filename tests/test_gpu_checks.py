"""The bounds-checked debug build (libcryptotrain_checks.so, -DHE_CHECKS):
every kernel access is checked against the device ranges a call may touch,
a violation is skipped (no trap) and reported by the entry point as
HE_ERR_INVALID_ARG.  The library is loaded in a child process
(CRYPTOTRAIN_LIB=checks) that runs tests/checks_child.py: a small layer equal
to the oracle with no violation, a store into memory left out of the ranges
reported and skipped, and normal results once the exclusion is cleared."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bounds_checked_build():
    sys.path.insert(0, ROOT)
    from paper_2409_16675_gb300 import build as b
    b.build_checks()  # already built by the package build; rebuilt only if stale
    env = dict(os.environ, CRYPTOTRAIN_LIB="checks")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checks_child.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "checks ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
