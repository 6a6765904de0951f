"""The check build (libwrs_check.so, WRS_CHECK=1) on the parity shapes of
every builder: each bucket stored exactly once, no failed index or
end-of-subproblem check, tables equal to the oracle's.  The cases run in a
child process because the binding loads one library per process."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_check_build_every_bucket_once_and_no_failed_check():
    env = dict(os.environ, WRS_CHECK="1")
    r = subprocess.run([sys.executable, "-m", "tests._check_run"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=1200)
    print(r.stdout[-4000:])
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "check build: all cases passed" in r.stdout
