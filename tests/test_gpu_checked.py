"""The range-checked build (LB_CHECKED) in a process of its own: valid inputs give the
oracle's results with no check firing, and a planted out-of-range column is recorded as
LB_ERR_OUT_OF_RANGE by every kernel that gathers by column (see tests/checked_cases.py)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_range_checked_build():
    env = dict(os.environ, LBSPMV_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_cases.py")], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, f"{r.stdout[-2000:]}\n{r.stderr[-4000:]}"
    assert "checked build" in r.stdout
