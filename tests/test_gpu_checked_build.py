"""The self-checked build (-DPEOS_CHECKED) over a battery of every search variant: no
index or list-invariant check fires, and every result equals the normal build's."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from tests.checked_battery import battery

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    import paper_2402_11354_gb300 as P
    P.load()
    return P


def test_checked_build_finds_nothing_and_changes_nothing(P, tmp_path):
    from paper_2402_11354_gb300 import build as B
    lib = B.build(checked=True)
    path = str(tmp_path / "checked.npz")
    env = dict(os.environ, PEOS_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-m", "tests.checked_battery", path], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    report = json.loads(r.stdout.strip().splitlines()[-1])
    assert "self-checked" in report["version"]
    assert report["violations"] is not None and set(report["violations"].values()) == {0}, report
    assert P.check_read() is None  # this process runs the normal build
    mine = battery(P)
    got = np.load(path)
    assert set(got.files) == set(mine)
    for key in mine:
        assert np.array_equal(got[key].view(np.uint32), mine[key].view(np.uint32)), key
