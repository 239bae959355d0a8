"""The debug build (MF_DEBUG: device checks of indices and of the block data
structures' invariants, which record a failure and clamp instead of
faulting) on every path of the filter: each call agrees with the oracle and
no check fails; the self-test's deliberate failure reaches the host once and
is cleared by the read."""
import json
import os
import subprocess
import sys

import pytest

from paper_1406_1717_gb300 import build as mfbuild

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_all_paths_clean():
    mfbuild.build(debug=True)
    env = dict(os.environ, MF_DEBUG="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "debug_cases.py")],
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(res["cases"]) >= 20
    for c in res["cases"]:
        assert c["parity"], c
        assert c["failed_checks"] == 0, c
    assert res["selftest"] == [1, 999, 42]
    assert res["after_selftest"] == [0, 0, 0]
