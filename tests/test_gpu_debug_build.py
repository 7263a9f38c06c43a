"""The NRR_DEBUG build (address checks in every load and store of the
stencil, boundary and residual kernels; no memory checker runs where this
library runs) on a workload that reaches every such kernel: no access falls
outside the library's allocations, and the final states equal the release
build's bit for bit (the checks change no arithmetic)."""
from __future__ import annotations

import json
import os
import subprocess
import sys

import pytest

from paper_2501_14030_gb300 import nrr

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.slow
def test_debug_build_refuses_no_access_and_matches_release(gpu):
    from paper_2501_14030_gb300 import build
    from tests import debug_workload
    build.build(debug=True)  # a few minutes: the checks multiply the code
    env = dict(os.environ, NRR_DEBUG="1")
    r = subprocess.run([sys.executable, "-m", "tests.debug_workload"], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stderr[-3000:]
    dbg = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert dbg["check"]["enabled"], "the subprocess did not load the debug build"
    assert dbg["check"]["refused"] == 0, dbg["check"]
    assert dbg["check"]["first_bad"] == 0
    rel = debug_workload.run()
    assert not rel["check"]["enabled"]
    assert len(rel["digests"]) >= 40
    assert rel["digests"] == dbg["digests"]
