"""The check build (libfss_check.so, FSS_CHECK_BOUNDS=1): device-side index
checks on the data-dependent indices of every kernel, and 256-byte canaries
after every workspace region, reported through fss_read_status as
FSS_ERR_BOUNDS without any fault.  tests/check_bounds_probe.py runs in a
process of its own (the library is chosen when the binding loads it): a
clean frame reports FSS_OK, and each planted corruption of the index data is
refused by its check and named.  The rest of the GPU suite can be run on the
check build with FSS_CHECK_BOUNDS=1 in the environment.
"""
import json
import os
import subprocess
import sys

import pytest

from paper_2604_10951_gb300 import _lib as L
from paper_2604_10951_gb300.build import LIB_CHECK

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_check_build_refuses_and_reports_corrupt_indices():
    assert os.path.exists(LIB_CHECK), "the check build is compiled by build()"
    env = dict(os.environ, FSS_CHECK_BOUNDS="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "check_bounds_probe.py")], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["clean"] == [L.FSS_OK, ""] and out["clean_after"] == [L.FSS_OK, ""], out
    expect = {"range": "tile range", "item": "pair-list item", "position": "saved list position",
              "canary": "pair list"}
    for case, words in expect.items():
        status, msg = out[case]
        assert status == L.FSS_ERR_BOUNDS, (case, out[case])
        assert words in msg, (case, msg)
