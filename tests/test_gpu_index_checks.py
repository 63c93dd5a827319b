"""The index-checked build (libtga_check.so) on small parity cases (marked gpu).

This build stands in for a device memory checker: every indexed access of
the search state and the instance is checked against its array's extent,
and a failed check is recorded instead of touching memory outside the
array.  A child process (tests/index_check_cases.py, TGA_INDEX_CHECKS=1)
runs stepwise, whole-descent (persistent, graph and host-launched), pickup,
swaps-of-runs, edge-based and batched cases against the oracle and asserts
that no check failed.
"""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_cases_pass_every_index_check():
    from paper_2506_17357_gb300 import build
    build.build()                                   # both libraries (no-op when up to date)
    env = dict(os.environ, TGA_INDEX_CHECKS="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "index_check_cases.py")], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["ok"] and len(line["cases"]) >= 20, line
    print(json.dumps(line))


def test_release_build_reports_no_checks():
    """The release library answers the report call and says it has no checks."""
    from paper_2506_17357_gb300 import instances as I
    from paper_2506_17357_gb300 import tga as T
    assert os.path.basename(T.LIB_PATH) == "libtga.so"
    inst = I.cvrp_uniform(20, 1)
    ls = T.LocalSearch(inst, I.random_split_solution(inst, 2), I.MASK_ALL).build()
    try:
        assert T.tga_get_bounds_report(ls.ctx) == {"checked": False, "site": 0, "index": 0, "limit": 0}
    finally:
        ls.close()
