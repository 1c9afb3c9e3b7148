"""The checked build on the GPU: kernels that verify every index they use
(libddm_checked.so, DDM_CHECKED) run the one-shot, staged, chunked,
compressed, batched and refit paths without finding an index out of bounds,
and give the oracle's pairs.  It stands in for the sanitizers, which are not
available here.  Run in a child process, so that it loads only the checked
library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_runs_clean():
    sys.path.insert(0, ROOT)
    import __graft_entry__
    __graft_entry__.build()
    env = dict(os.environ, DDM_LIBRARY="checked")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_workload.py")],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked build ok" in r.stdout
