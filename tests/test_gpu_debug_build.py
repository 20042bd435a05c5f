"""The PLQ_DEBUG build: device bounds guards (an out-of-range index is recorded as
PLQ_ERR_BOUNDS in the context's status word and redirected inside the buffer, so a
guard that fires shows as a status instead of a fault) in the hopping kernels (every
launch kind), the row-streamed kernel and the persistent batched CG.  As a stand-in
for a device memory checker, the battery in debug_battery.py runs those kernels on
ragged lattices through the debug library in a child process and requires correct
results with a clean status word after every launch."""
import json
import os
import subprocess
import sys

import pytest

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_debug_build_runs_clean():
    from paper_1405_0700_gb300 import _build

    lib = _build.build(debug=True)
    env = dict(os.environ, PLQ_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_battery.py")], env=env, capture_output=True,
                       text=True, timeout=1200)
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert lines, r.stdout[-2000:] + r.stderr[-4000:]
    rep = json.loads(lines[-1])
    assert rep["library"].endswith("libplq_debug.so")
    assert rep["checks"] >= 60 and not rep["failures"], rep
    assert r.returncode == 0
