"""The checked build: the kernels' bounds tests (PA_CHECKED) compiled in.

Its tests look at the indices the kernels take from device data (a gather's
parent slot, a replica's energy bin) and set the run's error flag instead of
an access outside an array.  On valid runs none may fire and the results must
be the plain build's: the smoke run against the oracle and the edge cases of
every row geometry and bit count run here on libpa_gb300_checked.so (selected
through PA_LIBRARY in a child process)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_gives_the_oracle_results():
    from paper_1704_01888_gb300 import build

    lib = build.build(checked=True)
    env = dict(os.environ, PA_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", "import __graft_entry__ as g; g.smoke()"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "smoke ok" in r.stdout, r.stdout + r.stderr
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_gpu_parity.py", "-q", "-x", "-m", "gpu",
                        "-k", "edge_cases or launch_shapes"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
