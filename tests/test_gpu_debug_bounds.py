"""The bounds-checking debug library (a stand-in for a memory checker): every
kernel family runs once through it, from small plans to the 4M-point
clustered plane at N = 2048 in both precisions, and no kernel computes a
shared- or global-memory index or a TMA coordinate outside the extent of the
buffer it addresses (the library skips and counts such accesses instead of
making them)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_no_kernel_access_leaves_its_buffer():
    from paper_1308_6644_gb300 import _build
    lib = _build.build_debug()
    env = dict(os.environ, NUASM_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "debug_bounds_run.py")], env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    records = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(records) >= 25
    bad = [rec for rec in records if rec["hits"] != 0]
    assert not bad, bad
