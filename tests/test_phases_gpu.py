"""The phase-timing build of the library (KNN_PHASE_TIMING): per-phase clock
totals of the round-loop kernel, read through knn_phase_clocks, in a process
of its own (a process loads one build of the library)."""

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_phase_shares_of_a_small_step():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--profile-step", "--phases", "--nq", "64", "--steps", "2",
           "--warmup", "3", "--B0", "8", "--B", "8", "--grow", "1", "--threads", "1024", "--c-alpha", "1e-3"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    sh = out["phase_clock_shares"]
    total = sum(sh["rounds"].values()) + sum(sh["round0"].values())
    assert abs(total - 1.0) < 1e-3 and out["phase_clocks_total"] > 0
    # every query runs round 0 and at least one later round: sampled gathers
    # and the round-0 filter (or round-0 sums) both take time
    assert sh["rounds"]["gather"] > 0 and sh["round0"]["gather"] > 0 and sh["rounds"]["output"] > 0
    assert "gather_phase_dram" not in out  # 64 queries: not the captured configuration
