"""The timeout path of the row passes' bounded bulk-copy waits, made to run
out without a fault: in the checked build the barriers expect 16 bytes more
than their copies deliver (cbp_check_expire_waits), every copy lands, no
phase completes, each wait expires and the kernel leaves.  Every pair then
reports CBP_ERR_TIMEOUT, and the same calls with the waits restored give the
results they gave before (the context stays usable).  Generic and
in-register row passes; in a child process (the checked build)."""
from __future__ import annotations

import json
import os
import subprocess
import sys
from pathlib import Path

import pytest

pytestmark = pytest.mark.gpu

ROOT = Path(__file__).resolve().parents[1]


def test_expired_copy_waits_report_timeout():
    env = dict(os.environ, CBP_LIBRARY="checks")
    r = subprocess.run([sys.executable, str(ROOT / "tests" / "_timeout_run.py")], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert all(s == 0 for st in out["before"] for s in st), out["before"]
    assert all(s == out["timeout_status"] for st in out["expired"] for s in st), out["expired"]
    assert all(s == 0 for st in out["after"] for s in st), out["after"]
    assert out["same_after"]
