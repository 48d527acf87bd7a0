"""The bounds-checked build (libcbp_checks.so: the library compiled with
-DCBP_CHECKS, where a failed index check on a kernel's main stores or
shared-memory staging sets a bit of its source file's check word and skips
the access) runs small cases of every kernel family with no failed check.
It runs in a child process, since a process loads one of the two builds."""
from __future__ import annotations

import json
import os
import subprocess
import sys
from pathlib import Path

import pytest

pytestmark = pytest.mark.gpu

ROOT = Path(__file__).resolve().parents[1]


def test_checked_build_finds_no_bad_index():
    env = dict(os.environ, CBP_LIBRARY="checks")
    r = subprocess.run([sys.executable, str(ROOT / "tests" / "_checks_run.py")], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["library"] == "libcbp_checks.so"
    assert len(out["words"]) == 6 and all(w == 0 for w in out["words"]), out["words"]
