"""GPU: the debug build (device-side index checks, -DMFA_DEBUG; the stand-in for a memory
sanitizer) raises no flag over a spread of valid workloads of every kernel family, and the
release build reports itself as such."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_debug_build_raises_no_index_flag():
    from paper_2312_15073_gb300 import build
    lib = build.build(debug=True)
    env = dict(os.environ, MFA_LIB=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_workload.py")], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    status = json.loads(r.stdout.strip().splitlines()[-1])
    assert status == {"debug_build": True, "flags": 0, "count": 0}, status


def test_release_build_reports_no_checks():
    from paper_2312_15073_gb300 import build
    build.build()
    import paper_2312_15073_gb300 as mfa
    if os.environ.get("MFA_LIB"):
        pytest.skip("MFA_LIB selects another library")
    assert mfa.debug_status() == {"debug_build": False, "flags": 0, "count": 0}
