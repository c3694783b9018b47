"""The staged step's bounded waits: when a stage's copies can never complete (a test hook
makes the producer expect bytes that are never sent), every wait gives up after its clock
budget (~1 s), the kernel records the expiry in the workspace's status word and returns, and
the next synchronous call reports LBM_ERR_TIMEOUT.  The context stays usable: the solver then
steps normally.  Runs in a child process so the hook's environment variable is read fresh."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import sys
    sys.path.insert(0, %r)
    import numpy as np
    from paper_2002_02503_gb300 import fields, lbm
    dims = (64, 16, 8)
    rho, u = fields.random_smooth_fields(dims, 3, salt=80)
    s = lbm.Solver("D3Q19", dims, 0.6, 3, "f32")
    s.set_fields(rho, u)
    lbm.lbm_set_kernel(s.handle, 1, 1, 256)
    s.step(1)
    try:
        s.conservation()
        print("NO-TIMEOUT")
    except lbm.LbmError as e:
        print("STATUS", e.status)
    lbm.lbm_set_kernel(s.handle, 0, 1, 256)
    s.set_fields(rho, u)
    s.step(5)
    c = s.conservation()
    print("AFTER", np.isfinite(c).all())
    s.close()
""") % ROOT


def test_staged_wait_expiry_is_reported_and_recoverable():
    env = dict(os.environ, LBM_TEST_STAGED_EXTRA_TX="16")
    r = subprocess.run([sys.executable, "-c", CHILD], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr
    assert "STATUS 6" in r.stdout, r.stdout  # LBM_ERR_TIMEOUT
    assert "AFTER True" in r.stdout, r.stdout
