"""The C-ABI from plain C: tests/c_client/lbm_c_client.c (no Python, no PyTorch; it owns its
device workspace and stream) compiles against include/lbm.h with gcc, and on a GPU its output
equals the Python path's for the same solve."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2002_02503_gb300 import fields, lbm

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "c_client", "lbm_c_client.c")
CUDA = "/usr/local/cuda"


def _compile(out, link):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    cmd = [gcc, "-std=c99", "-O2", "-Wall", "-Wextra", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(CUDA, "include"), SRC]
    if link:
        pkg = os.path.dirname(lbm.LIB_PATH)
        cmd += ["-o", out, "-L", pkg, "-llbm_gb300", "-L", os.path.join(CUDA, "lib64"), "-lcudart", "-lm",
                "-Wl,-rpath," + pkg, "-Wl,-rpath," + os.path.join(CUDA, "lib64")]
    else:
        cmd += ["-c", "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert "warning" not in r.stderr, r.stderr


def test_c_client_compiles_as_c99(tmp_path):
    _compile(str(tmp_path / "client.o"), link=False)


@pytest.mark.gpu
def test_c_client_matches_python_path(tmp_path):
    lbm.lib()
    exe = str(tmp_path / "client")
    _compile(exe, link=True)
    n, steps = 24, 50
    r = subprocess.run([exe, str(n), str(steps)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = dict((ln.split()[0] + (ln.split()[1] if ln.startswith("cell") else ""), ln.split()) for ln in
                 r.stdout.splitlines())
    assert int(lines["t"][1]) == steps
    s = lbm.Solver("D3Q19", (n,) * 3, 0.6, 3, "f32")
    rho, u = fields.taylor_green_3d((n,) * 3, 0.05, 1.0 / 3.0)
    s.set_fields(rho, u)
    s.step(steps)
    cons = s.conservation()
    r_py, u_py = s.moments()
    s.close()
    got = np.array([float(v) for v in lines["conservation"][1:]])
    # the two clients evaluate the same analytic fields (libm and numpy may differ in the last
    # bit of a double), so the comparison is at the FP32 storage's level
    np.testing.assert_allclose(got[0], cons[0], rtol=1e-9)
    np.testing.assert_allclose(got[1:], cons[1:], rtol=0, atol=1e-7 * cons[0])
    C = n ** 3
    for c in (0, C // 3 + 5, C - 1):
        vals = np.array([float(v) for v in lines["cell" + str(c)][2:]])
        np.testing.assert_allclose(vals[0], r_py[c], rtol=1e-6)
        np.testing.assert_allclose(vals[1:], u_py[:, c], rtol=0, atol=1e-7)
