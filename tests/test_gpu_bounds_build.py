"""The bounds-check build (liblbm_gb300_bounds.so, compiled with LBM_DEBUG_BOUNDS): every
kernel checks each load and store index against the buffer or velocity plane it addresses,
skips an access outside it and records the event, and the next synchronising call returns
LBM_ERR_BOUNDS.  compute-sanitizer is closed on this machine; this build stands in for its
out-of-bounds check.

The test builds that library (minutes, on the first run) and runs, in a child process that
loads it, the odd-size and degenerate lattices, every kernel configuration and variant
(register pull at every cells per thread, staged bulk copies, flat pairs), the storage forms,
the reductions and pools: any index outside its buffer fails them with LBM_ERR_BOUNDS."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [
    "tests/test_gpu_edges.py::test_degenerate_and_odd_sizes",
    "tests/test_gpu_edges.py::test_zero_steps_is_a_no_op",
    "tests/test_gpu_edges.py::test_whole_chunk_loads_on_short_rows",
    "tests/test_gpu_parity.py::test_every_kernel_configuration",
    "tests/test_gpu_parity.py::test_staged_variant_matches_oracle",
    "tests/test_gpu_parity.py::test_flat_pair_variant_on_odd_lattices",
    "tests/test_gpu_parity.py::test_conservation_and_mode_reductions_match_fields",
    "tests/test_gpu_parity.py::test_energy_flux_term_matches_oracle",
    "tests/test_gpu_parity.py::test_bgk_comparison_mode_matches_oracle",
    "tests/test_gpu_fixed_point.py::test_every_cells_per_thread_agrees",
    "tests/test_gpu_reference_storage.py::test_every_kernel_configuration",
    "tests/test_gpu_reference_storage.py::test_reductions_match_pulled_moments",
    "tests/test_gpu_pool.py::test_result_same_alone_and_in_mix",
    "tests/test_gpu_pool.py::test_pool_matches_oracle_on_small_odd_lattice",
    "tests/test_gpu_pool.py::test_cells_per_thread_of_the_batched_step",
]


@pytest.fixture(scope="module")
def bounds_env():
    from paper_2002_02503_gb300 import build

    build.build(bounds_check=True)
    return dict(os.environ, LBM_BOUNDS_CHECK="1")


def test_child_process_loads_the_bounds_check_build(bounds_env):
    code = "from paper_2002_02503_gb300 import lbm; import sys; sys.exit(0 if lbm.lbm_bounds_checked() else 3)"
    r = subprocess.run([sys.executable, "-c", code], env=bounds_env, cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr


def test_kernels_stay_inside_their_buffers(bounds_env):
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider"] + CASES,
                       env=bounds_env, cwd=ROOT, capture_output=True, text=True, timeout=3000)
    tail = (r.stdout + r.stderr)[-4000:]
    print(tail)
    assert r.returncode == 0, tail
    assert "LBM_ERR_BOUNDS" not in r.stdout
