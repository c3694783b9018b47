"""Edge cases of the CUDA library: degenerate lattice sizes, a no-op step, and the largest
lattice of the benchmark family that one GPU holds.

* 1x1x1 (D3Q19) and 3x3x3 (D3Q39, the smallest its velocities allow) periodic lattices and odd
  sizes, against the oracle;
* the register pull's whole-chunk loads (D3Q39 and the reference-velocity forms) on rows of one
  to four chunks, where the periodic wrap of the neighbour chunks folds back onto the thread's
  own chunk or its nearest neighbour, for every cells-per-thread the width admits, against the
  oracle;
* n = 0 steps changes nothing;
* a uniform state (rho = 1, u = U everywhere) is left uniform by the collision and the
  streaming: every cell must hold the same stored values to the last bit, on D3Q19 1024^3 with
  FP16 storage (81.6 GB of distributions), with mass and momentum kept to the storage rounding.
"""
import numpy as np
import pytest

import oracle
from paper_2002_02503_gb300 import fields, lbm

from _lbmtest import TOL_F32, TOL_ROUND, oracle_reference, rel_f, rel_u, to_lib_order

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,K,dims", [("D3Q19", 3, (1, 1, 1)), ("D3Q19", 2, (5, 7, 9)), ("D3Q39", 4, (3, 3, 3)),
                                         ("D3Q39", 4, (7, 5, 3)), ("D2Q9", 3, (1, 1, 1)), ("D2Q9", 3, (3, 11, 1)),
                                         ("D3Q27", 3, (2, 3, 1)), ("D3Q15", 3, (9, 1, 5))])
def test_degenerate_and_odd_sizes(name, K, dims):
    D = lbm.lbm_lattice_info(name)["D"]
    rho, u = fields.random_fields(dims, D, salt=60)
    f_ref, r_ref, u_ref = oracle_reference(name, K, 0.6, dims, rho, u, 20)
    s = lbm.Solver(name, dims, 0.6, K, "f32")
    s.set_fields(rho, u)
    s.step(20)
    r, uu = s.moments()
    s.close()
    assert rel_f(r, r_ref) < TOL_F32
    assert rel_u(uu, u_ref) < TOL_F32


@pytest.mark.parametrize("name,K,storage,dims", [("D3Q39", 4, "f32", (4, 5, 3)), ("D3Q39", 4, "f32", (8, 3, 3)),
                                                 ("D3Q39", 3, "f16", (8, 4, 3)), ("D3Q19", 3, "f16r", (4, 3, 5)),
                                                 ("D3Q19", 2, "f16r", (2, 3, 3)), ("D3Q27", 3, "bf16r", (8, 3, 2))])
def test_whole_chunk_loads_on_short_rows(name, K, storage, dims):
    """Rows of nx / V = 1, 2 or 4 chunks: the neighbour chunks of the x shifts (up to 3 on D3Q39,
    two chunks away for two cells per thread) wrap onto the row's own chunks.  Each built
    cells-per-thread against the oracle after 10 steps (white-noise fields) and against one cell
    per thread (the direct shifted loads)."""
    D = lbm.lbm_lattice_info(name)["D"]
    rho, u = fields.random_fields(dims, D, salt=62)
    f_ref, r_ref, u_ref = oracle_reference(name, K, 0.6, dims, rho, u, 10)
    tol = TOL_F32 if storage == "f32" else TOL_ROUND[storage.rstrip("r")]
    results = {}
    for V in (1, 2, 4, 8):
        if dims[0] % V:
            continue
        s = lbm.Solver(name, dims, 0.6, K, storage)
        try:
            lbm.lbm_set_kernel(s.handle, 0, V, 128)
        except lbm.LbmError:  # not every cells-per-thread is built for every lattice and order
            s.close()
            continue
        s.set_fields(rho, u)
        s.step(10)
        r, uu = s.moments()
        results[V] = s.f()
        s.close()
        assert rel_u(uu, u_ref) < tol, (V, rel_u(uu, u_ref))
        assert rel_f(r, r_ref) < tol, V
    assert len(results) >= 2
    if storage == "f32":
        f_want = to_lib_order(name, f_ref)
        for V, f in results.items():
            assert rel_f(f, f_want) < TOL_F32, V
    for V, f in results.items():
        np.testing.assert_allclose(f, results[1], rtol=tol, atol=tol * np.abs(results[1]).max())


def test_zero_steps_is_a_no_op():
    dims = (16, 8, 4)
    rho, u = fields.random_fields(dims, 3, salt=61)
    s = lbm.Solver("D3Q19", dims, 0.6, 3, "f32")
    s.set_fields(rho, u)
    a = np.empty(s.raw_bytes(), dtype=np.uint8)
    lbm.lbm_get_distributions(s.handle, a)
    s.step(0)
    b = np.empty_like(a)
    assert lbm.lbm_get_distributions(s.handle, b) == 0
    np.testing.assert_array_equal(a, b)
    s.close()


def test_uniform_flow_stays_uniform_at_maximum_size():
    import torch

    dims = (1024, 1024, 1024)
    C = 1024 ** 3
    U = (0.05, -0.02, 0.01)
    rho = torch.ones(C, dtype=torch.float64, device="cuda")
    u = torch.empty((3, C), dtype=torch.float64, device="cuda")
    for a in range(3):
        u[a].fill_(U[a])
    s = lbm.Solver("D3Q19", dims, 0.55, 3, "f16")
    s.set_fields(rho, u)
    del rho, u
    torch.cuda.empty_cache()
    c0 = s.conservation()
    s.step(10)
    c1 = s.conservation()
    # FP16 storage rounds each stored value (|h| ~ 0.15, half an ulp ~ 6e-5): the sums agree to that
    np.testing.assert_allclose(c1[0], c0[0], rtol=2e-4)
    np.testing.assert_allclose(c1[1:], c0[1:], rtol=0, atol=2e-4 * c0[0])
    raw = torch.empty(s.raw_bytes(), dtype=torch.uint8, device="cuda")
    lbm.lbm_get_distributions(s.handle, raw)
    planes = raw.view(torch.int16).view(19, C)
    first = planes[:, :1]
    assert bool((planes == first).all())  # every cell holds the same 19 stored values
    s.close()
    del raw, planes
    torch.cuda.empty_cache()
    np.testing.assert_allclose(c1[1:] / c1[0], U, rtol=2e-3)
