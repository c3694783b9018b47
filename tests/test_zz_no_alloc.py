"""lbm_conservation_noalloc: the allocation-free form of the mass/momentum sums.

Some callers cannot call cudaMalloc at all: a plugin whose host framework owns
every byte of device memory through its own pool, a process whose memory is
already reserved by another allocator, or a latency-critical loop where an
allocation (which may synchronise the device) is not allowed.  This entry point
serves them from a fixed scratch array inside the library.  The test calls it
through the C-ABI on a solver's stored distributions and compares it with the
existing lbm_conservation, twice in a row (the shared scratch keeps the previous
call's contents, which must not leak into the next result)."""
import ctypes

import numpy as np
import pytest

from paper_2002_02503_gb300 import fields, lbm

pytestmark = pytest.mark.gpu

RTOL = 1e-12  # the conservation sums are FP64 on both paths; only the summation order differs


def _raw_on_device(s):
    import torch

    raw = torch.empty(s.raw_bytes(), dtype=torch.uint8, device="cuda")
    lbm.lbm_get_distributions(s.handle, raw)
    return raw


@pytest.mark.parametrize("name,storage,dims", [("D3Q19", "f32", (40, 26, 14)), ("D3Q39", "f16", (28, 18, 10)),
                                               ("D2Q9", "f64", (72, 44, 1))])
def test_noalloc_matches_conservation_twice(name, storage, dims):
    import torch

    torch.cuda.set_device(0)
    D = lbm.lbm_lattice_info(name)["D"]
    kmax = lbm.lbm_lattice_info(name)["kmax"]
    rho, u = fields.random_smooth_fields(dims, D, salt=21)
    s = lbm.Solver(name, dims, 0.6, kmax, storage)
    s.set_fields(rho, u)
    for steps in (3, 7):  # two calls in a row, on different states
        s.step(steps)
        want = s.conservation()
        raw = _raw_on_device(s)
        out = np.zeros(4)
        lbm.lbm_conservation_noalloc(name, storage, dims, 1.0, raw, out)
        np.testing.assert_allclose(out[0], want[0], rtol=RTOL)
        np.testing.assert_allclose(out[1:], want[1:], rtol=0, atol=RTOL * want[0])
        out_dev = torch.zeros(4, dtype=torch.float64, device="cuda")
        lbm.lbm_conservation_noalloc(name, storage, dims, 1.0, raw, out_dev)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out_dev.cpu().numpy(), out)
    s.close()


def test_noalloc_rejects_too_many_planes():
    import torch

    raw = torch.zeros(19 * 4 * 8, dtype=torch.uint8, device="cuda")
    out = np.zeros(4)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_conservation_noalloc("D3Q19", "f32", (1, 1, 4097), 1.0, raw, out)
    assert e.value.status == lbm.LBM_ERR_INVALID_ARG
    assert b"4096" in lbm.lib().lbm_last_error()
    d = (ctypes.c_int64 * 3)(1, 1, 4)
    assert lbm.lib().lbm_conservation_noalloc(1, 0, d, 1.0, None, None, 0, None) == lbm.LBM_ERR_INVALID_ARG
