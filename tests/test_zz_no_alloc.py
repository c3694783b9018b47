"""lbm_conservation_noalloc: the allocation-free form of the mass/momentum sums.

Some callers cannot call cudaMalloc at all: a plugin whose host framework owns
every byte of device memory through its own pool, a process whose memory is
already reserved by another allocator, or a latency-critical loop where an
allocation (which may synchronise the device) is not allowed.  This entry point
serves them from a fixed scratch array inside the library.  The tests call it
through the C-ABI on a solver's stored distributions and compare it with the
existing lbm_conservation, twice in a row (the shared scratch keeps the previous
call's contents, which must not leak into the next result), at the largest
accepted number of z-planes, after a larger call on the same array, against the
oracle's own sums, and with the device's free memory unchanged by the calls."""
import ctypes

import numpy as np
import pytest

from paper_2002_02503_gb300 import fields, lbm

from _lbmtest import oracle_reference

pytestmark = pytest.mark.gpu

RTOL = 1e-12  # the conservation sums are FP64 on both paths; only the summation order differs


def _raw_on_device(s):
    import torch

    raw = torch.empty(s.raw_bytes(), dtype=torch.uint8, device="cuda")
    lbm.lbm_get_distributions(s.handle, raw)
    return raw


def _check_against_solver(name, storage, dims, s, raw):
    import torch

    want = s.conservation()
    out = np.zeros(4)
    lbm.lbm_conservation_noalloc(name, storage, dims, 1.0, raw, out)
    np.testing.assert_allclose(out[0], want[0], rtol=RTOL)
    np.testing.assert_allclose(out[1:], want[1:], rtol=0, atol=RTOL * want[0])
    out_dev = torch.zeros(4, dtype=torch.float64, device="cuda")
    lbm.lbm_conservation_noalloc(name, storage, dims, 1.0, raw, out_dev)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out_dev.cpu().numpy(), out)
    return out


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
        _check_against_solver(name, storage, dims, s, _raw_on_device(s))
    s.close()


def test_noalloc_largest_nz_then_smaller_nz():
    """nz = 4096 (the limit the scratch array is sized for), then a smaller nz on the same array:
    the second call reads only the planes it wrote itself."""
    import torch

    torch.cuda.set_device(0)
    results = []
    for dims in ((4, 3, 4096), (6, 5, 9)):
        rho, u = fields.random_smooth_fields(dims, 3, salt=22)
        s = lbm.Solver("D3Q19", dims, 0.7, 3, "f32")
        s.set_fields(rho, u)
        s.step(2)
        results.append(_check_against_solver("D3Q19", "f32", dims, s, _raw_on_device(s)))
        s.close()
    assert results[0][0] > results[1][0] * 100  # the first sum covered far more cells


def test_noalloc_sums_match_the_oracle():
    """Mass and momentum of the oracle's own run (Eq. mme summed over the lattice, FP64) against
    the allocation-free sums over the GPU's FP64 state after the same steps."""
    import torch

    torch.cuda.set_device(0)
    name, K, tau, dims = "D3Q19", 3, 0.6, (12, 10, 8)
    rho, u = fields.random_smooth_fields(dims, 3, salt=23)
    _, r_ref, u_ref = oracle_reference(name, K, tau, dims, rho, u, 5)
    want = np.concatenate([[r_ref.sum()], (r_ref * u_ref).sum(1)])
    s = lbm.Solver(name, dims, tau, K, "f64")
    s.set_fields(rho, u)
    s.step(5)
    out = np.zeros(4)
    lbm.lbm_conservation_noalloc(name, "f64", dims, 1.0, _raw_on_device(s), out)
    s.close()
    np.testing.assert_allclose(out[0], want[0], rtol=1e-12)
    np.testing.assert_allclose(out[1:], want[1:], rtol=0, atol=1e-12 * want[0])


def test_noalloc_allocates_nothing():
    """After one warm-up call (which commits the library's module on the device), repeated calls
    leave torch's allocator and the device's free memory unchanged."""
    import torch

    torch.cuda.set_device(0)
    dims = (16, 12, 10)
    rho, u = fields.random_smooth_fields(dims, 3, salt=24)
    s = lbm.Solver("D3Q19", dims, 0.6, 3, "f32")
    s.set_fields(rho, u)
    raw = _raw_on_device(s)
    out = np.zeros(4)
    lbm.lbm_conservation_noalloc("D3Q19", "f32", dims, 1.0, raw, out)
    torch.cuda.synchronize()
    cudart = ctypes.CDLL("libcudart.so.13") if _has("libcudart.so.13") else None
    free0 = _free_bytes(cudart)
    alloc0 = torch.cuda.memory_allocated()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(20):
        lbm.lbm_conservation_noalloc("D3Q19", "f32", dims, 1.0, raw, out)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.memory_reserved() == reserved0
    if free0 is not None:
        assert _free_bytes(cudart) == free0
    s.close()


def _has(soname):
    try:
        ctypes.CDLL(soname)
        return True
    except OSError:
        return False


def _free_bytes(cudart):
    if cudart is None:
        return None
    free, total = ctypes.c_size_t(), ctypes.c_size_t()
    if cudart.cudaMemGetInfo(ctypes.byref(free), ctypes.byref(total)) != 0:
        return None
    return free.value


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
