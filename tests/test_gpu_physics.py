"""Full-size physics checks of the CUDA library against the oracle.

* Galilean invariance (shear wave u_y = 0.01 sin(2 pi x / 192) on a uniform background
  U_x in {0, 0.1, 0.2}, tau = 0.6, 2000 steps).  The field varies only in x, so a
  192 x 3 x 3 lattice is an exact stand-in for 192^3.
  - FP32, full 192^3 lattice (the configuration as stated): decay rates within 2e-3 of the
    oracle's -- the wave loses only ~7% over the fit window, and the stored values grow with
    the background speed (h ~ 3 c.U), so FP32 rounding of ~1e-7 in u shows up at 1e-4 to 1e-3
    in the rate -- and the Galilean error at the highest supported order far below the prior
    form's (K = 2).
  - FP64 storage, 192 x 3 x 3: decay rates within 1e-9 of the oracle's, which resolves the
    ordering |gamma(U)/gamma(0) - 1| falling with every added order K (Sec. 4: errors move to
    higher powers of the velocity), including D3Q39's K = 3 -> 4 step (~1e-4, below FP32
    resolution at this length).
* Precision of the storage forms (Taylor-Green u0 = 0.05, tau = 0.52, 500 steps, 64^3):
  FP32 within 1e-5 of the FP64 oracle on u, 16-bit fixed point (range 1/4) within 3e-4, the
  reference-velocity forms within 2e-4 (FP16) and 1e-3 (BF16).  Plain shifted FP16 sits near
  1e-3 and does not meet it reliably: its error is the accumulated half-precision rounding of
  the stored values, a different realisation for every grouping of the FP32 collision
  arithmetic (8.9e-4 and 1.15e-3 measured with two groupings; a CPU model of the same step
  gives 7.6e-4 with exact arithmetic and 1.12e-3 to 1.21e-3 in three realisations with
  FP32-sized noise before each rounding).
  It is recorded as missing the bound, with a regression ceiling; BF16 (8-bit significand)
  misses 1e-3 and is reported the same way.
"""
import numpy as np
import pytest

import oracle
from paper_2002_02503_gb300 import fields, lbm

from _lbmtest import TOL_F32, TOL_U16, rel_f, rel_u

pytestmark = pytest.mark.gpu

N = 192
T_FIT = (100, 2000)


def _gpu_rate(name, K, U, storage="f32", ny=N):
    dims = (N, ny, ny)
    rho, u = fields.shear_wave(dims, 0.01, 3, 1, 0, background=(U, 0.0, 0.0))
    s = lbm.Solver(name, dims, 0.6, K, storage)
    s.set_fields(rho, u)
    del rho, u
    if ny == N:
        lbm.lbm_autotune(s.handle, 3)
    s.step(T_FIT[0])
    a0 = abs(s.mode((1, 0, 0), 1))
    s.step(T_FIT[1] - T_FIT[0])
    a1 = abs(s.mode((1, 0, 0), 1))
    s.close()
    return -np.log(a1 / a0) / (T_FIT[1] - T_FIT[0])


_ORACLE = {}


def _oracle_rate(name, K, U):
    key = (name, K, U)
    if key in _ORACLE:
        return _ORACLE[key]
    dims = (N, 3, 3)
    rho, u = fields.shear_wave(dims, 0.01, 3, 1, 0, background=(U, 0.0, 0.0))
    f = oracle.init_eq(name, K, dims, rho, u)
    x = np.arange(N)
    amps = []
    for steps in (T_FIT[0], T_FIT[1] - T_FIT[0]):
        f = oracle.run(name, K, 0.6, dims, f, steps)
        _, uu = oracle.moments(name, dims, f)
        uy = uu[1].reshape(3, 3, N).mean(axis=(0, 1))
        amps.append(abs(np.sum(uy * np.exp(-2j * np.pi * x / N))))
    _ORACLE[key] = -np.log(amps[1] / amps[0]) / (T_FIT[1] - T_FIT[0])
    return _ORACLE[key]


@pytest.mark.parametrize("name,Ks", [("D3Q27", [2, 3]), ("D3Q39", [2, 3, 4])])
def test_galilean_invariance_fp32_full_size(name, Ks):
    err = {}
    for K in Ks:
        g = {U: _gpu_rate(name, K, U) for U in (0.0, 0.1, 0.2)}
        for U in (0.0, 0.2):
            ref = _oracle_rate(name, K, U)
            assert abs(g[U] / ref - 1) < 2e-3, (name, K, U, g[U], ref)
        err[K] = [abs(g[U] / g[0.0] - 1) for U in (0.1, 0.2)]
        print("FP32 192^3 %s K=%d gamma(0)=%.6e |gamma(U)/gamma(0)-1| U=0.1: %.3e U=0.2: %.3e" % (
            name, K, g[0.0], err[K][0], err[K][1]))
    assert err[Ks[-1]][1] < 0.05 * err[Ks[0]][1], err
    nu = lbm.lbm_lattice_info(name)["T0"] * (0.6 - 0.5)
    k = 2 * np.pi / N
    assert abs(g[0.0] / (nu * k * k) - 1) < 0.01


@pytest.mark.parametrize("name,Ks", [("D3Q27", [2, 3]), ("D3Q39", [2, 3, 4, 5])])
def test_galilean_invariance_ordering_fp64(name, Ks):
    err = {}
    for K in Ks:
        g = {U: _gpu_rate(name, K, U, storage="f64", ny=3) for U in (0.0, 0.1, 0.2)}
        if K <= 4:
            for U in (0.0, 0.1, 0.2):
                ref = _oracle_rate(name, K, U)
                assert abs(g[U] / ref - 1) < 1e-9, (name, K, U, g[U], ref)
        err[K] = [abs(g[U] / g[0.0] - 1) for U in (0.1, 0.2)]
        print("FP64 %s K=%d gamma(0)=%.9e |gamma(U)/gamma(0)-1| U=0.1: %.3e U=0.2: %.3e" % (
            name, K, g[0.0], err[K][0], err[K][1]))
    for lo, hi in zip(Ks[:-1], Ks[1:]):
        if hi == 5:
            continue  # K = 5 is reported, not ordered: the paper prints forms up to K = 4
        assert err[hi][0] < err[lo][0] and err[hi][1] < err[lo][1], err


@pytest.fixture(scope="module")
def taylor_green_reference():
    dims = (64, 64, 64)
    rho, u = fields.taylor_green_3d(dims, 0.05, 1.0 / 3.0)
    f = oracle.run("D3Q19", 2, 0.52, dims, oracle.init_eq("D3Q19", 2, dims, rho, u), 500)
    r_ref, u_ref = oracle.moments("D3Q19", dims, f)
    return dims, rho, u, r_ref, u_ref


_ERRORS = {}


def _storage_error(taylor_green_reference, storage):
    if storage in _ERRORS:
        return _ERRORS[storage]
    dims, rho, u, r_ref, u_ref = taylor_green_reference
    s = lbm.Solver("D3Q19", dims, 0.52, 2, storage, storage_range=0.25 if storage == "q16" else None)
    s.set_fields(rho, u)
    s.step(500)
    r, uu = s.moments()
    s.close()
    eu, er = rel_u(uu, u_ref), rel_f(r, r_ref)
    print("D3Q19 64^3 Taylor-Green tau=0.52 K=2, %s storage, 500 steps: rel u error %.3e, rel rho error %.3e" % (
        storage, eu, er))
    _ERRORS[storage] = eu
    return eu


@pytest.mark.parametrize("storage,tol", [("f32", TOL_F32), ("q16", 3e-4), ("f16r", 2e-4), ("bf16r", TOL_U16)])
def test_storage_precision_taylor_green_500_steps(taylor_green_reference, storage, tol):
    """Error of each storage form after 500 steps against the FP64 oracle on 64^3 (the 16-bit
    workload, tau = 0.52, at a size the oracle finishes in seconds; the stated sizes are checked
    in test_gpu_storage_accuracy.py, where plain FP16 misses the target).  The fixed-point form
    runs with range 1/4 (|h| reaches about 0.16 in this flow)."""
    assert _storage_error(taylor_green_reference, storage) < tol


@pytest.mark.xfail(strict=False, reason="plain FP16 storage does not reliably meet 1e-3 on u at 64^3 "
                                        "(measured 8.9e-4 and 1.15e-3 with two groupings of the FP32 collision)")
def test_f16_storage_meets_u_bound_at_64(taylor_green_reference):
    """The 16-bit target (1e-3 on u) for plain FP16 storage at 64^3: near the bound, on either side
    of it depending on the rounding realisation, so recorded as not met (not strict)."""
    assert _storage_error(taylor_green_reference, "f16") < TOL_U16


def test_f16_storage_error_regression_at_64(taylor_green_reference):
    """FP16's error at 64^3 (8.9e-4 and 1.15e-3 measured) must not grow past 1.5e-3."""
    assert _storage_error(taylor_green_reference, "f16") < 1.5e-3


@pytest.mark.xfail(strict=True, reason="BF16 storage misses the 1e-3 bound on u already at 64^3 (measured 4.9e-2)")
def test_bf16_storage_meets_u_bound_at_64(taylor_green_reference):
    """The 16-bit target (1e-3 on u) for BF16 storage: recorded as failing -- an 8-bit significand
    rounds the momentum-carrying values at ~4e-4 each step."""
    assert _storage_error(taylor_green_reference, "bf16") < TOL_U16


def test_bf16_storage_error_regression_at_64(taylor_green_reference):
    """BF16's measured miss at 64^3 (4.9e-2) must not grow."""
    assert _storage_error(taylor_green_reference, "bf16") < 1.25 * 4.9e-2
