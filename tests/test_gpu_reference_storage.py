"""The 16-bit storage forms with a per-cell reference velocity (LBM_STORE_F16_REF "f16r",
LBM_STORE_BF16_REF "bf16r") against the FP64 oracle.

Each cell stores, beside its Q values, a = u / T0 rounded to the 16-bit type, and each value
as the residual h_i - r_i, r_i = s + s^2 / 2 with s = c_i . a of the cell that wrote it; the
reader adds r_i back in FP32.
The method's arithmetic is unchanged (Eq. lbe, Eq. lbe-reg in FP32); only what is rounded
changes.  Checks: the stored reference and residuals after lbm_set_fields, parity with the
oracle on every lattice and truncation order, every kernel configuration, BGK and the
energy-flux term, checkpoints, determinism, the FP64 reductions, and the calls that do not
take these forms."""
import numpy as np
import pytest

import oracle
from paper_2002_02503_gb300 import fields, lbm

from _lbmtest import DIMS, TOL_ROUND, TOL_U16, oracle_reference, perm_lib_to_oracle, rel_f, rel_u, to_lib_order

pytestmark = pytest.mark.gpu

CASES = [("D2Q9", 2), ("D2Q9", 3), ("D3Q15", 3), ("D3Q19", 2), ("D3Q19", 3), ("D3Q27", 3), ("D3Q39", 4),
         ("D3Q39", 5)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    lbm.lib()
    yield
    torch.cuda.synchronize()


def _raw(s):
    raw = np.empty(s.raw_bytes(), dtype=np.uint8)
    t = lbm.lbm_get_distributions(s.handle, raw)
    return raw, t


def _planes(raw, storage, Q, D, C):
    """(distribution planes [Q, C], reference planes [D, C]) of a raw state, as float64."""
    if storage == "f16r":
        v = raw.view(np.float16).astype(np.float64)
    else:
        v = (raw.view(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    v = v.reshape(Q + D, C)
    return v[:Q], v[Q:]


@pytest.mark.parametrize("name", ["D2Q9", "D3Q19", "D3Q39"])
@pytest.mark.parametrize("storage", ["f16r", "bf16r"])
def test_set_fields_stores_reference_and_residuals(name, storage):
    """After lbm_set_fields: the reference planes hold u / T0 of each cell rounded to the 16-bit
    type (exactly), and residual plus r_i of the position reproduce the scaled equilibrium
    of the oracle (Eq. hermite) at the cell the value belongs to, within one rounding of the
    residual."""
    import torch

    info = lbm.lbm_lattice_info(name)
    Q, D, T0 = info["Q"], info["D"], info["T0"]
    dims = DIMS[name]
    C = int(np.prod(dims))
    K = info["kmax"]
    rho, u = fields.random_smooth_fields(dims, D, salt=41)
    s = lbm.Solver(name, dims, 0.7, K, storage)
    s.set_fields(rho, u)
    raw, t = _raw(s)
    s.close()
    assert t == 0
    d, a = _planes(raw, storage, Q, D, C)
    want_a = u.astype(np.float32) * np.float32(1.0 / T0)  # u / T0 as the kernel forms it, in FP32
    if storage == "f16r":
        np.testing.assert_array_equal(a, want_a.astype(np.float16).astype(np.float64))
    else:
        bf = torch.from_numpy(want_a).to(torch.bfloat16).float().double().numpy()
        np.testing.assert_array_equal(a, bf)
    # the oracle's f^eq at each cell, scaled and shifted, moved to the stored position x - c_i
    feq = to_lib_order(name, oracle.init_eq(name, K, dims, rho, u))
    nx, ny, nz = dims
    unit = 2.0 ** -11 if storage == "f16r" else 2.0 ** -8
    for i in range(Q):
        c = info["c"][i]
        h = (feq[i] - info["w"][i]) / info["w"][i]
        h_at = np.roll(h.reshape(nz, ny, nx), (-c[2], -c[1], -c[0]), axis=(0, 1, 2)).reshape(C)  # value at x - c
        sc = sum(c[k] * a[k] for k in range(D))
        shift = sc + 0.5 * sc * sc  # r_i = s + s^2 / 2
        resid = h_at - shift
        got = d[i] + shift
        # one rounding of the residual (relative, or FP16's subnormal spacing near 0) + FP32
        bound = unit * np.abs(resid) + (2.0 ** -25 if storage == "f16r" else 0.0) + 1e-6 * (np.abs(h_at) + 1e-3)
        assert np.all(np.abs(got - h_at) <= bound), (name, i, float(np.max(np.abs(got - h_at) - bound)))


@pytest.mark.parametrize("name,K", CASES)
def test_smooth_fields_match_oracle(name, K):
    dims = DIMS[name]
    D = lbm.lbm_lattice_info(name)["D"]
    rho, u = fields.random_smooth_fields(dims, D, config_index=0, salt=K)
    f_ref, r_ref, u_ref = oracle_reference(name, K, 0.55, dims, rho, u, 100)
    s = lbm.Solver(name, dims, 0.55, K, "f16r")
    s.set_fields(rho, u)
    s.step(100)
    r, uu = s.moments()
    f = s.f()
    s.close()
    eu, er, ef = rel_u(uu, u_ref), rel_f(r, r_ref), rel_f(f, to_lib_order(name, f_ref))
    print("%s K=%d f16r 100 steps: u %.2e rho %.2e f %.2e" % (name, K, eu, er, ef))
    assert eu < TOL_U16 and er < TOL_U16 and ef < TOL_U16


@pytest.mark.parametrize("storage", ["f16r", "bf16r"])
def test_every_kernel_configuration(storage):
    """Every cells-per-thread and block size of the register pull against the oracle (white
    noise, 10 steps, the 16-bit rounding bound) and against each other."""
    name, K = "D3Q19", 3
    dims = DIMS[name]
    rho, u = fields.random_fields(dims, 3, salt=42)
    f_ref, r_ref, u_ref = oracle_reference(name, K, 0.6, dims, rho, u, 10)
    results = []
    for V in (1, 2, 4, 8):
        if dims[0] % V:
            continue
        for block in (128, 256):
            s = lbm.Solver(name, dims, 0.6, K, storage)
            lbm.lbm_set_kernel(s.handle, 0, V, block)
            s.set_fields(rho, u)
            s.step(10)
            r, uu = s.moments()
            f = s.f()
            s.close()
            assert rel_u(uu, u_ref) < TOL_ROUND[storage[:-1]], (V, block)
            results.append(f)
    assert len(results) >= 4
    for f in results[1:]:
        np.testing.assert_allclose(f, results[0], rtol=TOL_ROUND[storage[:-1]])


def test_bgk_and_energy_flux_run_on_reference_storage():
    name, K = "D3Q39", 4
    dims = DIMS[name]
    rho, u = fields.random_smooth_fields(dims, 3, salt=43)
    f0 = oracle.init_eq(name, K, dims, rho, u)
    for model, theta in (("bgk", 0.0), ("filtered", 0.5)):
        f_ref = oracle.run(name, K, 0.7, dims, f0, 20, model=model, theta=theta)
        r_ref, u_ref = oracle.moments(name, dims, f_ref)
        s = lbm.Solver(name, dims, 0.7, K, "f16r")
        lbm.lbm_set_collision(s.handle, model)
        lbm.lbm_set_energy_flux(s.handle, theta)
        s.set_fields(rho, u)
        s.step(20)
        r, uu = s.moments()
        s.close()
        assert rel_u(uu, u_ref) < TOL_U16, model
        assert rel_f(r, r_ref) < TOL_U16, model


def test_checkpoint_round_trip_and_determinism():
    """The raw state (distribution and reference planes) restores bit for bit, and the same
    input gives the same stored bits."""
    name, K = "D3Q27", 3
    dims = DIMS[name]
    rho, u = fields.random_fields(dims, 3, salt=44)
    a = lbm.Solver(name, dims, 0.6, K, "f16r")
    a.set_fields(rho, u)
    a.step(7)
    raw, t = _raw(a)
    assert raw.size == (27 + 3) * int(np.prod(dims)) * 2 and t == 7
    a.step(9)
    final_a, _ = _raw(a)
    b = lbm.Solver(name, dims, 0.6, K, "f16r")
    lbm.lbm_set_distributions(b.handle, raw, t)
    b.step(9)
    final_b, tb = _raw(b)
    assert tb == 16
    np.testing.assert_array_equal(final_a, final_b)
    c = lbm.Solver(name, dims, 0.6, K, "f16r")
    c.set_fields(rho, u)
    c.step(16)
    final_c, _ = _raw(c)
    np.testing.assert_array_equal(final_a, final_c)
    for s in (a, b, c):
        s.close()


def test_reductions_match_pulled_moments():
    name, K = "D3Q19", 3
    dims = DIMS[name]
    rho, u = fields.random_fields(dims, 3, salt=45)
    s = lbm.Solver(name, dims, 0.6, K, "f16r")
    s.set_fields(rho, u)
    s.step(5)
    r, uu = s.moments()
    cons = s.conservation()
    np.testing.assert_allclose(cons[0], r.sum(), rtol=1e-12)
    np.testing.assert_allclose(cons[1:], (r * uu).sum(1), rtol=0, atol=1e-10 * r.sum())
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ph = 2 * np.pi * (x / nx).reshape(-1)
    want = np.sum(uu[1] * np.exp(-1j * ph))
    assert abs(s.mode((1, 0, 0), 1) - want) < 1e-10 * np.abs(uu[1]).sum()
    s.close()


def test_calls_that_do_not_take_the_reference_forms():
    import torch

    name, dims = "D3Q19", (32, 16, 8)
    s = lbm.Solver(name, dims, 0.6, 3, "f16r")
    for variant, V in ((1, 1), (2, 2)):  # staged and flat-pair variants
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_set_kernel(s.handle, variant, V, 128)
        assert e.value.status == lbm.LBM_ERR_UNSUPPORTED
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_set_storage_range(s.handle, 1.0)
    assert e.value.status == lbm.LBM_ERR_UNSUPPORTED
    s.close()
    raw = torch.zeros(22 * 32 * 16 * 8 * 2, dtype=torch.uint8, device="cuda")
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_conservation_noalloc(name, "f16r", dims, 1.0, raw, np.zeros(4))
    assert e.value.status == lbm.LBM_ERR_UNSUPPORTED
    with pytest.raises(lbm.LbmError) as e:
        lbm.Pool(name, 3, "f16r", arena_bytes=64 << 20, max_slots=4)
    assert e.value.status == lbm.LBM_ERR_UNSUPPORTED
