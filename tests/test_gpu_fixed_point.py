"""The 16-bit fixed-point storage form (LBM_STORE_Q16) through the C-ABI.

h = q 2^e with q in [-32768, 32767] stored as q + 2^15 and the range R = 2^(e + 15) a power
of two.  Checked here: the decoder is exact (integer codes in, FP64 values out, compared
bit for bit), the encoder rounds to nearest with ties to even, a value beyond the range is
reported as LBM_ERR_RANGE (a state whose next step leaves the range, as the oracle's own step
shows) while the same state in a wider range is not, and results match the FP64 oracle; the same
for pools of the fixed-point form."""
import numpy as np
import pytest

import oracle
from paper_2002_02503_gb300 import fields, lbm

from _lbmtest import DIMS, TOL_U16, oracle_reference, perm_lib_to_oracle, rel_f, rel_u, to_lib_order

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    lbm.lib()
    yield
    torch.cuda.synchronize()


def _pull(info, dims, stored):
    """Pre-collision f_i(x) = g_i(x - c_i) of stored planes g (library order)."""
    nx, ny, nz = dims
    out = np.empty_like(stored)
    for i in range(info["Q"]):
        cx, cy, cz = info["c"][i]
        out[i] = np.roll(stored[i].reshape(nz, ny, nx), (cz, cy, cx), axis=(0, 1, 2)).reshape(-1)
    return out


@pytest.mark.parametrize("R", [2.0 ** -8, 0.25, 1.0, 2.0 ** 8])
def test_decode_is_exact(R):
    name, dims = "D3Q19", (20, 9, 7)
    info = lbm.lbm_lattice_info(name)
    C = int(np.prod(dims))
    g = np.random.default_rng(31).integers(0, 65536, size=(info["Q"], C), dtype=np.uint16)
    g[:, 0], g[:, 1] = 0, 65535  # both ends of the code range
    s = lbm.Solver(name, dims, 0.6, 3, "q16", rho0=1.0, storage_range=R)
    lbm.lbm_set_distributions(s.handle, g, 0)
    f = s.f()
    s.close()
    step = R / 32768.0
    h = (g.astype(np.float64) - 32768.0) * step  # exact: |q| < 2^15 and step a power of two
    w = info["w"][:, None]
    want = _pull(info, dims, w * h + w * 1.0)  # the library's FP64 decode: w h + w rho0
    np.testing.assert_array_equal(f, want)


def test_encode_rounds_to_nearest_even():
    """At u = 0 the truncated equilibrium is h_i = rho - rho0 exactly, so rho - rho0 = (k + frac) 2^e
    must store code 2^15 + round_half_even(k + frac) for every velocity."""
    name, dims, R = "D3Q19", (16, 8, 6), 1.0
    info = lbm.lbm_lattice_info(name)
    C = int(np.prod(dims))
    step = R / 32768.0
    rg = np.random.default_rng(32)
    k = rg.integers(-30000, 30000, size=C).astype(np.float64)
    frac = rg.choice([0.0, 0.25, 0.5, 0.75, -0.5], size=C)
    k[:2], frac[:2] = (-32768.0, 32767.0), 0.0  # both ends of the range are representable
    q = k + frac
    rho = 1.0 + q * step
    u = np.zeros((3, C))
    s = lbm.Solver(name, dims, 0.6, 3, "q16", storage_range=R)
    s.set_fields(rho, u)
    raw = np.empty(info["Q"] * C, dtype=np.uint16)
    lbm.lbm_get_distributions(s.handle, raw)
    s.close()
    code = 32768 + np.rint(q)  # numpy rounds halves to even
    nx, ny, nz = dims
    want = np.empty((info["Q"], C))
    for i in range(info["Q"]):  # stored g_i(y) = f_i(y + c_i)
        cx, cy, cz = info["c"][i]
        want[i] = np.roll(code.reshape(nz, ny, nx), (-cz, -cy, -cx), axis=(0, 1, 2)).reshape(-1)
    np.testing.assert_array_equal(raw.reshape(info["Q"], C).astype(np.float64), want)


def _implosion(info, dims, R, code):
    """Every moving velocity carries h = code 2^e toward one cell x0; everything else is h = 0."""
    nx, ny, nz = dims
    C = nx * ny * nz
    stored = np.full((info["Q"], C), 32768, dtype=np.uint16)
    x0 = (3, 4, 5)
    for i in range(1, info["Q"]):
        c = info["c"][i]
        x, y, z = ((x0[0] - c[0]) % nx, (x0[1] - c[1]) % ny, (x0[2] - c[2]) % nz)
        stored[i, x + nx * (y + ny * z)] = 32768 + code
    return stored, x0[0] + nx * (x0[1] + ny * x0[2])


def test_value_beyond_the_range_is_reported():
    name, dims, K, tau = "D3Q19", (8, 8, 8), 3, 0.55
    info = lbm.lbm_lattice_info(name)
    R = 0.25
    stored, cell = _implosion(info, dims, R, 32767)  # h = R (1 - 2^-15) on the incoming links
    h0 = (stored.astype(np.float64) - 32768) * (R / 32768)
    # the oracle's step of the same state: the rest population of x0 leaves the range
    w = info["w"][:, None]
    f0 = _pull(info, dims, w * h0 + w)
    f0o = np.empty_like(f0)
    f0o[perm_lib_to_oracle(name)] = f0
    f1 = to_lib_order(name, oracle.run(name, K, tau, dims, f0o, 1))
    h_rest = (f1[0, cell] - info["w"][0]) / info["w"][0]
    assert h_rest > R, h_rest

    s = lbm.Solver(name, dims, tau, K, "q16", storage_range=R)
    lbm.lbm_set_distributions(s.handle, stored, 0)
    s.step(1)
    with pytest.raises(lbm.LbmError) as e:
        s.moments()
    assert e.value.status == lbm.LBM_ERR_RANGE
    s.close()

    # the same physical state in twice the range: no report, and the step matches the oracle
    stored2, _ = _implosion(info, dims, 2 * R, 16384)
    s = lbm.Solver(name, dims, tau, K, "q16", storage_range=2 * R)
    lbm.lbm_set_distributions(s.handle, stored2, 0)
    s.step(1)
    f = s.f()
    s.close()
    assert np.max(np.abs(f - f1) / np.abs(f1)) < 2 * R / 32768


def test_set_fields_beyond_the_range_is_reported():
    dims = (16, 16, 16)
    rho, u = fields.taylor_green_3d(dims, 0.05, 1.0 / 3.0)  # |h| up to about 0.16
    s = lbm.Solver("D3Q19", dims, 0.6, 3, "q16", storage_range=2.0 ** -4)
    with pytest.raises(lbm.LbmError) as e:
        s.set_fields(rho, u)
    assert e.value.status == lbm.LBM_ERR_RANGE
    lbm.lbm_set_storage_range(s.handle, 0.25)
    s.set_fields(rho, u)  # fits now
    s.close()
    # the range is [-R, R): at u = 0, h = rho - rho0 for every velocity
    s = lbm.Solver("D3Q19", dims, 0.6, 3, "q16", storage_range=0.25)
    C = 16 ** 3
    zero = np.zeros((3, C))
    s.set_fields(np.full(C, 1.0 - 0.25), zero)
    s.set_fields(np.full(C, 1.0 + 0.25 * (1 - 2.0 ** -15)), zero)
    with pytest.raises(lbm.LbmError) as e:
        s.set_fields(np.full(C, 1.0 + 0.25), zero)
    assert e.value.status == lbm.LBM_ERR_RANGE
    s.close()


def test_range_must_be_a_power_of_two_and_floating_forms_have_none():
    s = lbm.Solver("D3Q19", DIMS["D3Q19"], 0.6, 3, "q16")
    for bad in (0.3, -1.0, 2.0 ** -9, 2.0 ** 9, float("nan")):  # (0 selects the automatic range)
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_set_storage_range(s.handle, bad)
        assert e.value.status == lbm.LBM_ERR_INVALID_ARG
    s.close()
    s = lbm.Solver("D3Q19", DIMS["D3Q19"], 0.6, 3, "f16")
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_set_storage_range(s.handle, 1.0)
    assert e.value.status == lbm.LBM_ERR_UNSUPPORTED
    s.close()


CASES = [("D2Q9", 3), ("D3Q15", 3), ("D3Q19", 2), ("D3Q19", 3), ("D3Q27", 3), ("D3Q39", 4), ("D3Q39", 5)]


@pytest.mark.parametrize("name,K", CASES)
def test_smooth_fields_match_oracle(name, K):
    """Smooth seeded fields (u0 = 0.05), 100 steps, range 1/2: within the 16-bit bound on u."""
    dims = DIMS[name]
    D = lbm.lbm_lattice_info(name)["D"]
    rho, u = fields.random_smooth_fields(dims, D, config_index=0, salt=K)
    f_ref, r_ref, u_ref = oracle_reference(name, K, 0.55, dims, rho, u, 100)
    s = lbm.Solver(name, dims, 0.55, K, "q16", storage_range=0.5)
    s.set_fields(rho, u)
    s.step(100)
    r, uu = s.moments()
    f = s.f()
    s.close()
    eu = rel_u(uu, u_ref)
    print("%s K=%d q16 rel u %.3e rel f %.3e" % (name, K, eu, rel_f(f, to_lib_order(name, f_ref))))
    assert eu < TOL_U16
    assert rel_f(f, to_lib_order(name, f_ref)) < TOL_U16


@pytest.mark.parametrize("V", [2, 4, 8])
def test_every_cells_per_thread_agrees(V):
    """The register-pull variants differ in how they load and in how the FP32 arithmetic is
    issued (V >= 2 runs two cells per pass on the paired FP32 instructions, which round some
    sums differently).  A one-step difference in a code then spreads through the neighbours, so
    each run carries its own rounding noise of the size of the fixed-point error itself: both
    stay within the 16-bit bound of the FP64 oracle, and no code differs by more than a few
    grid steps."""
    name, K, dims, tau, steps = "D3Q19", 3, (64, 20, 12), 0.6, 40
    rho, u = fields.random_smooth_fields(dims, 3, config_index=0, salt=41)
    _, r_ref, u_ref = oracle_reference(name, K, tau, dims, rho, u, steps)
    raws = []
    for v in (1, V):
        s = lbm.Solver(name, dims, tau, K, "q16", storage_range=0.5)
        lbm.lbm_set_kernel(s.handle, 0, v, 128)
        s.set_fields(rho, u)
        s.step(steps)
        raw = np.empty(s.raw_bytes() // 2, dtype=np.uint16)
        lbm.lbm_get_distributions(s.handle, raw)
        raws.append(raw)
        r, uu = s.moments()
        s.close()
        assert rel_u(uu, u_ref) < TOL_U16, v
        assert rel_f(r, r_ref) < TOL_U16, v
    assert np.max(np.abs(raws[0].astype(np.int64) - raws[1].astype(np.int64))) <= 16


@pytest.mark.parametrize("name,K,V", [("D3Q19", 2, 4), ("D3Q39", 4, 2)])
@pytest.mark.parametrize("shift", [False, True])
def test_register_capped_configurations_match_oracle(name, K, V, shift):
    """The fixed-point steps that run under a register cap (D3Q19 K = 2 with four cells per
    thread, D3Q39 K = 4 with two), forced, without and with a reference shift: within the
    16-bit bound of the FP64 oracle after 100 steps."""
    dims = DIMS[name]
    D = lbm.lbm_lattice_info(name)["D"]
    rho, u = fields.random_smooth_fields(dims, D, config_index=0, salt=53 + K)
    f_ref, r_ref, u_ref = oracle_reference(name, K, 0.55, dims, rho, u, 100)
    s = lbm.Solver(name, dims, 0.55, K, "q16", storage_range=0.5,
                   storage_reference=(0.02, -0.01, 0.01) if shift else None)
    lbm.lbm_set_kernel(s.handle, 0, V, 128)
    assert lbm.lbm_get_kernel(s.handle) == (0, V, 128)
    s.set_fields(rho, u)
    s.step(100)
    r, uu = s.moments()
    f = s.f()
    s.close()
    eu = rel_u(uu, u_ref)
    print("%s K=%d V=%d shift=%s q16 rel u %.3e" % (name, K, V, shift, eu))
    assert eu < TOL_U16
    assert rel_f(f, to_lib_order(name, f_ref)) < TOL_U16


def test_bgk_and_energy_flux_run_on_fixed_point():
    name, K, dims = "D3Q19", 3, DIMS["D3Q19"]
    rho, u = fields.random_smooth_fields(dims, 3, config_index=0, salt=42)
    for model, theta in (("bgk", 0.0), ("filtered", 0.7)):
        _, r_ref, u_ref = oracle_reference_model(name, K, 0.6, dims, rho, u, 50, model, theta)
        s = lbm.Solver(name, dims, 0.6, K, "q16", storage_range=0.5)
        lbm.lbm_set_collision(s.handle, model)
        lbm.lbm_set_energy_flux(s.handle, theta)
        s.set_fields(rho, u)
        s.step(50)
        r, uu = s.moments()
        s.close()
        assert rel_u(uu, u_ref) < TOL_U16, model


def oracle_reference_model(name, K, tau, dims, rho, u, steps, model, theta):
    f0 = oracle.init_eq(name, K, dims, rho, u)
    f = oracle.run(name, K, tau, dims, f0, steps, model=model, theta=theta)
    r, uu = oracle.moments(name, dims, f)
    return f, r, uu


def _converging_pair(n, a):
    """u_x = +a at x = 3 and -a at x = 4, rest at rho = 1: at tau = 0.51 max|h| grows from 0.238 to
    0.258 at the third step for a = 0.074 (the oracle's own run), across the range 1/4."""
    C = n ** 3
    x = np.arange(C) % n
    u = np.zeros((3, C))
    u[0] = a * np.where(x == 3, 1.0, np.where(x == 4, -1.0, 0.0))
    return np.ones(C), u


def test_dynamic_range_exit_is_reported_by_the_solver():
    rho, u = _converging_pair(8, 0.074)
    f = oracle.init_eq("D3Q19", 2, (8, 8, 8), rho, u)
    w = oracle.lattice("D3Q19")["w"][:, None]
    hmax = [np.abs((f - w) / w).max()]
    for _ in range(3):
        f = oracle.run("D3Q19", 2, 0.51, (8, 8, 8), f, 1)
        hmax.append(np.abs((f - w) / w).max())
    assert hmax[0] < 0.25 * 0.97 and hmax[3] > 0.25 * 1.02, hmax
    s = lbm.Solver("D3Q19", (8, 8, 8), 0.51, 2, "q16", storage_range=0.25)
    s.set_fields(rho, u)  # fits at t = 0
    s.step(3)
    with pytest.raises(lbm.LbmError) as e:
        s.moments()
    assert e.value.status == lbm.LBM_ERR_RANGE
    s.close()


def test_pool_fixed_point():
    """A fixed-point pool: results match the single-lattice fixed-point solver and the oracle within
    the 16-bit bound, a request's result is the same alone and in a mix, and a request that leaves
    the range is reported on its own result while the others are unaffected."""
    def run(reqs, R=0.25):
        pool = lbm.Pool("D3Q19", 2, "q16", 1 << 30, 16, storage_range=R)
        ids = [pool.submit(d, tau, rho, u, n) for d, tau, rho, u, n in reqs]
        assert all(i is not None for i in ids)
        while not all(pool.poll(i)[0] for i in ids):
            pool.advance(7)
            pool.sync()
        out = []
        for (d, _, _, _, _), i in zip(reqs, ids):
            try:
                out.append(pool.result(i, int(np.prod(d))))
            except lbm.LbmError as e:
                out.append(e.status)
        pool.close()
        return out

    good = []
    for side, u0 in ((24, 0.04), (27, 0.03)):
        d = (side,) * 3
        rho, u = fields.taylor_green_3d(d, u0, 1.0 / 3.0)
        good.append((d, 0.6, rho, u, 40))
    rho_b, u_b = _converging_pair(8, 0.074)
    bad = ((8, 8, 8), 0.51, rho_b, u_b, 10)
    mixed = run([good[0], bad, good[1]])
    assert mixed[1] == lbm.LBM_ERR_RANGE
    alone = run([good[0]])
    np.testing.assert_array_equal(alone[0][1], mixed[0][1])
    for k, (d, tau, rho, u, n) in zip((0, 2), good):
        _, r_ref, u_ref = oracle_reference("D3Q19", 2, tau, d, rho, u, n)
        assert rel_u(mixed[k][1], u_ref) < TOL_U16
        assert rel_f(mixed[k][0], r_ref) < TOL_U16
        s = lbm.Solver("D3Q19", d, tau, 2, "q16", storage_range=0.25)
        s.set_fields(rho, u)
        s.step(n)
        r1, u1 = s.moments()
        s.close()
        assert rel_u(mixed[k][1], u1) < TOL_U16
    # in twice the range the same request runs through
    wide = run([bad], R=0.5)
    assert not isinstance(wide[0], int)
    # f^eq beyond the range is refused at admission; the pool's range changes only when empty
    pool = lbm.Pool("D3Q19", 2, "q16", 1 << 28, 4, storage_range=2.0 ** -4)
    d = (16, 16, 16)
    rho, u = fields.taylor_green_3d(d, 0.05, 1.0 / 3.0)
    with pytest.raises(lbm.LbmError) as e:
        pool.submit(d, 0.6, rho, u, 5)
    assert e.value.status == lbm.LBM_ERR_RANGE
    assert pool.stats()["resident"] == 0
    lbm.lbm_pool_set_storage_range(pool.handle, 0.25)
    rid = pool.submit(d, 0.6, rho, u, 5)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_pool_set_storage_range(pool.handle, 0.5)
    assert e.value.status == lbm.LBM_ERR_BUSY
    while not pool.poll(rid)[0]:
        pool.advance(5)
        pool.sync()
    pool.result(rid, 16 ** 3)
    pool.close()


def test_checkpoint_round_trip_in_fixed_point():
    """A fixed-point checkpoint restores bit for bit into a solver with the same range (the codes
    carry no range of their own), and the ranges read back as set."""
    name, K, dims = "D3Q27", 3, DIMS["D3Q27"]
    rho, u = fields.random_smooth_fields(dims, 3, salt=12)
    a = lbm.Solver(name, dims, 0.6, K, "q16", storage_range=0.5)
    assert lbm.lbm_get_storage_range(a.handle) == 0.5
    a.set_fields(rho, u)
    a.step(10)
    raw = np.empty(a.raw_bytes(), dtype=np.uint8)
    t = lbm.lbm_get_distributions(a.handle, raw)
    a.step(10)
    fa = np.empty_like(raw)
    lbm.lbm_get_distributions(a.handle, fa)
    b = lbm.Solver(name, dims, 0.6, K, "q16", storage_range=0.5)
    lbm.lbm_set_distributions(b.handle, raw, t)
    b.step(10)
    fb = np.empty_like(raw)
    assert lbm.lbm_get_distributions(b.handle, fb) == 20
    np.testing.assert_array_equal(fa, fb)
    a.close()
    b.close()
    pool = lbm.Pool("D3Q19", 2, "q16", 1 << 24, 4, storage_range=2.0 ** -3)
    assert lbm.lbm_pool_get_storage_range(pool.handle) == 0.125
    pool.close()


def test_range_report_belongs_to_the_state_it_came_from():
    """A range exit is reported once, by the next synchronising call (a checkpoint read included);
    replacing the state (set_fields, set_distributions) starts with a clean record."""
    rho_b, u_b = _converging_pair(8, 0.074)
    s = lbm.Solver("D3Q19", (8, 8, 8), 0.51, 2, "q16", storage_range=0.25)
    s.set_fields(rho_b, u_b)
    s.step(3)  # leaves the range
    raw = np.empty(s.raw_bytes(), dtype=np.uint8)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_get_distributions(s.handle, raw)
    assert e.value.status == lbm.LBM_ERR_RANGE
    s.step(3)  # leaves it again (garbage in, flagged out)
    rho, u = fields.taylor_green_3d((8, 8, 8), 0.02, 1.0 / 3.0)
    s.set_fields(rho, u)  # a new state: the pending report is dropped, not blamed on it
    s.step(2)
    s.moments()
    good = np.empty_like(raw)
    lbm.lbm_get_distributions(s.handle, good)
    s.set_fields(rho_b, u_b)
    s.step(3)
    lbm.lbm_set_distributions(s.handle, good, 2)  # restoring a valid checkpoint also starts clean
    s.step(1)
    s.moments()
    s.close()


@pytest.mark.parametrize("u0,want", [(0.05, 0.25), (0.005, 2.0 ** -5)])
def test_automatic_range(u0, want):
    """Range 0 = automatic: set_fields measures max|h| of f^eq and takes the smallest power of two
    R >= 1.25 max|h|; the run then matches the oracle within the 16-bit bound."""
    name, K, dims = "D3Q19", 3, (32, 24, 16)
    rho, u = fields.taylor_green_3d(dims, u0, 1.0 / 3.0)
    # the largest |h| of the truncated equilibrium, from the oracle (h = (f - w rho0) / w)
    f0 = oracle.init_eq(name, K, dims, rho, u)
    w = oracle.lattice(name)["w"][:, None]
    hmax = np.abs((f0 - w) / w).max()
    assert want / 2 < 1.25 * hmax <= want
    s = lbm.Solver(name, dims, 0.6, K, "q16", storage_range=0.0)
    s.set_fields(rho, u)
    assert lbm.lbm_get_storage_range(s.handle) == want
    s.step(40)
    r, uu = s.moments()
    _, r_ref, u_ref = oracle_reference(name, K, 0.6, dims, rho, u, 40)
    assert rel_u(uu, u_ref) < TOL_U16
    lbm.lbm_set_storage_range(s.handle, 1.0)  # an explicit range turns the automatic choice off
    s.set_fields(rho, u)
    assert lbm.lbm_get_storage_range(s.handle) == 1.0
    s.close()


def test_pool_automatic_range_per_request():
    """A fixed-point pool with range 0 gives each request the smallest power of two >= 1.25 max|h|
    of its own f^eq; results match the oracle within the 16-bit bound."""
    pool = lbm.Pool("D3Q19", 2, "q16", 1 << 28, 8, storage_range=0.0)
    assert lbm.lbm_pool_get_storage_range(pool.handle) == 0.0
    reqs = []
    for side, u0, want in ((20, 0.05, 0.25), (17, 0.005, 2.0 ** -5)):
        d = (side,) * 3
        rho, u = fields.taylor_green_3d(d, u0, 1.0 / 3.0)
        rid = pool.submit(d, 0.6, rho, u, 30)
        assert lbm.lbm_pool_request_range(pool.handle, rid) == want
        reqs.append((d, rho, u, rid))
    while not all(pool.poll(r[3])[0] for r in reqs):
        pool.advance(10)
        pool.sync()
    for d, rho, u, rid in reqs:
        rr, uu = pool.result(rid, int(np.prod(d)))
        _, r_ref, u_ref = oracle_reference("D3Q19", 2, 0.6, d, rho, u, 30)
        assert rel_u(uu, u_ref) < TOL_U16
    pool.close()


def _href(info, U, rho0=1.0):
    """The reference shift of lbm_set_storage_reference, written from its header statement."""
    c = info["c"].astype(np.float64)
    s = c @ np.asarray(U, dtype=np.float64) / info["T0"]
    v2 = float(np.dot(U, U)) / info["T0"]
    return rho0 * (s + 0.5 * (s * s - v2))


def test_decode_with_reference_shift_is_exact():
    name, dims, R, U = "D3Q27", (12, 7, 5), 0.125, (0.1, -0.05, 0.02)
    info = lbm.lbm_lattice_info(name)
    C = int(np.prod(dims))
    g = np.random.default_rng(33).integers(0, 65536, size=(info["Q"], C), dtype=np.uint16)
    s = lbm.Solver(name, dims, 0.6, 3, "q16", storage_range=R, storage_reference=U)
    lbm.lbm_set_distributions(s.handle, g, 0)
    f = s.f()
    s.close()
    step = R / 32768.0
    k = np.rint(_href(info, U) / step)  # the shift in whole grid steps
    h = (g.astype(np.float64) - 32768.0 + k[:, None]) * step
    w = info["w"][:, None]
    # h decodes exactly; w h + w rho0 may round once (fused) or twice, hence the few ulp --
    # far below the one-step (~1e-6) error a wrong shift would make
    np.testing.assert_allclose(f, _pull(info, dims, w * h + w * 1.0), rtol=4e-16, atol=0)


def _decoded(name, dims, R, U, g):
    s = lbm.Solver(name, dims, 0.6, 3, "q16", storage_range=R)
    if U is not None:
        lbm.lbm_set_storage_reference(s.handle, U)
    lbm.lbm_set_distributions(s.handle, g, 0)
    f = s.f()
    s.close()
    return f


def test_reference_shift_arguments():
    """Invalid references are refused and leave the solver's shift as it was; the floating forms
    have no shift; on D2Q9 the third component is ignored."""
    name, dims, R = "D3Q19", (12, 7, 5), 0.25
    info = lbm.lbm_lattice_info(name)
    g = np.full((info["Q"], int(np.prod(dims))), 32768, dtype=np.uint16)  # h = 0 before the shift
    s = lbm.Solver(name, dims, 0.6, 3, "q16", storage_range=R, storage_reference=(0.1, 0.0, 0.0))
    for bad in ((0.6, 0.0, 0.0), (float("nan"), 0.0, 0.0), (0.0, float("inf"), 0.0), (0.3, 0.3, 0.3)):
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_set_storage_reference(s.handle, bad)
        assert e.value.status == lbm.LBM_ERR_INVALID_ARG, bad
    lbm.lbm_set_distributions(s.handle, g, 0)
    f_after = s.f()
    s.close()
    np.testing.assert_array_equal(f_after, _decoded(name, dims, R, (0.1, 0.0, 0.0), g))
    assert not np.array_equal(f_after, _decoded(name, dims, R, None, g))  # the shift is still on
    s = lbm.Solver(name, dims, 0.6, 3, "f16")
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_set_storage_reference(s.handle, (0.1, 0.0, 0.0))
    assert e.value.status == lbm.LBM_ERR_UNSUPPORTED
    s.close()
    d2 = (16, 10, 1)
    g2 = np.random.default_rng(5).integers(0, 65536, size=(9, 160), dtype=np.uint16)
    np.testing.assert_array_equal(_decoded("D2Q9", d2, R, (0.1, 0.05, 0.4), g2),
                                  _decoded("D2Q9", d2, R, (0.1, 0.05, 0.0), g2))


@pytest.mark.parametrize("name,K", [("D3Q27", 3), ("D3Q39", 4)])
def test_reference_shift_on_a_background_flow(name, K):
    """A shear wave (0.01) on U_x = 0.1: with the storage shifted by the equilibrium at U, the
    automatic range shrinks and the fixed-point run stays within the 16-bit bound of the oracle,
    where without the shift it does not."""
    dims, steps = (48, 6, 6), 300
    info = lbm.lbm_lattice_info(name)
    rho, u = fields.shear_wave(dims, 0.01, 3, 1, 0, background=(0.1, 0.0, 0.0))
    _, r_ref, u_ref = oracle_reference(name, K, 0.6, dims, rho, u, steps)
    errs, ranges = {}, {}
    for ref in (None, (0.1, 0.0, 0.0)):
        s = lbm.Solver(name, dims, 0.6, K, "q16", storage_range=0.0, storage_reference=ref)
        s.set_fields(rho, u)
        ranges[ref is not None] = lbm.lbm_get_storage_range(s.handle)
        s.step(steps)
        r, uu = s.moments()
        s.close()
        errs[ref is not None] = rel_u(uu[1], u_ref[1])  # the decaying wave component
    print(name, K, "ranges", ranges, "rel u_y", errs)
    assert ranges[True] <= ranges[False] / 4
    assert errs[True] < TOL_U16
    assert errs[True] < errs[False] / 2
