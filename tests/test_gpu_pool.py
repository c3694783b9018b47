"""Batched multi-lattice step and the continuous-batching pool (through the C-ABI).

Each request's result must not depend on what else is resident: the same request run
alone and in a mix gives identical results, both match the single-lattice solver within
the FP32 tolerance, and small cases match the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2002_02503_gb300 import fields, lbm, serve

from _lbmtest import TOL_F32, TOL_ROUND, rel_f, rel_u

pytestmark = pytest.mark.gpu


def _tg(side, u0):
    return fields.taylor_green_3d((side,) * 3, u0, 1.0 / 3.0)


def _run_pool(reqs, chunk=7, arena=2 << 30, submit_after=None, kernel=None):
    """reqs: list of (side, tau, u0, steps).  submit_after[k] = chunk index at which request k joins.
    kernel: (cells per thread, block) of the batched step, or None for the default."""
    pool = lbm.Pool("D3Q19", 3, "f32", arena, 64)
    if kernel is not None:
        lbm.lbm_pool_set_kernel(pool.handle, *kernel)
    submit_after = submit_after or [0] * len(reqs)
    ids = {}
    out = {}
    c = 0
    while len(out) < len(reqs):
        for k, (side, tau, u0, steps) in enumerate(reqs):
            if k not in ids and submit_after[k] <= c:
                rho, u = _tg(side, u0)
                rid = pool.submit((side,) * 3, tau, rho, u, steps)
                assert rid is not None
                ids[k] = rid
        pool.advance(chunk)
        c += 1
        pool.sync()
        for k, rid in ids.items():
            if k in out:
                continue
            done, sd = pool.poll(rid)
            if done:
                out[k] = pool.result(rid, reqs[k][0] ** 3)
        assert c < 10000
    pool.close()
    return out


def _single(side, tau, u0, steps):
    s = lbm.Solver("D3Q19", (side,) * 3, tau, 3, "f32")
    rho, u = _tg(side, u0)
    s.set_fields(rho, u)
    s.step(steps)
    r = s.moments()
    s.close()
    return r


def test_result_same_alone_and_in_mix():
    target = (33, 0.7, 0.05, 40)
    alone = _run_pool([target])[0]
    mix = [(20, 0.9, 0.03, 13), target, (47, 0.55, 0.08, 61), (12, 0.6, 0.02, 5), (64, 0.52, 0.07, 29)]
    joined = [0, 2, 0, 1, 3]  # the target joins while others run; some leave before it ends
    res = _run_pool(mix, submit_after=joined)
    np.testing.assert_array_equal(res[1][0], alone[0])
    np.testing.assert_array_equal(res[1][1], alone[1])
    r1, u1 = _single(*target)
    assert rel_f(alone[0], r1) < TOL_F32
    assert rel_u(alone[1], u1) < TOL_F32
    for k, req in enumerate(mix):  # every other member matches its own single-lattice run
        r, u = _single(*req)
        assert rel_f(res[k][0], r) < TOL_F32
        assert rel_u(res[k][1], u) < TOL_F32


def test_pool_matches_oracle_on_small_odd_lattice():
    side, tau, u0, steps = 13, 0.6, 0.05, 30
    res = _run_pool([(side, tau, u0, steps), (17, 0.8, 0.03, 11)], chunk=4)[0]
    rho, u = _tg(side, u0)
    d = (side,) * 3
    f = oracle.run("D3Q19", 3, tau, d, oracle.init_eq("D3Q19", 3, d, rho, u), steps)
    r_ref, u_ref = oracle.moments("D3Q19", d, f)
    assert rel_f(res[0], r_ref) < TOL_F32
    assert rel_u(res[1], u_ref) < TOL_F32


def test_admission_by_memory_and_zero_steps():
    side = 32
    per = lbm.lbm_pool_request_bytes("D3Q19", (side,) * 3, "f32")
    pool = lbm.Pool("D3Q19", 3, "f32", 2 * per + (1 << 20), 64)
    rho, u = _tg(side, 0.05)
    a = pool.submit((side,) * 3, 0.7, rho, u, 5)
    b = pool.submit((side,) * 3, 0.7, rho, u, 0)
    assert a is not None and b is not None
    assert pool.submit((side,) * 3, 0.7, rho, u, 5) is None  # arena full: BUSY
    done, _ = pool.poll(b)
    assert done
    r0, u0 = pool.result(b, side ** 3)
    np.testing.assert_allclose(u0, u, rtol=0, atol=1e-7)  # zero steps: moments of f^eq(rho, u)
    c = pool.submit((side,) * 3, 0.7, rho, u, 5)  # room again
    assert c is not None
    while not (pool.poll(a)[0] and pool.poll(c)[0]):
        pool.advance(3)
        pool.sync()
    pool.result(a, side ** 3)
    pool.result(c, side ** 3)
    assert pool.stats()["resident"] == 0
    pool.close()


def test_pool_autotune_keeps_results():
    """Tuning launches write only the idle buffers: after autotuning, the results equal bit for bit
    those of a pool set to the configuration the tuner chose."""
    reqs = [(24, 0.7, 0.05, 20), (31, 0.6, 0.04, 20)]
    pool = lbm.Pool("D3Q19", 3, "f32", 1 << 30, 64)
    ids = []
    for side, tau, u0, steps in reqs:
        rho, u = _tg(side, u0)
        ids.append(pool.submit((side,) * 3, tau, rho, u, steps))
    us = lbm.lbm_pool_autotune(pool.handle, 2)
    assert us > 0
    chosen = lbm.lbm_pool_get_kernel(pool.handle)
    assert chosen[0] in (1, 2, 4) and chosen[1] in (128, 256)
    base = _run_pool(reqs, kernel=chosen)
    while not all(pool.poll(i)[0] for i in ids):
        pool.advance(7)
        pool.sync()
    for k, i in enumerate(ids):
        r, u = pool.result(i, reqs[k][0] ** 3)
        np.testing.assert_array_equal(u, base[k][1])
    pool.close()


def test_served_results_same_as_alone():
    """A short Poisson trace through the continuous-batching server: sampled results equal the
    same requests run alone on the single-lattice path, within the FP32 tolerance."""
    trace = serve.make_trace(24, rate=400.0, salt=3, side=(16, 48), steps=(20, 120))
    keep = {0, 5, 11, 23}
    stats, res = serve.serve_pool(trace, chunk=16, arena_bytes=4 << 30, keep=keep)
    assert stats["solves"] == 24
    for i in keep:
        r = trace[i]
        rr, uu = _single(r["side"], r["tau"], r["u0"], r["steps"])
        assert rel_f(res[i][0], rr) < TOL_F32
        assert rel_u(res[i][1], uu) < TOL_F32
    plain, pres = serve.serve_plain(trace, keep=keep)
    assert plain["solves"] == 24
    for i in keep:
        np.testing.assert_allclose(pres[i][1], res[i][1], rtol=0, atol=TOL_F32 * np.abs(res[i][1]).max())


@pytest.mark.parametrize("lattice,K,storage,sides", [("D3Q19", 3, "f16", [20, 33]), ("D3Q39", 4, "f32", [9, 14]),
                                                     ("D3Q27", 2, "bf16", [12, 17])])
def test_pool_other_classes_match_single_lattice(lattice, K, storage, sides):
    """Pools of other (lattice, K, storage) classes against the single-lattice solver."""
    T0 = lbm.lbm_lattice_info(lattice)["T0"]
    pool = lbm.Pool(lattice, K, storage, 1 << 30, 16)
    ids = []
    for side in sides:
        rho, u = fields.taylor_green_3d((side,) * 3, 0.05, T0)
        ids.append(pool.submit((side,) * 3, 0.65, rho, u, 25))
    while not all(pool.poll(i)[0] for i in ids):
        pool.advance(10)
        pool.sync()
    tol = {"f32": TOL_F32, **TOL_ROUND}[storage]  # a one-ulp flip of a 16-bit value
    for side, rid in zip(sides, ids):
        r, u = pool.result(rid, side ** 3)
        s = lbm.Solver(lattice, (side,) * 3, 0.65, K, storage)
        rho0, u0 = fields.taylor_green_3d((side,) * 3, 0.05, T0)
        s.set_fields(rho0, u0)
        s.step(25)
        rs, us = s.moments()
        s.close()
        assert rel_f(r, rs) < tol
        assert rel_u(u, us) < tol
    pool.close()


def test_cells_per_thread_of_the_batched_step():
    """Two and four x-neighbours per thread (every nx: the pool pads rows to a multiple of 4 with
    periodic images) against one cell per thread: the same fields within the FP32 tolerance, and
    a request's result does not depend on the residents."""
    reqs = [(24, 0.7, 0.05, 30), (25, 0.6, 0.04, 30), (40, 0.55, 0.06, 17), (7, 0.65, 0.03, 21)]
    one = _run_pool(reqs, kernel=(1, 256))
    for cpt in (2, 4):
        many = _run_pool(reqs, kernel=(cpt, 128))
        for k, (side, tau, u0, steps) in enumerate(reqs):
            assert rel_f(many[k][0], one[k][0]) < TOL_F32
            assert rel_u(many[k][1], one[k][1]) < TOL_F32
            r, u = _single(side, tau, u0, steps)
            assert rel_u(many[k][1], u) < TOL_F32
        for k in (0, 1, 3):  # nx = 24, 25 and 7 (pads of 0, 3 and 1 cells), alone against the mix
            alone = _run_pool([reqs[k]], kernel=(cpt, 128))[0]
            np.testing.assert_array_equal(alone[1], many[k][1])
    pool = lbm.Pool("D3Q19", 3, "f32", 1 << 24, 4)
    assert lbm.lbm_pool_get_kernel(pool.handle) == (4, 128)
    for bad in [(3, 0), (0, 96), (8, 128)]:
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_pool_set_kernel(pool.handle, *bad)
        assert e.value.status == lbm.LBM_ERR_UNSUPPORTED
    pool.close()


def test_served_accuracy_by_storage_form():
    """Requests drawn like the serving trace, served by pools of each storage form, against the FP32
    single-lattice solver.  The FP32 pool agrees within the FP32 tolerance, and the fixed-point
    pool with each request's own range (range 0) within the 16-bit bound.  FP16 and the
    fixed-point pool with one range for all are measured and reported (their error grows as a
    request's flow decays, since rounding then weighs more next to u); the check on them is a
    sanity bound of 1e-2 of the initial amplitude, which catches a wrong range or a mixed-up
    result."""
    acc = serve.served_accuracy(n=8, salt=24)  # six of the eight flows stay live
    print(acc)
    assert acc["live_requests"] >= 4
    assert acc["f32"]["max_rel_u_live"] < TOL_F32
    assert acc["f32"]["max_du_over_u0"] < TOL_F32
    for form in ("f16", "q16 (range 0.5)"):
        assert acc[form]["max_du_over_u0"] < 1e-2, form
    # with each request's own range the fixed-point pool holds the 16-bit bound
    assert acc["q16 (range auto)"]["max_rel_u_live"] < 1e-3
    assert acc["q16 (range auto)"]["max_du_over_u0"] < 1e-3


def test_cancelled_request_leaves_the_others_unchanged():
    """Host-side fault injection: a request withdrawn mid-run (and one withdrawn before its first
    step) frees its memory, and the requests that stay give bit for bit the results they give when
    the withdrawn ones never existed."""
    reqs = [(28, 0.7, 0.05, 60), (21, 0.6, 0.04, 60), (35, 0.8, 0.06, 45)]
    base = _run_pool([reqs[0], reqs[2]], kernel=(2, 128))
    pool = lbm.Pool("D3Q19", 3, "f32", 1 << 30, 16)
    lbm.lbm_pool_set_kernel(pool.handle, 2, 128)
    free0 = pool.stats()["free_bytes"]
    ids = []
    for side, tau, u0, steps in reqs:
        rho, u = _tg(side, u0)
        ids.append(pool.submit((side,) * 3, tau, rho, u, steps))
    rho, u = _tg(16, 0.03)
    never = pool.submit((16,) * 3, 0.7, rho, u, 100)
    lbm.lbm_pool_cancel(pool.handle, never)  # before any step
    pool.advance(14)
    pool.advance(14)
    lbm.lbm_pool_cancel(pool.handle, ids[1])  # with chunks in flight
    with pytest.raises(lbm.LbmError) as e:
        pool.poll(ids[1])
    assert e.value.status == lbm.LBM_ERR_NOT_FOUND
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_pool_cancel(pool.handle, ids[1])
    assert e.value.status == lbm.LBM_ERR_NOT_FOUND
    while not (pool.poll(ids[0])[0] and pool.poll(ids[2])[0]):
        pool.advance(14)
        pool.sync()
    r0 = pool.result(ids[0], 28 ** 3)
    r2 = pool.result(ids[2], 35 ** 3)
    assert pool.stats()["resident"] == 0 and pool.stats()["free_bytes"] == free0
    pool.close()
    np.testing.assert_array_equal(r0[1], base[0][1])
    np.testing.assert_array_equal(r2[1], base[1][1])


def test_many_small_requests_under_memory_pressure():
    """300 requests of sides 3-20 (odd and even, so both cell-pair modes), random tau and 0-40
    steps, through an arena that holds about a third of them at once: requests are admitted as
    others' results free memory, and every result matches its own single-lattice run."""
    g = np.random.default_rng(99)
    reqs = [(int(g.integers(3, 21)), float(g.uniform(0.52, 1.0)), float(g.uniform(0.01, 0.08)),
             int(g.integers(0, 41))) for _ in range(300)]
    per = [lbm.lbm_pool_request_bytes("D3Q19", (sd,) * 3, "f32") for sd, _, _, _ in reqs]
    pool = lbm.Pool("D3Q19", 3, "f32", sum(per) // 3 + (1 << 20), 512)
    free0 = pool.stats()["free_bytes"]
    todo = list(range(len(reqs)))
    ids, out = {}, {}
    rounds = 0
    while len(out) < len(reqs):
        while todo:
            sd, tau, u0, n = reqs[todo[0]]
            rho, u = _tg(sd, u0)
            rid = pool.submit((sd,) * 3, tau, rho, u, n)
            if rid is None:
                break
            ids[todo.pop(0)] = rid
        pool.advance(13)
        pool.sync()
        for k, rid in list(ids.items()):
            if pool.poll(rid)[0]:
                out[k] = pool.result(rid, reqs[k][0] ** 3)
                del ids[k]
        rounds += 1
        assert rounds < 1000
    assert pool.stats()["free_bytes"] == free0
    pool.close()
    for k, (sd, tau, u0, n) in enumerate(reqs):
        s = lbm.Solver("D3Q19", (sd,) * 3, tau, 3, "f32")
        rho, u = _tg(sd, u0)
        s.set_fields(rho, u)
        s.step(n)
        r, uu = s.moments()
        s.close()
        assert rel_f(out[k][0], r) < TOL_F32, k
        assert np.max(np.abs(out[k][1] - uu)) < TOL_F32 * u0, k


def test_two_threads_share_a_pool():
    """A pool serialises its own calls: two host threads submitting, advancing, polling and
    collecting their own requests on one pool at once get, bit for bit, the results the same
    requests give alone."""
    import threading

    g = np.random.default_rng(5)
    reqs = [(int(g.integers(8, 30)), float(g.uniform(0.55, 0.9)), float(g.uniform(0.02, 0.06)),
             int(g.integers(5, 60))) for _ in range(16)]
    pool = lbm.Pool("D3Q19", 3, "f32", 1 << 30, 64)
    lbm.lbm_pool_set_kernel(pool.handle, 2, 128)
    out, errors = {}, []

    def worker(ks):
        try:
            ids = {}
            for k in ks:
                sd, tau, u0, n = reqs[k]
                rho, u = _tg(sd, u0)
                rid = None
                while rid is None:
                    rid = pool.submit((sd,) * 3, tau, rho, u, n)
                ids[k] = rid
            while ids:
                pool.advance(9)
                for k, rid in list(ids.items()):
                    if pool.poll(rid)[0]:
                        out[k] = pool.result(rid, reqs[k][0] ** 3)
                        del ids[k]
                pool.stats()
        except Exception as e:  # reported by the main thread
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(range(j, 16, 2),)) for j in (0, 1)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not errors, errors
    assert pool.stats()["resident"] == 0
    pool.close()
    for k, req in enumerate(reqs):
        alone = _run_pool([req], kernel=(2, 128))[0]
        np.testing.assert_array_equal(out[k][1], alone[1])
