"""Pins of the oracle's per-cell collision against what the paper fixes (no GPU).

Each closed form below is retyped from the paper as it is printed there, and is
independent of the oracle's generic tensor-Hermite code:
  * Eq. filter-Pi (K=2), Eq. filter-1st (K=3), Eq. filter-2nd (K=4)
  * Eq. feq_full and Eq. filter-coll (compact, K -> infinity; Appendix proof)
Plus the properties the paper states: conservation (Eq. inv / Eq. conserv),
relative-frame Pi equal to absolute Pi (Sec. 3 after Eq. Q_def), the truncated
forms reproduce Pi (Sec. 3 after Eq. filter-2nd), the u = 0 limit is the prior
filtered form (Sec. 3 after Eq. filter-Pi), and the Galilean error moves to
higher powers of u as K grows (Sec. 4).
"""
import math

import numpy as np
import pytest

import oracle

ALL = ["D2Q9", "D3Q15", "D3Q19", "D3Q27", "D3Q39"]
KMAX = {"D2Q9": 3, "D3Q15": 3, "D3Q19": 3, "D3Q27": 3, "D3Q39": 5}


def _setup(name, seed=1, umag=0.1):
    lat = oracle.lattice(name)
    D = lat["D"]
    g = np.random.default_rng(seed)
    u = g.standard_normal(D)
    u *= umag / np.linalg.norm(u)
    P = g.standard_normal((D, D)) * 1e-3
    Pi = P + P.T
    c = lat["c"][:, :D].astype(np.float64)
    return lat, D, u, Pi, c


def printed_filter(K, lat, u, Pi):
    """Eq. filter-Pi / filter-1st / filter-2nd exactly as printed."""
    D, T0, w = lat["D"], lat["T0"], lat["w"]
    I = np.eye(D)
    out = np.zeros(lat["Q"])
    for i in range(lat["Q"]):
        c = lat["c"][i][:D].astype(np.float64)
        cc = np.outer(c, c) / T0 - I
        cu = (np.outer(c, u) + np.outer(u, c)) / T0
        s = c @ u / T0
        if K == 2:
            M = cc
        elif K == 3:
            M = (1 + s) * cc - cu
        elif K == 4:
            M = (1 + s + (c @ u) ** 2 / (2 * T0 ** 2) - (u @ u) / (2 * T0)) * cc - (1 + s) * cu + np.outer(u, u) / T0
        else:
            raise ValueError(K)
        out[i] = w[i] / (2 * T0) * np.sum(M * Pi)
    return out


def compact_feq(lat, rho, u):
    """Eq. feq_full: w_i exp(e_i/T0) rho exp(-(c_i - u)^2 / 2T0), e_i = c_i^2/2."""
    D, T0, w = lat["D"], lat["T0"], lat["w"]
    c = lat["c"][:, :D].astype(np.float64)
    return w * np.exp((c * c).sum(1) / (2 * T0)) * rho * np.exp(-((c - u) ** 2).sum(1) / (2 * T0))


def compact_fneq(lat, rho, u, Pi):
    """Eq. filter-coll: f^eq/(2 rho T0) [c'c'/T0 - I] : Pi with f^eq from Eq. feq_full."""
    D, T0 = lat["D"], lat["T0"]
    c = lat["c"][:, :D].astype(np.float64) - u
    feq = compact_feq(lat, rho, u)
    A = np.einsum("ia,ib,ab->i", c, c, Pi) / T0 - np.trace(Pi)
    return feq / (2 * rho * T0) * A


@pytest.mark.parametrize("name", ALL)
@pytest.mark.parametrize("K", [2, 3, 4])
def test_truncated_fneq_equals_printed_closed_forms(name, K):
    for seed in range(3):
        lat, D, u, Pi, _ = _setup(name, seed, umag=0.15)
        got = oracle.fneq_hat(name, K, u, Pi)
        want = printed_filter(K, lat, u, Pi)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-16 + 1e-13 * np.abs(want).max())


@pytest.mark.parametrize("name", ["D2Q9", "D3Q19", "D3Q39"])
def test_series_converge_to_compact_forms_with_paper_error_order(name):
    """Truncation error of Eq. hermite ~ |u|^(K+1), of Eq. hermite-coll ~ |u|^(K-1)."""
    lat, D, u, Pi, _ = _setup(name, 3, umag=0.1)
    rho = 1.07
    for K in range(2, 8):
        e_eq = [np.abs(oracle.feq(name, K, rho, s * u) - compact_feq(lat, rho, s * u)).max() for s in (1.0, 0.5)]
        e_ne = [np.abs(oracle.fneq_hat(name, K, s * u, Pi) - compact_fneq(lat, rho, s * u, Pi)).max()
                for s in (1.0, 0.5)]
        slope_eq = math.log2(e_eq[0] / e_eq[1])
        slope_ne = math.log2(e_ne[0] / e_ne[1])
        assert abs(slope_eq - (K + 1)) < 0.25, (name, K, slope_eq)
        assert abs(slope_ne - (K - 1)) < 0.25, (name, K, slope_ne)
    assert np.abs(oracle.feq(name, 10, rho, u) - compact_feq(lat, rho, u)).max() < 1e-12
    # The rho of Eq. feq_full cancels the 1/rho of Eq. filter-coll, so the series needs no density.
    assert np.abs(oracle.fneq_hat(name, 10, u, Pi) - compact_fneq(lat, rho, u, Pi)).max() < 1e-12


@pytest.mark.parametrize("name", ALL)
def test_feq_moments_exact(name):
    """sum f^eq = rho, sum c f^eq = rho u, sum cc f^eq = rho (T0 I + u u)  (Eq. Mflux with isotropy 4)."""
    lat, D, u, Pi, c = _setup(name, 4, umag=0.12)
    rho = 0.93
    for K in range(2, KMAX[name] + 1):
        f = oracle.feq(name, K, rho, u)
        assert abs(f.sum() - rho) < 1e-15
        np.testing.assert_allclose(c.T @ f, rho * u, atol=1e-15)
        np.testing.assert_allclose(np.einsum("ia,ib,i->ab", c, c, f), rho * (lat["T0"] * np.eye(D) + np.outer(u, u)),
                                   atol=1e-15)


def _random_f(lat, seed):
    g = np.random.default_rng(seed)
    return lat["w"] * (1.0 + 0.3 * g.standard_normal(lat["Q"])) + 0.002 * g.standard_normal(lat["Q"])


@pytest.mark.parametrize("name", ALL)
def test_collision_conserves_mass_momentum_and_reproduces_pi(name):
    lat, D, _, _, c = _setup(name)
    for K in range(2, KMAX[name] + 1):
        for seed in range(3):
            f = _random_f(lat, 10 + seed)
            r = oracle.collide(name, K, 0.7, f)
            fp = r["fpost"]
            assert abs(fp.sum() - f.sum()) < 1e-14  # Eq. inv / Eq. conserv
            np.testing.assert_allclose(c.T @ fp, c.T @ f, atol=1e-15)
            # relative-frame Pi (Eq. Pi_def) equals the absolute one (Eq. coeff-2)
            Pi_abs = np.einsum("ia,ib,i->ab", c, c, f - r["feq"])
            np.testing.assert_allclose(r["Pi"][:D, :D], Pi_abs, atol=1e-15)
            # truncated filtered part keeps zero mass/momentum and reproduces Pi
            fh = r["fhat"]
            assert abs(fh.sum()) < 1e-15
            np.testing.assert_allclose(c.T @ fh, 0, atol=1e-15)
            np.testing.assert_allclose(np.einsum("ia,ib,i->ab", c, c, fh), Pi_abs, atol=1e-15)
            # post-collision momentum flux relaxes: Pi' = (1 - 1/tau) Pi
            Pi_post = np.einsum("ia,ib,i->ab", c, c, fp - r["feq"])
            np.testing.assert_allclose(Pi_post, (1 - 1 / 0.7) * Pi_abs, atol=1e-15)


@pytest.mark.parametrize("name", ["D2Q9", "D3Q19", "D3Q27"])
def test_pi_not_reproduced_beyond_isotropy(name):
    """K = 2N is not supported by a class-4 lattice: the filtered Pi drifts (truncation rule, Sec. 3)."""
    lat, D, u, Pi, c = _setup(name, 5, umag=0.1)
    fh = oracle.fneq_hat(name, 4, u, Pi)
    err = np.abs(np.einsum("ia,ib,i->ab", c, c, fh) - Pi).max()
    assert err > 1e-9


@pytest.mark.parametrize("name", ALL)
def test_zero_velocity_reduces_to_prior_filtered_form(name):
    lat, D, _, Pi, c = _setup(name, 6)
    want = printed_filter(2, lat, np.zeros(D), Pi)
    for K in range(2, KMAX[name] + 1):
        np.testing.assert_allclose(oracle.fneq_hat(name, K, np.zeros(D), Pi), want, atol=1e-17)
        # whole collision: remove momentum exactly (sum w c c = T0 I) and compare with w rho + (1-1/tau) filter-Pi
        f = _random_f(lat, 20)
        j = c.T @ f
        f = f - lat["w"] * (c @ j) / lat["T0"]
        assert np.abs(c.T @ f).max() < 1e-16
        rho = f.sum()
        Pi_abs = np.einsum("ia,ib,i->ab", c, c, f) - rho * lat["T0"] * np.eye(D)
        r = oracle.collide(name, K, 0.8, f)
        np.testing.assert_allclose(r["fpost"], lat["w"] * rho + (1 - 1 / 0.8) * printed_filter(2, lat, np.zeros(D),
                                                                                              Pi_abs), atol=1e-16)


@pytest.mark.parametrize("name", ALL)
def test_tau_one_gives_equilibrium_and_filter_is_idempotent(name):
    lat, D, _, _, _ = _setup(name)
    for K in range(2, KMAX[name] + 1):
        f = _random_f(lat, 30)
        r = oracle.collide(name, K, 1.0, f)
        np.testing.assert_array_equal(r["fpost"], r["feq"])
        f1 = oracle.collide(name, K, 1e300, f)["fpost"]  # = f^eq + fhat (1 - 1/tau == 1)
        f2 = oracle.collide(name, K, 1e300, f1)["fpost"]
        np.testing.assert_allclose(f2, f1, atol=1e-16)


@pytest.mark.parametrize("name", ALL)
def test_bgk_comparison_operator(name):
    """Eq. BGK with the same truncated f^eq: conserves mass and momentum; on a state whose
    non-equilibrium part is already filtered it coincides with the filtered collision; on a
    general state the filter removes content BGK keeps (Sec. 1: unsupported higher moments)."""
    lat, D, _, _, c = _setup(name)
    for K in range(2, KMAX[name] + 1):
        f = _random_f(lat, 40 + K)
        fb = oracle.collide_bgk(name, K, 0.7, f)
        assert abs(fb.sum() - f.sum()) < 1e-14
        np.testing.assert_allclose(c.T @ fb, c.T @ f, atol=1e-15)
        np.testing.assert_allclose(fb, f - (f - oracle.feq(name, K, f.sum(), (c.T @ f) / f.sum())) / 0.7, atol=1e-15)
        f1 = oracle.collide(name, K, 1e300, f)["fpost"]  # f^eq + fhat: a filtered state
        np.testing.assert_allclose(oracle.collide_bgk(name, K, 0.7, f1), oracle.collide(name, K, 0.7, f1)["fpost"],
                                   atol=1e-15)
        assert np.abs(fb - oracle.collide(name, K, 0.7, f)["fpost"]).max() > 1e-6


# ---------------------------------------------------------------- energy-flux term (Eq. pq)
def _sym3(g):
    Q = g.standard_normal((3, 3, 3)) * 1e-3
    return (Q + Q.transpose(0, 2, 1) + Q.transpose(1, 0, 2) + Q.transpose(1, 2, 0) + Q.transpose(2, 0, 1)
            + Q.transpose(2, 1, 0)) / 6


def compact_fneq_q(lat, rho, u, Qt):
    """Eq. filter-Q with the 1/rho of Eq. filter-coll: f^eq/(6 rho T0^3) [c'c'c' - 3 c' T0 I] (.) Qt."""
    T0 = lat["T0"]
    c = lat["c"].astype(np.float64) - u
    feq = compact_feq(lat, rho, u)
    A = np.einsum("ia,ib,ic,abc->i", c, c, c, Qt) - 3 * T0 * np.einsum("ia,abb->i", c, Qt)
    return feq / (6 * rho * T0 ** 3) * A


def printed_filter2_theta_term(lat, Q):
    """The theta term of Eq. filter2 as printed: w/(6 T0^2) [ccc/T0 - 3 c I] (.) Q."""
    T0 = lat["T0"]
    c = lat["c"].astype(np.float64)
    A = np.einsum("ia,ib,ic,abc->i", c, c, c, Q) / T0 - 3 * np.einsum("ia,abb->i", c, Q)
    return lat["w"] / (6 * T0 ** 2) * A


@pytest.mark.parametrize("name", ["D3Q15", "D3Q19", "D3Q27", "D3Q39"])
def test_energy_flux_series_limits(name):
    lat = oracle.lattice(name)
    g = np.random.default_rng(9)
    Qt = _sym3(g)
    # u = 0, K = 3: the prior form's theta term (Eq. filter2)
    np.testing.assert_allclose(oracle.fneq_hat_q(name, 3, np.zeros(3), Qt), printed_filter2_theta_term(lat, Qt),
                               atol=1e-18)
    # compact-form limit (Eq. filter-Q) with error order |u|^(K-2)
    u = np.array([0.6, -0.3, 0.2])
    u *= 0.1 / np.linalg.norm(u)
    for K in range(3, 8):
        e = [np.abs(oracle.fneq_hat_q(name, K, s * u, Qt) - compact_fneq_q(lat, 1.3, s * u, Qt)).max()
             for s in (1.0, 0.5)]
        assert abs(math.log2(e[0] / e[1]) - (K - 2)) < 0.3, (K, e)
    want = compact_fneq_q(lat, 1.3, u, Qt)
    assert np.abs(oracle.fneq_hat_q(name, 10, u, Qt) - want).max() < 1e-7 * np.abs(want).max()  # ~V^8/8!


@pytest.mark.parametrize("name,Ks", [("D3Q15", [3]), ("D3Q19", [3]), ("D3Q27", [3]), ("D3Q39", [3, 4, 5])])
def test_energy_flux_term_adds_no_mass_momentum_or_stress(name, Ks):
    lat = oracle.lattice(name)
    c = lat["c"].astype(np.float64)
    g = np.random.default_rng(10)
    Qt = _sym3(g)
    u = np.array([0.05, -0.03, 0.02])
    for K in Ks:
        fq = oracle.fneq_hat_q(name, K, u, Qt)
        assert abs(fq.sum()) < 1e-18
        np.testing.assert_allclose(c.T @ fq, 0, atol=1e-18)
        np.testing.assert_allclose(np.einsum("ia,ib,i->ab", c, c, fq), 0, atol=1e-18)


def test_energy_flux_reproduced_where_the_lattice_supports_it():
    """On D3Q39 (2N = 6) the truncated series reproduces Qt for K <= 4 (orthogonality of H^(n) to
    cubic polynomials needs E^(n+3)); on class-4 lattices the third moment is not supported
    (c_a^3 = c_a there) and is not reproduced."""
    g = np.random.default_rng(11)
    Qt = _sym3(g)
    u = np.array([0.05, -0.03, 0.02])
    lat = oracle.lattice("D3Q39")
    cr = lat["c"].astype(np.float64) - u
    for K in (3, 4):
        fq = oracle.fneq_hat_q("D3Q39", K, u, Qt)
        np.testing.assert_allclose(np.einsum("ia,ib,ic,i->abc", cr, cr, cr, fq), Qt, atol=1e-17)
    lat = oracle.lattice("D3Q19")
    cr = lat["c"].astype(np.float64) - u
    fq = oracle.fneq_hat_q("D3Q19", 3, u, Qt)
    assert np.abs(np.einsum("ia,ib,ic,i->abc", cr, cr, cr, fq) - Qt).max() > 1e-5


@pytest.mark.parametrize("name", ["D3Q19", "D3Q39"])
def test_relative_energy_flux_and_theta_collision(name):
    """Qt of Eq. Q_def equals sum ccc f^neq - 3 sym(u Pi) (the Discussion's linear combination of the
    absolute flux and Pi u); the collision with the theta term still conserves mass and momentum."""
    lat = oracle.lattice(name)
    c = lat["c"].astype(np.float64)
    K = KMAX[name] if name != "D3Q39" else 4
    f = _random_f(lat, 50)
    r = oracle.collide(name, K, 0.7, f)
    rt = oracle.collide_theta(name, K, 0.7, 0.6, f)
    u, Pi = r["u"], r["Pi"]
    fneq = f - r["feq"]
    M3 = np.einsum("ia,ib,ic,i->abc", c, c, c, fneq)
    sym = np.einsum("a,bc->abc", u, Pi) + np.einsum("b,ac->abc", u, Pi) + np.einsum("c,ab->abc", u, Pi)
    np.testing.assert_allclose(rt["Qt"], M3 - sym, atol=1e-16)
    fp = rt["fpost"]
    assert abs(fp.sum() - f.sum()) < 1e-14
    np.testing.assert_allclose(c.T @ fp, c.T @ f, atol=1e-15)
    np.testing.assert_allclose(fp, r["fpost"] + (1 - 1 / 0.7) * 0.6 * rt["fhatq"], atol=1e-16)
    np.testing.assert_allclose(rt["fhatq"], oracle.fneq_hat_q(name, K, u, rt["Qt"]), atol=1e-18)


def _literal_step(lat, K, tau, dims, f):
    """One step written out from the paper with numpy, cell by cell: rho and u (Eq. mme);
    f^eq truncated at K from the explicit Hermite polynomials He_2..He_4 (Eq. hermite);
    f^neq = f - f^eq; Pi^neq in the relative frame (Eq. Pi_def); the printed filtered form
    (Eq. filter-Pi / filter-1st / filter-2nd); f' = f^eq + (1 - 1/tau) fhat (Eq. lbe-reg);
    then f_i(x + c_i) = f'_i(x) with periodic wrap (Eq. lbe)."""
    D, T0, w, Q = lat["D"], lat["T0"], lat["w"], lat["Q"]
    c = lat["c"][:, :D].astype(np.float64)
    nx, ny, nz = dims
    C = nx * ny * nz
    post = np.empty_like(f)
    for x in range(C):
        fx = f[:, x]
        rho = fx.sum()
        u = c.T @ fx / rho
        s = c @ u / T0
        v2 = u @ u / T0
        series = 1 + s + (s * s - v2) / 2
        if K >= 3:
            series = series + (s ** 3 - 3 * s * v2) / 6
        if K >= 4:
            series = series + (s ** 4 - 6 * s * s * v2 + 3 * v2 * v2) / 24
        feq = w * rho * series
        cr = c - u
        Pi = np.einsum("ia,ib,i->ab", cr, cr, fx - feq)
        post[:, x] = feq + (1 - 1 / tau) * printed_filter(K, lat, u, Pi)
    out = np.empty_like(f)
    for i in range(Q):
        a = post[i].reshape(nz, ny, nx)
        cx, cy, cz = (list(lat["c"][i]) + [0, 0])[:3]
        out[i] = np.roll(a, (int(cz), int(cy), int(cx)), axis=(0, 1, 2)).reshape(-1)
    return out


@pytest.mark.parametrize("name,K,dims", [("D2Q9", 2, (5, 4, 1)), ("D2Q9", 3, (4, 3, 1)), ("D3Q19", 3, (4, 3, 5)),
                                         ("D3Q27", 2, (3, 4, 3)), ("D3Q39", 4, (4, 3, 5))])
def test_whole_step_equals_literal_restatement(name, K, dims):
    """Brute force on tiny lattices: three steps of the oracle's grid update against the literal
    numpy restatement above (an independent route to every index: moments, truncation, the
    relative frame, the relaxation and the direction and wrap of the streaming)."""
    lat = oracle.lattice(name)
    C = int(np.prod(dims))
    g = np.random.default_rng(21)
    f = lat["w"][:, None] * (1.0 + 0.05 * g.standard_normal((lat["Q"], C)))
    # a mean flow so that every odd term of the truncation is exercised
    f = f * (1.0 + 0.3 * (lat["c"][:, :1] @ np.ones((1, C))))
    want = f
    for _ in range(3):
        want = _literal_step(lat, K, 0.7, dims, want)
    got = oracle.run(name, K, 0.7, dims, f, 3)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15)
