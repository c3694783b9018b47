"""The regrouping the CUDA collision uses for a velocity pair's two values (PairPoly in
csrc/lbm_core.cuh), checked on the host against the recursion-and-bracket form it replaces.

The kernels write the even and odd parts e, o of drho + rho (E_K - 1) + kappa [bracket] (the
truncated Eq. hermite and the bracket of Eq. hermite-coll, divided by w and shifted) as
polynomials in s = c.u/T0 and q = s^2 with per-cell coefficients.  This test restates both forms
in FP64 numpy from their definitions -- the Hermite recursion h_{n+1} = s h_n - n v2 h_{n-1}
with the brackets of K = 2..5, and the collected coefficients E0, E1, O0, O1 -- and checks that
they agree to rounding for random cells and velocities of every lattice shell, and that the
rest velocity's value is E0.  The GPU parity tests check the kernels themselves against the
oracle; this one pins the algebra of the regrouping.  No GPU."""
import numpy as np
import pytest

T0S = {"D3Q19": 1.0 / 3.0, "D3Q39": 2.0 / 3.0}


def _recursion_form(K, drho, rho, s, v2, A, B, R, kappa):
    h2 = s * s - v2
    h3 = s * (h2 - 2 * v2)
    h4 = s * h3 - 3 * v2 * h2
    h5 = s * h4 - 4 * v2 * h3
    fe = h2 / 2 + (h4 / 24 if K >= 4 else 0.0)
    fo = s + (h3 / 6 if K >= 3 else 0.0) + (h5 / 120 if K >= 5 else 0.0)
    if K == 2:
        be, bo = A, 0.0
    elif K == 3:
        be, bo = A, A * s - 2 * B
    elif K == 4:
        be, bo = A * (1 + h2 / 2) - 2 * B * s + R, A * s - 2 * B
    else:
        e2 = 1 + h2 / 2
        be, bo = A * e2 - 2 * B * s + R, A * (s + h3 / 6) - 2 * B * e2 + R * s
    return drho + rho * fe + kappa * be, rho * fo + kappa * bo


def _polynomial_form(K, drho, rho, s, v2, Z, Bp, kt, kappaR):
    q = s * s
    a1 = 1 - v2 / 2
    if K <= 3:
        E0 = drho - rho / 2 * v2 - kt
        e = E0 + Z + rho / 2 * q
        o = rho * s if K == 2 else s * (rho * a1 - kt + Z + rho / 6 * q) + Bp
        return e, o, E0
    E0 = drho + rho * (v2 * v2 / 8 - v2 / 2) + kappaR - kt * a1
    E1 = rho * (0.5 - v2 / 4) - kt / 2
    e = E0 + a1 * Z + q * (E1 + Z / 2 + rho / 24 * q) + Bp * s
    if K == 4:
        o = s * (rho * a1 - kt + Z + rho / 6 * q) + Bp
    else:
        O0 = rho * (1 - v2 / 2 + v2 * v2 / 8) - kt * a1 + kappaR
        O1 = rho * (1.0 / 6 - v2 / 12) - kt / 6
        o = s * (O0 + a1 * Z + q * (O1 + Z / 6 + rho / 120 * q)) + Bp * (a1 + q / 2)
    return e, o, E0


@pytest.mark.parametrize("K", [2, 3, 4, 5])
def test_pair_polynomial_equals_recursion_form(K):
    g = np.random.default_rng(20020250 + K)
    lattice = "D3Q39" if K >= 4 else "D3Q19"
    T0 = T0S[lattice]
    shells = [(1, 0, 0), (1, 1, 0), (1, -1, 0), (1, 1, 1), (1, -1, 1), (2, 0, 0), (2, 2, 0), (2, 0, -2), (3, 0, 0)]
    worst = 0.0
    for _ in range(300):
        drho = 0.05 * g.standard_normal()
        rho = 1.0 + drho
        u = 0.1 * g.standard_normal(3)
        us = u / T0
        P = 0.02 * g.standard_normal((3, 3))
        P = P + P.T  # Pi^neq
        v2, trP = u @ us, np.trace(P)
        Pu, R = P @ us, u @ (P @ us)
        kappa = g.uniform(0.05, 0.95) / (2 * T0)
        for c in shells:
            c = np.array(c, float)
            s = c @ us
            A, B = c @ P @ c / T0 - trP, c @ Pu
            e_ref, o_ref = _recursion_form(K, drho, rho, s, v2, A, B, R, kappa)
            Z, Bp = c @ (kappa / T0 * P) @ c, c @ (-2 * kappa * Pu)
            e, o, _ = _polynomial_form(K, drho, rho, s, v2, Z, Bp if K >= 3 else 0.0, kappa * trP, kappa * R)
            worst = max(worst, abs(e - e_ref), abs(o - o_ref))
        # the rest velocity (s = 0, A = -tr Pi, B = 0): its value is E0
        e0_ref, o0_ref = _recursion_form(K, drho, rho, 0.0, v2, -trP, 0.0, R, kappa)
        _, _, E0 = _polynomial_form(K, drho, rho, 0.0, v2, 0.0, 0.0, kappa * trP, kappa * R)
        assert o0_ref == 0.0
        worst = max(worst, abs(E0 - e0_ref))
    assert worst < 1e-13, worst


def test_a_dropped_term_is_detected():
    """The comparison above fails for a regrouping that drops a term (the q^2 term of the K = 4
    even part), so it is not vacuous."""
    drho, rho, s, v2, T0 = 0.01, 1.01, 0.3, 0.02, 1.0 / 3.0
    P = np.diag([0.01, -0.02, 0.015])
    kappa, c = 0.4, np.array([1.0, 1.0, 0.0])
    us = np.array([0.1, 0.05, 0.0])
    A, B, R = c @ P @ c / T0 - np.trace(P), c @ (P @ us), (us * T0) @ (P @ us)
    e_ref, _ = _recursion_form(4, drho, rho, s, v2, A, B, R, kappa)
    e, _, _ = _polynomial_form(4, drho, rho, s, v2, c @ (kappa / T0 * P) @ c, c @ (-2 * kappa * P @ us),
                               kappa * np.trace(P), kappa * R)
    assert abs(e - e_ref) < 1e-14
    assert abs((e - rho / 24 * s ** 4) - e_ref) > 1e-6
