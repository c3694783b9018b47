"""Pins of the oracle's lattice tables and Hermite tensors against what the paper
and mathematics fix (no GPU).

* Eq. iso: sum_i w_i c_i^[n] = T0^(n/2) Delta^n for even n <= 2N, 0 for odd n.
  Checked in exact rational arithmetic; the class 2N is found as the largest
  even order that holds, and compared with the paper's statements
  (tests/golden/paper_lattice_facts.txt).
* Eq. recurG: the tensor Hermite polynomials contracted with a vector a reduce to
  the scalar probabilists' Hermite polynomial, H^(n)(xi):a^[n] = |a|^n He_n(xi.a/|a|)
  (numpy.polynomial.hermite_e), are symmetric, match the explicit H^(2) and H^(3)
  written in the Appendix (Eq. Order0, Eq. Order1), and are orthogonal under
  the lattice weights up to the degree the isotropy supports.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from numpy.polynomial import hermite_e

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_lattice_facts.txt")
ALL = ["D2Q9", "D3Q15", "D3Q19", "D3Q27", "D3Q39"]


def _exact(lat):
    w = [Fraction(x).limit_denominator(5000) for x in lat["w"]]
    for wf, x in zip(w, lat["w"]):
        assert abs(float(wf) - x) < 1e-15
    T0 = Fraction(lat["T0"]).limit_denominator(100)
    return w, T0


def _delta_count(idx):
    """Number of perfect matchings of the multi-index into equal-index pairs (Delta^n entry)."""
    counts = {}
    for a in idx:
        counts[a] = counts.get(a, 0) + 1
    out = 1
    for k in counts.values():
        if k % 2:
            return 0
        out *= math.prod(range(k - 1, 0, -2))
    return out


def _isotropy_holds(lat, n):
    w, T0 = _exact(lat)
    D = lat["D"]
    for idx in itertools.combinations_with_replacement(range(D), n):
        E = sum((wi * math.prod(int(ci[a]) for a in idx) for wi, ci in zip(w, lat["c"])), Fraction(0))
        if n % 2:
            want = Fraction(0)
        else:
            want = T0 ** (n // 2) * _delta_count(idx)
        if E != want:
            return False
    return True


def _isotropy_class(lat):
    twoN = 0
    for n in range(1, 10):
        if not _isotropy_holds(lat, n):
            break
        if n % 2 == 0:
            twoN = n
    return twoN


def test_weights_sum_to_one_and_velocities_distinct():
    for name in ALL:
        lat = oracle.lattice(name)
        w, _ = _exact(lat)
        assert sum(w) == 1
        assert len({tuple(c) for c in lat["c"]}) == lat["Q"]
        assert all(x > 0 for x in w)
    assert [oracle.lattice(n)["Q"] for n in ALL] == [9, 15, 19, 27, 39]


def test_isotropy_class_matches_paper_statements():
    facts = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, twoN, rel, T0 = line.split()
        facts[name] = (int(twoN), rel, T0)
    for name, (twoN, rel, T0) in facts.items():
        lat = oracle.lattice(name)
        got = _isotropy_class(lat)
        if rel == "==":
            assert got == twoN, (name, got)
        else:
            assert got >= twoN, (name, got)
        if T0 != "-":
            assert Fraction(lat["T0"]).limit_denominator(100) == Fraction(T0)


def test_isotropy_class_all_lattices():
    # D3Q27 is not in the paper: the same identities give class 4 (E^(6) fails).
    assert [_isotropy_class(oracle.lattice(n)) for n in ALL] == [4, 4, 4, 4, 6]
    assert Fraction(oracle.lattice("D3Q39")["T0"]).limit_denominator(100) == Fraction(2, 3)


def _contract(H, a):
    out = H
    for _ in range(H.ndim):
        out = out @ a if out.ndim > 0 else out
    return float(out)


@pytest.mark.parametrize("name", ALL)
def test_hermite_tensor_reduces_to_scalar_hermite(name):
    lat = oracle.lattice(name)
    D, T0 = lat["D"], lat["T0"]
    g = np.random.default_rng(5)
    for i in range(lat["Q"]):
        xi = lat["c"][i][:D] / math.sqrt(T0)
        a = g.standard_normal(D)
        na = np.linalg.norm(a)
        for n in range(0, 7):
            H = oracle.hermite(name, i, n)
            lhs = _contract(H, a) if n else float(H)
            coef = np.zeros(n + 1)
            coef[n] = 1.0
            rhs = na ** n * hermite_e.hermeval(xi @ a / na, coef)
            assert abs(lhs - rhs) <= 1e-11 * max(1.0, abs(rhs)), (name, i, n, lhs, rhs)


@pytest.mark.parametrize("name", ["D2Q9", "D3Q39"])
def test_hermite_tensor_symmetric_and_explicit_low_orders(name):
    lat = oracle.lattice(name)
    D, T0 = lat["D"], lat["T0"]
    I = np.eye(D)
    for i in range(lat["Q"]):
        xi = lat["c"][i][:D] / math.sqrt(T0)
        H2 = oracle.hermite(name, i, 2)
        np.testing.assert_allclose(H2, np.outer(xi, xi) - I, atol=1e-14)  # Eq. Order0
        H3 = oracle.hermite(name, i, 3)
        want = (np.einsum("a,b,c->abc", xi, xi, xi) - np.einsum("a,bc->abc", xi, I)
                - np.einsum("b,ca->abc", xi, I) - np.einsum("c,ab->abc", xi, I))  # Eq. Order1
        np.testing.assert_allclose(H3, want, atol=1e-13)
        H5 = oracle.hermite(name, i, 5)
        for p in itertools.permutations(range(5)):
            np.testing.assert_allclose(np.transpose(H5, p), H5, atol=1e-12)


@pytest.mark.parametrize("name,twoN", [("D2Q9", 4), ("D3Q15", 4), ("D3Q19", 4), ("D3Q27", 4), ("D3Q39", 6)])
def test_hermite_orthogonality_under_lattice_weights(name, twoN):
    """sum_i w_i [H^(m):a^m][H^(n):b^n] = delta_mn n! (a.b)^n whenever m+n <= 2N+1."""
    lat = oracle.lattice(name)
    D = lat["D"]
    g = np.random.default_rng(7)
    a, b = g.standard_normal(D), g.standard_normal(D)
    for m in range(0, twoN):
        for n in range(0, twoN):
            if m + n > twoN + 1:
                continue
            s = 0.0
            for i in range(lat["Q"]):
                Hm = oracle.hermite(name, i, m)
                Hn = oracle.hermite(name, i, n)
                s += lat["w"][i] * (_contract(Hm, a) if m else float(Hm)) * (_contract(Hn, b) if n else float(Hn))
            want = math.factorial(n) * (a @ b) ** n if m == n else 0.0
            assert abs(s - want) < 1e-11, (name, m, n, s, want)
