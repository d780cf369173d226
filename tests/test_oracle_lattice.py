"""Pins for the oracle's lattice rule, CBC criterion, shifts and Gamma prefactor (paper Sec. III, Eqs. 16-21;
Sec. II, Eq. 2)."""
import math

import numpy as np
import pytest

from oracle import lattice as OL
from oracle import prefactor as PF


def test_primes_and_ladder():
    assert OL.prime_below(1 << 16) == 65521
    assert OL.prime_below(1 << 10) == 1021
    assert all(OL.is_prime(p) for p in (2, 3, 101, 1009, 65521))
    assert not any(OL.is_prime(p) for p in (1, 4, 1001, 65535))


def test_splitmix64_reference_vector():
    # published reference output of splitmix64 started from state 0: 0xE220A8397B1DCDAF
    x = OL.splitmix64_doubles(0, 1)[0]
    assert x == (0xE220A8397B1DCDAF >> 11) * 2.0 ** -53


def test_lattice_rule_exact_on_trigonometric_polynomials():
    n, s, H = 1021, 3, 2
    z = OL.cbc_plain(n, s)
    rng = np.random.default_rng(3)
    hs = np.array(np.meshgrid(*[np.arange(-H, H + 1)] * s, indexing="ij")).reshape(s, -1).T
    # no nonzero frequency of the polynomial lies in the dual lattice (brute force)
    dual = [h for h in hs if np.any(h) and int(np.dot(h, z)) % n == 0]
    assert dual == []
    a = rng.normal(size=len(hs)) + 1j * rng.normal(size=len(hs))
    a0 = a[np.all(hs == 0, axis=1)][0]
    for _ in range(3):
        delta = rng.random(6)
        x = OL.lattice_points(n, z, delta)
        f = np.exp(2j * np.pi * x @ hs.T) @ a
        assert abs(f.mean() - a0) < 1e-13
    # a frequency on the dual lattice is picked up with the phase of the shift
    hstar = np.array([(-z[1]) % n - n, 1, 0])
    assert int(np.dot(hstar, z)) % n == 0
    delta = rng.random(6)
    x = OL.lattice_points(n, z, delta)
    f = 0.3 + 0.7 * np.exp(2j * np.pi * x @ hstar)
    assert abs(f.mean() - (0.3 + 0.7 * np.exp(2j * np.pi * np.dot(hstar, delta[:3])))) < 1e-12


def test_cbc_criterion_closed_form_one_dim():
    # (1/n) sum_i B2(i/n) = 1/(6 n^2)  =>  e^2(z = 1) = pi^2 / (3 n^2)
    for n in (101, 1021):
        assert abs(OL.cbc_error2(n, [1]) - math.pi ** 2 / (3 * n * n)) < 1e-15


def _dual_sum(n, z2, H):
    h1 = np.arange(-H, H + 1)
    total = 0.0
    for h2 in range(-H, H + 1):
        cand = h1[((h1 + h2 * z2) % n) == 0]
        if h2 == 0:
            cand = cand[cand != 0]
        r1 = np.where(cand == 0, 1.0, 1.0 / np.where(cand == 0, 1, cand).astype(float) ** 2)
        total += (1.0 if h2 == 0 else 1.0 / h2 ** 2) * r1.sum()
    return total


def test_cbc_criterion_equals_dual_lattice_sum():
    # e^2(z) = sum over nonzero dual-lattice h of prod_j rho(h_j), rho(0) = 1, rho(h) = 1/h^2; the truncated
    # sum converges like 1/H, so extrapolate from H and 2H
    n, z2 = 31, 12
    s1, s2 = _dual_sum(n, z2, 2000), _dual_sum(n, z2, 4000)
    extrap = 2 * s2 - s1
    assert abs(extrap - OL.cbc_error2(n, [1, z2])) < 1e-5 * extrap


@pytest.mark.parametrize("n", [101, 1009])
def test_cbc_choice_is_exhaustive_argmin(n):
    z = OL.cbc_plain(n, 4)
    assert z[0] == 1
    for j in range(1, 4):
        errs = [OL.cbc_error2(n, z[:j] + [c]) for c in range(1, (n - 1) // 2 + 1)]
        best = min(errs)
        assert OL.cbc_error2(n, z[: j + 1]) <= best * (1 + 1e-9)


def test_cbc_error_decreases_along_ladder():
    errs = [OL.cbc_error2(n, OL.cbc_plain(n, 6)) for n in (251, 1021, 4093)]
    assert errs[0] > errs[1] > errs[2]
    # close to the O(n^-2+delta) rate of smooth periodic integrands
    assert errs[1] / errs[2] > 4.0


def test_zeta_closed_forms():
    assert abs(PF.zeta(2) - math.pi ** 2 / 6) < 1e-15
    assert abs(PF.zeta(4) - math.pi ** 4 / 90) < 1e-15
    assert abs(PF.zeta(6) - math.pi ** 6 / 945) < 1e-15


@pytest.mark.parametrize("n,a", [(1, 1), (2, 1), (3, 2), (0, 1), (-1, 2)])
def test_gamma_series_against_gamma_function(n, a):
    low, c = PF.gamma_shift_series(n, a, 6)
    for eps in (0.01, -0.013, 0.02):
        approx = sum(ck * eps ** (low + k) for k, ck in enumerate(c))
        assert abs(approx - math.gamma(n + a * eps)) <= 1e-11 * abs(math.gamma(n + a * eps))


def test_gamma_series_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    for n, a in [(2, 1), (3, 2), (0, 1), (-1, 2)]:
        low, c = PF.gamma_shift_series(n, a, 5)
        ref = mp.taylor(lambda e: mp.gamma(n + a * e) * e ** (-low), 0, 5, singular=True)
        assert max(abs(float(x) - y) for x, y in zip(ref, c)) < 1e-13 * max(1.0, max(abs(y) for y in c))
