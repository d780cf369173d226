"""Gamma-function prefactor of the Feynman-parameter representation as a Laurent series in eps (oracle).

Paper Sec. II, Eq. (2): I = Gamma(N_nu - L D/2) / prod_j Gamma(nu_j) * (projective integral), D = 4 - 2 eps,
so Gamma(N_nu - L D/2) = Gamma(n0 + L eps) with n0 = N_nu - 2L.  The sign (-1)^{N_nu} of Eq. (2) belongs to the
(q^2 - m^2) propagators of Eq. (1); with the (-q^2 + m^2) propagators of the paper's examples it is absent.

Series used (plain definitions):
  Gamma(n + x) = Gamma(n) exp( sum_{k>=1} psi^{(k-1)}(n) x^k / k! )            for integer n >= 1,
  psi(n) = -gamma_E + H_{n-1},  psi^{(m)}(n) = (-1)^{m+1} m! (zeta(m+1) - H^{(m+1)}_{n-1}),
  Gamma(n + x) = Gamma(1 + x) / prod_{j=n}^{0} (j + x)                           for integer n <= 0.
zeta(k) is summed directly with an Euler-Maclaurin tail.
"""
from __future__ import annotations

import math
from typing import List, Tuple

EULER_GAMMA = 0.57721566490153286060651209008240243


def zeta(k: int, n_terms: int = 40) -> float:
    """Riemann zeta(k), k >= 2: partial sum to n_terms plus the Euler-Maclaurin remainder."""
    if k < 2:
        raise ValueError("zeta(k) needs k >= 2")
    s = math.fsum(n ** (-k) for n in range(1, n_terms))
    N = float(n_terms)
    # tail sum_{n>=N} n^-k = N^{1-k}/(k-1) + N^-k/2 + sum_j B_2j/(2j)! (k)_{2j-1} N^{-k-2j+1}
    bern = [1.0 / 6, -1.0 / 30, 1.0 / 42, -1.0 / 30, 5.0 / 66]
    tail = N ** (1 - k) / (k - 1) + 0.5 * N ** (-k)
    rising = float(k)  # (k)(k+1)...(k+2j-2)
    for j, b in enumerate(bern, start=1):
        tail += b / math.factorial(2 * j) * rising * N ** (-k - 2 * j + 1)
        rising *= (k + 2 * j - 1) * (k + 2 * j)
    return s + tail


def _exp_series(p: List[float], order: int) -> List[float]:
    """exp of a power series with p[0] = 0, truncated at x^order: E_n = (1/n) sum_k k p_k E_{n-k}."""
    e = [0.0] * (order + 1)
    e[0] = 1.0
    for n in range(1, order + 1):
        e[n] = sum(k * p[k] * e[n - k] for k in range(1, n + 1) if k < len(p)) / n
    return e


def _mul(a, b, order):
    out = [0.0] * (order + 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            if i + j <= order:
                out[i + j] += x * y
    return out


def gamma_shift_series(n: int, scale: int, order: int) -> Tuple[int, List[float]]:
    """Laurent series of Gamma(n + scale*eps): returns (lowest power, coefficients) up to eps^order."""
    if scale == 0:
        raise ValueError("scale must be nonzero")
    if n >= 1:
        p = [0.0] * (order + 1)
        for k in range(1, order + 1):
            m = k - 1
            if m == 0:
                psi = -EULER_GAMMA + math.fsum(1.0 / j for j in range(1, n))
            else:
                psi = (-1) ** (m + 1) * math.factorial(m) * (
                    zeta(m + 1) - math.fsum(j ** (-(m + 1)) for j in range(1, n)))
            p[k] = psi * scale ** k / math.factorial(k)
        e = _exp_series(p, order)
        return 0, [math.factorial(n - 1) * c for c in e]
    # n <= 0: Gamma(1 + x) / prod_{j=n}^{0} (j + x), with x = scale*eps; one pole from j = 0
    low, g1 = gamma_shift_series(1, scale, order + 1)
    # 1/(j + x) for j < 0: -(1/|j|) sum_k (x/|j|)^k ... as a series in eps; 1/x = eps^-1 / scale
    ser = g1[:]
    for j in range(n, 0):
        inv = [(1.0 / j) * (-scale / j) ** k for k in range(order + 2)]
        ser = _mul(ser, inv, order + 1)
    # divide by x = scale*eps: lowest power -1
    return -1, [c / scale for c in ser[: order + 2]]


def prefactor_series(n_nu: int, loops: int, nu: List[int], order_max: int) -> Tuple[int, List[float]]:
    """Gamma(N_nu - L D/2)/prod Gamma(nu_j) = Gamma(N_nu - 2L + L eps)/prod Gamma(nu_j): (lowest power, coeffs)
    with coefficients for eps^low .. eps^order_max."""
    low, c = gamma_shift_series(n_nu - 2 * loops, loops, order_max - (-1) + 1)
    norm = 1.0
    for v in nu:
        norm *= math.gamma(v)
    c = [x / norm for x in c][: order_max - low + 1]
    return low, c
