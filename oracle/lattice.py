"""Rank-1 lattice rule, random shifts and component-by-component (CBC) generating vectors (oracle).

Paper Sec. III.
  * Eq. (17): x_i = {i z / n}, i = 0..n-1, z an integer vector with components coprime to n.
  * Eqs. (18)-(20): m independent shifts Delta_k ~ U[0,1]^s; Q_k = (1/n) sum_i f({i z/n + Delta_k});
    mean of the Q_k; unbiased mean-square error sum_k (Q_k - Qbar)^2 / (m(m-1)).
  * CBC (Sec. III, after Eq. 20): the paper gives no criterion; this oracle takes the shift-averaged
    worst-case error of the weighted Korobov space with smoothness 2 and unit weights,
        e^2(z) = -1 + (1/n) sum_i prod_j (1 + 2 pi^2 B2({i z_j / n})),   B2(x) = x^2 - x + 1/6,
    z_1 = 1, each later z_j the minimiser over 1 <= z_j <= (n-1)/2 (ties -> smallest z_j).
  * Lattice sizes: the largest prime below 2^k.
  * Shifts drawn from a seed use splitmix64 (Steele, Lea, Flood 2014), 53-bit doubles, 6 per shift.
"""
from __future__ import annotations

import math
from typing import List

import numpy as np

MASK64 = (1 << 64) - 1


def is_prime(n: int) -> bool:
    if n < 2:
        return False
    if n % 2 == 0:
        return n == 2
    d = 3
    while d * d <= n:
        if n % d == 0:
            return False
        d += 2
    return True


def prime_below(limit: int) -> int:
    """Largest prime strictly below `limit`."""
    n = limit - 1
    while not is_prime(n):
        n -= 1
    return n


def splitmix64_doubles(seed: int, count: int) -> List[float]:
    """`count` doubles in [0,1) from splitmix64 started at state `seed` (top 53 bits of each output)."""
    state = seed & MASK64
    out = []
    for _ in range(count):
        state = (state + 0x9E3779B97F4A7C15) & MASK64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        z ^= z >> 31
        out.append((z >> 11) * (1.0 / (1 << 53)))
    return out


def seeded_shifts(seed: int, m: int) -> np.ndarray:
    """m shift vectors of 6 components each, shift k = draws 6k..6k+5 of splitmix64(seed)."""
    return np.array(splitmix64_doubles(seed, 6 * m), dtype=np.float64).reshape(m, 6)


def lattice_points(n: int, z, shift=None) -> np.ndarray:
    """All n points {i z / n + shift} as an (n, s) array (Eqs. 17-18)."""
    z = np.asarray(z, dtype=np.int64)
    i = np.arange(n, dtype=np.int64)[:, None]
    x = ((i * z[None, :]) % n).astype(np.float64) / n
    if shift is not None:
        x = x + np.asarray(shift, dtype=np.float64)[None, : len(z)]
        x = np.where(x >= 1.0, x - 1.0, x)
    return x


def b2(x):
    return x * x - x + 1.0 / 6.0


def cbc_error2(n: int, z) -> float:
    """e^2(z) of the module docstring, evaluated directly."""
    x = lattice_points(n, z)
    return float(np.mean(np.prod(1.0 + 2.0 * math.pi ** 2 * b2(x), axis=1)) - 1.0)


def cbc_plain(n: int, dim: int, tie_rel: float = 1e-10) -> List[int]:
    """CBC search by exhaustive evaluation of every candidate at every component (O(dim n^2))."""
    i = np.arange(n, dtype=np.int64)
    z = [1]
    p = 1.0 + 2.0 * math.pi ** 2 * b2(((i * 1) % n) / n)
    cand = np.arange(1, (n - 1) // 2 + 1, dtype=np.int64)
    for _ in range(1, dim):
        vals = np.empty(len(cand))
        scale = np.empty(len(cand))
        block = max(1, int(4e6 // n))
        for a in range(0, len(cand), block):
            c = cand[a:a + block]
            om = 2.0 * math.pi ** 2 * b2(((i[None, :] * c[:, None]) % n) / n)
            terms = p[None, :] * om
            vals[a:a + block] = terms.sum(axis=1)
            scale[a:a + block] = np.abs(terms).sum(axis=1)
        best = vals.min()
        tol = tie_rel * scale.max()
        zj = int(cand[np.nonzero(vals <= best + tol)[0][0]])
        z.append(zj)
        p = p * (1.0 + 2.0 * math.pi ** 2 * b2(((i * zj) % n) / n))
    return z
