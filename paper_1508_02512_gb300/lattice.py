"""Generating vectors for the shifted rank-1 lattice rule (paper Sec. III, Eq. 17 and the CBC remark after
Eq. 20), computed by the fast component-by-component construction.

Criterion: the shift-averaged worst-case error of the unit-weight Korobov space of smoothness 2,
    e^2(z) = -1 + (1/n) sum_{i<n} prod_j (1 + omega({i z_j / n})),  omega(x) = 2 pi^2 (x^2 - x + 1/6).
With z_1..z_{j-1} fixed, the choice of z_j minimises T(c) = sum_i p(i) omega(i c mod n / n), where
p(i) = prod_{k<j} (1 + omega(i z_k mod n / n)); ties within 1e-10 * max_c sum_i |p(i) omega(i c)| go to the
smallest c in 1..(n-1)/2.

Fast evaluation (Nuyens and Cools, 2006): for prime n, i = g^a and c = g^b with g a primitive root, so
i c = g^{a+b} and T over all candidates is one cyclic cross-correlation of length n-1, done with FFTs.

Running this module writes the built-in lattice table of the C library (csrc/lattice_table.h): the largest
prime below 2^k with its 6-component vector, for k = 10..26.
"""
from __future__ import annotations

import math
import os
import sys
from typing import List

import numpy as np

LADDER_LOG2 = tuple(range(10, 27))
DIM = 6


def _is_prime(n: int) -> bool:
    if n < 2:
        return False
    for p in (2, 3, 5, 7, 11, 13):
        if n % p == 0:
            return n == p
    # deterministic Miller-Rabin for n < 3.3e24
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for a in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def largest_prime_below(limit: int) -> int:
    n = limit - 1
    while not _is_prime(n):
        n -= 1
    return n


def _prime_factors(n: int) -> List[int]:
    out, p = [], 2
    while p * p <= n:
        if n % p == 0:
            out.append(p)
            while n % p == 0:
                n //= p
        p += 1
    if n > 1:
        out.append(n)
    return out


def primitive_root(n: int) -> int:
    qs = _prime_factors(n - 1)
    g = 2
    while any(pow(g, (n - 1) // q, n) == 1 for q in qs):
        g += 1
    return g


def _powers(g: int, n: int) -> np.ndarray:
    """g^a mod n for a = 0..n-2, by blocks of sqrt(n) (int64 products stay below 2^62)."""
    m = n - 1
    B = int(math.isqrt(m)) + 1
    small = np.empty(B, dtype=np.int64)
    v = 1
    for a in range(B):
        small[a] = v
        v = v * g % n
    gB = pow(g, B, n)
    big = np.empty((m + B - 1) // B, dtype=np.int64)
    v = 1
    for k in range(len(big)):
        big[k] = v
        v = v * gB % n
    out = (big[:, None] * small[None, :]) % n
    return out.ravel()[:m]


def _omega(k: np.ndarray, n: int) -> np.ndarray:
    x = k.astype(np.float64) / n
    return 2.0 * math.pi ** 2 * (x * x - x + 1.0 / 6.0)


def fast_cbc(n: int, dim: int = DIM, tie_rel: float = 1e-10) -> List[int]:
    if not _is_prime(n):
        raise ValueError("fast CBC needs a prime lattice size")
    m = n - 1
    g = primitive_root(n)
    gp = _powers(g, n)                       # gp[a] = g^a
    om_g = _omega(gp, n)                     # omega(g^c / n)
    F_om = np.fft.rfft(om_g)
    F_abs = np.fft.rfft(np.abs(om_g))
    om0 = 1.0 / 6.0 * 2.0 * math.pi ** 2     # omega(0)
    p = 1.0 + om_g                           # p(g^a) with z_1 = 1
    p0 = 1.0 + om0
    z = [1]
    # candidate c = g^b has representative min(c, n - c); T is symmetric under c -> n - c
    for _ in range(1, dim):
        corr = np.fft.irfft(np.conj(np.fft.rfft(p)) * F_om, n=m)        # sum_a p[a] om[a + b]
        scl = np.fft.irfft(np.conj(np.fft.rfft(np.abs(p))) * F_abs, n=m)
        T = p0 * om0 + corr
        S = abs(p0 * om0) + scl
        cand = gp  # c = g^b
        rep = np.minimum(cand, n - cand)
        best = T.min()
        tol = tie_rel * S.max()
        ok = T <= best + tol
        zj = int(rep[ok].min())
        z.append(zj)
        # update p(i) for i = g^a: omega(i zj) = omega(g^{a + log zj})
        b = int(np.nonzero(gp == zj)[0][0])
        p = p * (1.0 + np.roll(om_g, -b))
        p0 = p0 * (1.0 + om0)
    return z


def ladder(log2s=LADDER_LOG2, dim: int = DIM):
    return [(largest_prime_below(1 << k), fast_cbc(largest_prime_below(1 << k), dim)) for k in log2s]


def write_header(path: str, entries) -> None:
    lines = ["/* Built-in rank-1 lattices: largest prime n below 2^k and its fast-CBC generating vector (unit-weight",
             " * Korobov space, smoothness 2).  Written by `python -m paper_1508_02512_gb300.lattice`; do not edit. */",
             "#pragma once", "#include <stdint.h>", "",
             f"#define QMC_BUILTIN_LATTICES {len(entries)}",
             "static const struct { int64_t n; uint32_t z[6]; } qmc_builtin_lattice[QMC_BUILTIN_LATTICES] = {"]
    for n, z in entries:
        lines.append("    {%dLL, {%s}}," % (n, ", ".join(str(v) for v in z)))
    lines.append("};")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    logs = tuple(int(a) for a in sys.argv[1:]) or LADDER_LOG2
    entries = []
    for k in logs:
        n = largest_prime_below(1 << k)
        z = fast_cbc(n)
        print(k, n, z, flush=True)
        entries.append((n, z))
    write_header(os.path.join(here, "csrc", "lattice_table.h"), entries)
