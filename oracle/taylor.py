"""Sector integrals with endpoint exponents alpha_j <= -1 of any order, by the Taylor subtraction of Eq. (11)
(oracle; test use only).

Paper Sec. II, Eqs. (10)-(12): for a variable with t^{a + b eps} and a = -1 - p (p >= 0),

    int_0^1 t^{a+b eps} f(t) dt = int_0^1 t^{a+b eps} [f(t) - sum_{k<=p} f^(k)(0) t^k / k!] dt
                                  + sum_{k<=p} f^(k)(0) / (k! (a + k + 1 + b eps)),

applied to every such variable of a sector (the operators for different variables commute).  The C oracle
implements p = 0 (every workload of the paper has alpha >= -1); this module takes any p, for undeformed sectors
with F~ > 0 (the Euclidean region), and is slow: plain numpy over the lattice points.

Per point, with S the singular variables and f = g the rest of the sector integrand (D, the monomials of the
other variables, Ut^{eU(eps)} Ft^{-eF(eps)}), every variable j in S is in one of three roles: its value t_j
(factor t_j^{a_j + b_j eps}), a subtracted Taylor term (-t_j^k t_j^{a_j + b_j eps} f^(k)/k! at t_j = 0) or a
pole term (f^(k)/k! at t_j = 0 divided by a_j + k + 1 + b_j eps).  The Taylor coefficients of g in the variables
set to zero come from truncated power series: Ut and Ft restricted to degrees <= p_j in those variables, then
Ut^{a(eps)} = Ut(0)^{a(eps)} sum_n binom(a(eps), n) Q^n with Q = Ut/Ut(0) - 1.  Every quantity is a truncated
series in eps, kept from eps^0 to eps^M, M = kmax + sigma; a pole term with a_j + k + 1 = 0 shifts its product
down one order, and the result occupies the slots of the C oracle: slot n holds eps^(n - sigma).
"""
from __future__ import annotations

import math
from typing import Dict, List, Tuple

import numpy as np

from . import integrate as OI


# ------------------------------------------------------------------ eps series (last axis = order 0..M)
def _smul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Product of eps series (broadcast over leading axes), truncated at the common length."""
    M = a.shape[-1]
    out = np.zeros(np.broadcast_shapes(a.shape, b.shape), dtype=np.float64)
    for i in range(M):
        out[..., i:] += a[..., i: i + 1] * b[..., : M - i]
    return out


def _sexp(x: np.ndarray, M: int) -> np.ndarray:
    """exp(x eps) as a series: x^n / n!."""
    out = np.empty(x.shape + (M,))
    c = np.ones_like(x)
    for n in range(M):
        out[..., n] = c
        c = c * x / (n + 1)
    return out


def _binom_series(a0: float, a1: float, n: int, M: int) -> np.ndarray:
    """binom(a0 + a1 eps, n) as a series in eps."""
    out = np.zeros(M)
    out[0] = 1.0
    for i in range(n):
        fac = np.zeros(M)
        fac[0] = (a0 - i) / (i + 1)
        if M > 1:
            fac[1] = a1 / (i + 1)
        out = _smul(out, fac)
    return out


# ------------------------------------------------------------------ truncated power series in the zeroed variables
def _jet_poly(c: np.ndarray, x: np.ndarray, t: np.ndarray, Z: List[int], p: Dict[int, int]):
    """Polynomial sum_i c_i prod_j t_j^{x_ij} with the variables of Z expanded at 0 up to degree p_j:
    {multi-index over Z: value per point}."""
    jet: Dict[Tuple[int, ...], np.ndarray] = {}
    rest = [j for j in range(t.shape[1]) if j not in Z]
    for ci, xi in zip(c, x):
        k = tuple(int(xi[j]) for j in Z)
        if any(kj > p[j] for kj, j in zip(k, Z)):
            continue
        v = np.full(t.shape[0], float(ci))
        for j in rest:
            if xi[j]:
                v = v * t[:, j] ** int(xi[j])
        jet[k] = jet.get(k, 0.0) + v
    return jet


def _jet_mul(a, b, Z, p, series: bool):
    out = {}
    for ka, va in a.items():
        for kb, vb in b.items():
            k = tuple(x + y for x, y in zip(ka, kb))
            if any(kj > p[j] for kj, j in zip(k, Z)):
                continue
            v = _smul(va, vb) if series else va * vb
            out[k] = out[k] + v if k in out else v
    return out


def _jet_power(jet, a0: float, a1: float, Z, p, M: int):
    """jet^(a0 + a1 eps) for a jet whose constant term is positive: a jet of eps series (points x M)."""
    zero = tuple(0 for _ in Z)
    P0 = jet[zero]
    if np.any(P0 <= 0.0):
        raise ValueError("polynomial not positive at the expansion point (only F~ > 0 sectors are supported)")
    lead = (P0 ** a0)[:, None] * _sexp(a1 * np.log(P0), M)
    Q = {k: v / P0 for k, v in jet.items() if k != zero}
    ntot = sum(p[j] for j in Z)
    acc = {zero: np.ones((P0.shape[0], 1)) * _binom_series(a0, a1, 0, M)[None, :]}
    Qn = {zero: np.ones(P0.shape[0])}
    for n in range(1, ntot + 1):
        Qn = _jet_mul(Qn, Q, Z, p, series=False)
        bn = _binom_series(a0, a1, n, M)
        for k, v in Qn.items():
            term = v[:, None] * bn[None, :]
            acc[k] = acc[k] + term if k in acc else term
    return {k: _smul(lead, v) for k, v in acc.items()}


# ------------------------------------------------------------------ the subtracted sector integrand
SMALL_T = 0.02      # below it a remainder comes from its series
SERIES_TERMS = 10   # Taylor terms of that series (0.02^10 ~ 1e-17 relative truncation)
def transform(r: int, x: np.ndarray):
    """t = phi_r(x), 1 - t = phi_r(1 - x) and w = phi_r'(x) of Eq. (21), generalised to order r:
    phi_r(x) = c_r int_0^x u^r (1-u)^r du, c_r = (2r+1)!/(r!)^2."""
    c = math.factorial(2 * r + 1) / math.factorial(r) ** 2

    def phi(u):
        return c * sum(math.comb(r, k) * (-1) ** k * u ** (r + k + 1) / (r + k + 1) for k in range(r + 1))

    return phi(x), phi(1.0 - x), c * x ** r * (1.0 - x) ** r


def point_series(sec: OI.NumSector, e4, t: np.ndarray, kmax: int) -> np.ndarray:
    """Sector integrand (without the transform weight) at the points t[npts, dim], as slots 0..M
    (slot n = coefficient of eps^(n - sigma), sigma = number of variables with alpha <= -1)."""
    if sec.kind != OI.KIND_POS:
        raise ValueError("Taylor-subtraction oracle: undeformed sectors with F~ > 0 only")
    eU0, eU1, eF0, eF1 = e4
    d = sec.dim
    S = [j for j in range(d) if sec.A[j] <= -1]
    for j in S:
        if sec.B[j] == 0:
            raise ValueError("alpha <= -1 with beta = 0 is not regulated")
    sigma = len(S)
    M = kmax + sigma + 1                     # series length (orders 0..kmax+sigma)
    p = {j: -int(sec.A[j]) - 1 for j in S}
    npts = t.shape[0]
    logt = np.log(t)
    # factors of the non-singular variables (value mode always): t^A exp(B eps log t)
    base = np.full((npts, M), 0.0)
    base[:, 0] = sec.D
    for j in range(d):
        if j in S:
            continue
        if sec.A[j] or sec.B[j]:
            f = (t[:, j] ** int(sec.A[j]))[:, None] * _sexp(sec.B[j] * logt[:, j], M)
            base = _smul(base, f)
    # t_j^{a + b eps} of the singular variables (value and subtracted roles)
    tpow = {j: (t[:, j] ** int(sec.A[j]))[:, None] * _sexp(sec.B[j] * logt[:, j], M) for j in S}
    out = np.zeros((npts, M))
    # The remainder f(t) - sum_{k<=p} f^(k)(0) t^k / k! loses every digit to cancellation where t^{p+1} is
    # below the rounding of f: there (t_j < SMALL_T) it is taken from its own series, the Taylor terms
    # p < k <= p + SERIES_TERMS, instead of the difference.
    small = {j: t[:, j] < SMALL_T for j in S}
    q = {j: p[j] + SERIES_TERMS for j in S}
    for zmask in range(1 << sigma):
        Z = [S[i] for i in range(sigma) if (zmask >> i) & 1]
        ju = _jet_poly(sec.cU, sec.xU, t, Z, q)
        jf = _jet_poly(sec.cF, sec.xF, t, Z, q)
        g = _jet_mul(_jet_power(ju, eU0, eU1, Z, q, M), _jet_power(jf, -eF0, -eF1, Z, q, M), Z, q, series=True)
        values = [j for j in S if j not in Z]
        vfac = np.ones((npts, M))
        vfac[:, 1:] = 0.0
        for j in values:  # the value term of a remainder taken as a difference
            vfac = _smul(vfac, tpow[j] * (~small[j])[:, None])
        for tmask in range(1 << len(Z)):
            T = [Z[i] for i in range(len(Z)) if (tmask >> i) & 1]
            Y = [j for j in Z if j not in T]
            for k, ck in g.items():
                kk = dict(zip(Z, k))
                if any(kk[j] > p[j] for j in T):
                    continue  # pole terms stop at the subtraction order
                term = _smul(_smul(base, ck), vfac)
                shift = 0
                for j in T:
                    c = int(sec.A[j]) + kk[j] + 1
                    if c == 0:
                        term = term / sec.B[j]
                        shift += 1
                    else:
                        ser = np.array([(-sec.B[j] / c) ** m / c for m in range(M)])
                        term = _smul(term, ser[None, :])
                for j in Y:
                    # remainder as a difference (k <= p, subtracted) or as its series (k > p), never both
                    sel = ~small[j] if kk[j] <= p[j] else small[j]
                    sgn = -1.0 if kk[j] <= p[j] else 1.0
                    term = _smul(term, (sgn * sel * t[:, j] ** kk[j])[:, None] * tpow[j])
                # eps^(n - shift) -> slot n - shift + sigma; keep orders <= kmax
                lo = sigma - shift
                out[:, lo: M] += term[:, : M - lo]
    return out


def lattice_sums(sec: OI.NumSector, e4, n: int, z, shifts, r: int, kmax: int) -> np.ndarray:
    """Per-shift sums over the n lattice points of w(x) * integrand(t(x)): array[m, M + 1] (real)."""
    d = sec.dim
    idx = np.arange(n, dtype=np.int64)
    zz = np.asarray(z, dtype=np.int64)[:d]
    res = []
    for delta in np.asarray(shifts, dtype=np.float64).reshape(-1, 6):
        x = (idx[:, None] * zz[None, :] % n) / n + delta[None, :d]
        x = np.where(x >= 1.0, x - 1.0, x)
        ok = np.all(x > 0.0, axis=1)          # the weight vanishes at x = 0
        t, _, w = transform(r, x[ok])
        vals = point_series(sec, e4, t, kmax)
        res.append((np.prod(w, axis=1)[:, None] * vals).sum(axis=0))
    return np.array(res)


def integrate(problem: "OI.Problem", n: int, z, shifts, r: int):
    """Mean and error of the Laurent coefficients (orders order_min..order_max), as oracle.integrate.integrate."""
    per = []
    for sec in problem.sectors:
        per.append(lattice_sums(sec, problem.e4, n, z, shifts, r, problem.kmax).astype(np.complex128))
    Q = OI.combine(problem, per, n)
    mean, err = OI.mean_and_error(Q)
    return mean, err
