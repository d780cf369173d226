"""Shifted rank-1 lattice integration of a decomposed integral (oracle; test use only).

Paper Sec. III, Eqs. (16)-(20), applied to the sector integrals of Sec. II, Eq. (9):
    Q_k(eps) = Pre(eps) * sum_sectors (1/n) sum_{i<n} w(x) I_sector(t(x), eps),  x = {i z/n + Delta_k},
    Qbar = (1/m) sum_k Q_k,   err^2 = sum_k |Q_k - Qbar|^2 / (m (m-1))   (re and im variances added),
with Pre(eps) = Gamma(N_nu - L D/2)/prod Gamma(nu_j) (oracle.prefactor).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Dict, List, Optional

import numpy as np

from . import feynman as fy
from . import native
from . import prefactor as pf
from . import sectors as sd

KIND_POS, KIND_NEG, KIND_DEFORM = 0, 1, 2


@dataclass
class NumSector:
    dim: int
    kind: int
    A: np.ndarray
    B: np.ndarray
    D: float
    cU: np.ndarray
    xU: np.ndarray
    cF: np.ndarray
    xF: np.ndarray

    @property
    def sigma(self) -> int:
        """Variables with an endpoint singularity (alpha <= -1; the C integrand takes alpha = -1 only)."""
        return int(np.sum(self.A <= -1))


def numeric_sectors(sectors: List[sd.Sector], point: Dict[str, float]) -> List[NumSector]:
    """Evaluate the exact coefficient linear forms at the kinematic point and classify each sector by the
    signs of Ft's coefficients: all positive -> Ft > 0 on the cube; all negative -> Ft < 0; otherwise the
    sector is deformed (Sec. II, Eq. 14)."""
    out = []
    for s in sectors:
        d = s.dim

        def arrays(poly):
            keys = sorted(poly)
            c = np.array([fy.lf_eval(poly[k], point) for k in keys], dtype=np.float64)
            x = np.array(keys, dtype=np.int32).reshape(len(keys), d)
            keep = c != 0.0
            return np.ascontiguousarray(c[keep]), np.ascontiguousarray(x[keep])

        cU, xU = arrays(s.U)
        cF, xF = arrays(s.F)
        zero = tuple([0] * d)
        if not np.any(np.all(xU == 0, axis=1)) or not np.any(np.all(xF == 0, axis=1)):
            raise sd.DecompositionError(f"constant term vanishes at this kinematic point in sector {s.label}")
        if np.all(cF > 0):
            kind = KIND_POS
        elif np.all(cF < 0):
            kind = KIND_NEG
        else:
            kind = KIND_DEFORM
        out.append(NumSector(d, kind, np.array(s.A, dtype=np.int32), np.array(s.B, dtype=np.int32), float(s.D),
                             cU, xU, cF, xF))
    return out


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _sector_args(sec: NumSector, e4, lam: float, r: int, M: int):
    c = ctypes
    e4 = np.ascontiguousarray(np.array(e4, dtype=np.int32))
    keep = [sec.A, sec.B, e4, sec.cU, sec.xU, sec.cF, sec.xF]
    args = [sec.dim, sec.kind, _ptr(sec.A, c.c_int), _ptr(sec.B, c.c_int), sec.D, _ptr(e4, c.c_int),
            len(sec.cU), _ptr(sec.cU, c.c_double), _ptr(sec.xU, c.c_int), len(sec.cF), _ptr(sec.cF, c.c_double),
            _ptr(sec.xF, c.c_int), float(lam), int(r), int(M)]
    return args, keep


def point_series(sec: NumSector, e4, x, lam: float, r: int, kmax: int):
    """w(x) * I_sector(t(x)) for orders -sigma .. kmax (complex array) and the sign-failure flag."""
    M = kmax + sec.sigma
    nout = M + 1
    args, keep = _sector_args(sec, e4, lam, r, M)
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    out = np.zeros(2 * nout)
    f = native.lib().oracle_point(*args, _ptr(x, ctypes.c_double), _ptr(out, ctypes.c_double), nout)
    if f < 0:
        raise ValueError("oracle_point rejected its arguments")
    return out[0::2] + 1j * out[1::2], f


def lattice_sums(sec: NumSector, e4, n: int, z, shifts, lam: float, r: int, kmax: int,
                 nthreads: Optional[int] = None, with_scale: bool = False):
    """Per-shift sums over the n lattice points: (sums[m, nout] complex, l1[m, nout], fails[m]); with_scale adds
    l1c[m, nout], the summed magnitude of the terms that the endpoint subtraction cancels (Sec. II, after
    Eq. 12: the subtracted remainder suffers from large cancellation) -- the scale of rounding differences."""
    M = kmax + sec.sigma
    nout = M + 1
    args, keep = _sector_args(sec, e4, lam, r, M)
    z = np.ascontiguousarray(np.asarray(z, dtype=np.int64)[: sec.dim])
    sh = np.ascontiguousarray(np.asarray(shifts, dtype=np.float64).reshape(-1, 6))
    m = sh.shape[0]
    sums = np.zeros(2 * m * nout)
    l1 = np.zeros(m * nout)
    l1c = np.zeros(m * nout)
    fails = np.zeros(m, dtype=np.int64)
    nt = nthreads or os.cpu_count() or 1
    rc = native.lib().oracle_lattice_sums(*args, nout, int(n), _ptr(z, ctypes.c_longlong),
                                          _ptr(sh, ctypes.c_double), m, nt, _ptr(sums, ctypes.c_double),
                                          _ptr(l1, ctypes.c_double), _ptr(l1c, ctypes.c_double),
                                          _ptr(fails, ctypes.c_longlong))
    if rc != 0:
        raise ValueError("oracle_lattice_sums rejected its arguments")
    s = sums[0::2] + 1j * sums[1::2]
    if with_scale:
        return s.reshape(m, nout), l1.reshape(m, nout), fails, l1c.reshape(m, nout)
    return s.reshape(m, nout), l1.reshape(m, nout), fails


@dataclass
class Problem:
    """A decomposed integral at one kinematic point, ready for lattice sums."""
    topo: object
    sectors: List[NumSector]
    e4: tuple
    pre_low: int
    pre: List[float]
    order_min: int
    order_max: int

    @property
    def kmax(self) -> int:
        """Highest eps order each sector integral is needed to."""
        return self.order_max - self.pre_low


def make_problem(topo, point: Dict[str, float], order_min: int, order_max: int, strategy: str = "iterated",
                 sectors=None) -> Problem:
    if sectors is None:
        sectors = sd.decompose(topo, sd.zero_invariants_of(topo, point), strategy)
    nsec = numeric_sectors(sectors, point)
    nu = [p.nu for p in topo.props]
    n_nu = sum(nu)
    (eU0, eU1), (eF0, eF1) = sd.exponents_eU_eF(n_nu, topo.loops)
    low, pre = pf.prefactor_series(n_nu, topo.loops, nu, order_max + 8)
    return Problem(topo, nsec, (eU0, eU1, eF0, eF1), low, pre, order_min, order_max)


def combine(problem: Problem, per_sector_sums: List[np.ndarray], n: int):
    """Per-shift Laurent coefficients Q_k for orders order_min..order_max from per-sector sums
    (sums[m, sigma+kmax+1], orders -sigma..kmax)."""
    m = per_sector_sums[0].shape[0]
    lo = problem.order_min - problem.pre_low  # lowest sector order that can reach order_min
    kmin_all = min(-s.sigma for s in problem.sectors)
    lo = min(lo, kmin_all)
    width = problem.kmax - lo + 1
    tot = np.zeros((m, width), dtype=np.complex128)
    for sec, sums in zip(problem.sectors, per_sector_sums):
        for idx in range(sums.shape[1]):
            order = idx - sec.sigma
            if order >= lo:
                tot[:, order - lo] += sums[:, idx] / n
    nord = problem.order_max - problem.order_min + 1
    Q = np.zeros((m, nord), dtype=np.complex128)
    for o in range(problem.order_min, problem.order_max + 1):
        acc = np.zeros(m, dtype=np.complex128)
        for a in range(lo, problem.kmax + 1):
            pidx = o - a - problem.pre_low
            if 0 <= pidx < len(problem.pre):
                acc += problem.pre[pidx] * tot[:, a - lo]
        Q[:, o - problem.order_min] = acc
    return Q


def mean_and_error(Q: np.ndarray):
    """Eqs. (19)-(20): mean over shifts and the standard error sqrt(var_re + var_im)."""
    m = Q.shape[0]
    mean = Q.mean(axis=0)
    if m < 2:
        return mean, np.full(mean.shape, np.inf)
    var = (np.sum((Q.real - mean.real) ** 2, axis=0) + np.sum((Q.imag - mean.imag) ** 2, axis=0)) / (m * (m - 1))
    return mean, np.sqrt(var)


def _lams(problem: Problem, lam):
    if np.ndim(lam) == 0:
        return [float(lam)] * len(problem.sectors)
    if len(lam) != len(problem.sectors):
        raise ValueError("one lambda per sector expected")
    return [float(x) for x in lam]


def integrate(problem: Problem, n: int, z, shifts, lam, r: int, nthreads: Optional[int] = None):
    """One lattice size: returns (mean[orders], err[orders], Q[m, orders], per-sector sums, fails).
    `lam` is one deformation parameter for all sectors or a list with one per sector."""
    per = []
    fails = 0
    for sec, la in zip(problem.sectors, _lams(problem, lam)):
        s, _, f = lattice_sums(sec, problem.e4, n, z, shifts, la, r, problem.kmax, nthreads)
        per.append(s)
        fails += int(f.sum())
    Q = combine(problem, per, n)
    mean, err = mean_and_error(Q)
    return mean, err, Q, per, fails


def adapt_lambda(problem: Problem, n: int, z, shifts, lam0: float, r: int, max_halvings: int = 6,
                 nthreads: Optional[int] = None):
    """Reading of Sec. II, Eq. (14) (lambda must keep Im Ft(z) < 0): start every deformed sector at lam0 and
    halve its lambda while any point of the lattice gives Im Ft(z) > 0, at most `max_halvings` times.
    Returns (per-sector lambdas, per-sector halvings); raises if a sector still fails after the cap."""
    lams, halv = [], []
    for sec in problem.sectors:
        la, h = float(lam0), 0
        if sec.kind == KIND_DEFORM:
            while True:
                _, _, f = lattice_sums(sec, problem.e4, n, z, shifts, la, r, problem.kmax, nthreads)
                if f.sum() == 0:
                    break
                if h == max_halvings:
                    raise RuntimeError("deformation keeps failing the sign check after the halving cap")
                la *= 0.5
                h += 1
        lams.append(la)
        halv.append(h)
    return lams, halv
