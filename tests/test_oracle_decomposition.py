"""Pins for the oracle's sector decomposition (paper Sec. II, Eqs. 3-9).

* the massless box splits into 4 primary x 3 = 12 sectors, with the exponents of Eq. (9);
* the massless bubble's sectors carry t^{-eps} (alpha = 0, beta = -1) and (1+t)^{-2+2eps};
* the sum over sectors of the (finite) undecomposed integrand equals a direct adaptive cubature of the
  Feynman-parameter integral over the simplex (Eq. 2), for the Euclidean massive box and triangle;
* each leaf polynomial has a nonzero constant term (the factorised form of Eqs. 7-8).
"""
from collections import Counter

import numpy as np
import pytest
from scipy import integrate as si

import workloads as W
from oracle import feynman as fy
from oracle import integrate as OI
from oracle import sectors as sd

MASSLESS_LEGS = ("pp1", "pp2", "pp3", "pp4")


def test_massless_box_twelve_sectors():
    secs = sd.decompose(W.box(False), MASSLESS_LEGS)
    assert len(secs) == 12
    assert Counter(len(s.singular) for s in secs) == {2: 8, 1: 4}
    for s in secs:
        assert len(s.U) >= 1 and (0, 0, 0) in s.U and (0, 0, 0) in s.F
        # massless box: A in {-1, 0}, beta = -1 on singular variables (from F^{-(2+eps)}), U exponent 2 eps
        assert set(s.A) <= {-1, 0}
        for a, b in zip(s.A, s.B):
            if a == -1:
                assert b != 0


def test_bubble_exponents():
    secs = sd.decompose(W.bubble(False), ("",))
    assert len(secs) == 2
    for s in secs:
        assert s.A == [0] and s.B == [-1]
        assert fy.substitute_invariants(s.U, {}) == {(0,): 1, (1,): 1}


@pytest.mark.parametrize("strategy", ["iterated", "hepp"])
def test_leaves_factorised(strategy):
    for topo in (W.box(False), W.box(True)):
        for s in sd.decompose(topo, MASSLESS_LEGS, strategy):
            assert (0,) * s.dim in s.U and (0,) * s.dim in s.F


def test_two_loop_decomposition_terminates_with_constant_terms():
    for topo in (W.double_box_planar(True), W.double_box_nonplanar(True)):
        secs = sd.decompose(topo, MASSLESS_LEGS)
        assert len(secs) > 7
        for s in secs:
            assert s.dim == 6 and (0,) * 6 in s.U and (0,) * 6 in s.F
            assert min(s.A) >= -1


def _gauss_cube(f, dim, n=28):
    x, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    grids = np.meshgrid(*([x] * dim), indexing="ij")
    pts = np.stack([g.ravel() for g in grids], axis=1)
    ww = np.ones(len(pts))
    for d in range(dim):
        ww *= np.meshgrid(*([w] * dim), indexing="ij")[d].ravel()
    return float(np.sum(ww * f(pts)))


def _sector_integrand_eps0(sec, e4):
    """Undecomposed-form sector integrand at eps = 0 for sectors without singular variables."""
    def f(t):
        def ev(c, x):
            return np.sum(c[None, :] * np.prod(t[:, None, :] ** x[None, :, :], axis=2), axis=1)
        U = ev(sec.cU, sec.xU)
        F = ev(sec.cF, sec.xF)
        mono = np.prod(t ** sec.A[None, :], axis=1)
        return sec.D * mono * U ** e4[0] * F ** (-e4[2])
    return f


@pytest.mark.parametrize("case", ["box", "triangle"])
def test_sectors_sum_to_simplex_integral(case):
    if case == "box":
        topo, pt = W.box(True), dict(s=-3.0, t=-2.0, msq=1.0)
    else:
        topo, pt = W.triangle_massive(), dict(pp3=-3.0, msq=1.0)
    prob = OI.make_problem(topo, pt, 0, 0)
    assert all(s.sigma == 0 for s in prob.sectors)
    total = sum(_gauss_cube(_sector_integrand_eps0(s, prob.e4), s.dim) for s in prob.sectors)
    # direct: Gamma(N - LD/2)/prod Gamma * int_simplex U^{eU0} / F^{eF0}, eps = 0 (prefactor = 1 here)
    U, F = fy.symanzik_momentum(topo)
    Un = fy.substitute_invariants(U, {**{k: 0 for k in topo.invariants}, **pt})
    Fn = fy.substitute_invariants(F, {**{k: 0 for k in topo.invariants}, **pt})

    def poly(p, x):
        return sum(float(c) * np.prod([xi ** e for xi, e in zip(x, k)]) for k, c in p.items())

    def integrand(*x):
        xs = list(x) + [1.0 - sum(x)]
        return poly(Un, xs) ** prob.e4[0] * poly(Fn, xs) ** (-prob.e4[2])

    if case == "box":
        ref, _ = si.tplquad(lambda x3, x2, x1: integrand(x1, x2, x3), 0, 1, 0, lambda x1: 1 - x1, 0,
                            lambda x1, x2: 1 - x1 - x2, epsabs=1e-13, epsrel=1e-11)
    else:
        ref, _ = si.dblquad(lambda x2, x1: integrand(x1, x2), 0, 1, 0, lambda x1: 1 - x1, epsabs=1e-14,
                            epsrel=1e-12)
    assert abs(total - ref) <= 1e-9 * abs(ref)
