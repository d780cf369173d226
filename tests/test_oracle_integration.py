"""Whole-chain pins for the oracle: decomposition + deformation + subtraction + eps expansion + shifted lattice
rule (paper Secs. II-III) against closed forms, quadrature and invariants.

Closed forms (all in the convention 1/(-q^2 + m^2 - i0), d^Dk/(i pi^{D/2}), D = 4 - 2 eps):
  * massless bubble: Gamma(eps) Gamma(1-eps)^2 / Gamma(2-2eps) (-p^2)^{-eps}, every order;
  * equal-mass bubble above threshold: 1/eps - gamma_E + 2 - ln m^2 - b ln((b+1)/(b-1)), b = sqrt(1-4m^2/(p^2+i0));
  * massive triangle with two massless legs: -(1/(2s)) ln^2((b-1)/(b+1)), b = sqrt(1-4m^2/(s+i0));
  * massless on-shell box: c_G/(st) {(2/eps^2)[(-s)^{-eps} + (-t)^{-eps}] - ln^2(s/t) - pi^2} + O(eps),
    c_G = Gamma(1+eps) Gamma(1-eps)^2 / Gamma(1-2eps).
Invariants: independence of lambda (Eq. 14) and of the decomposition strategy; deformed == undeformed below
threshold == direct simplex cubature; the shift-based error estimate of Eq. (20) covers the exact value at the
expected rate.
"""
import cmath
import math

import numpy as np
import pytest
from scipy import integrate as si
from scipy import special as sp

import workloads as W
from oracle import integrate as OI
from oracle import lattice as OL

GAMMA_E = 0.5772156649015329
LEGS0 = dict(pp1=0.0, pp2=0.0, pp3=0.0, pp4=0.0)


@pytest.fixture(scope="module")
def z4093():
    return OL.cbc_plain(4093, 6)


def laurent(f, kmin, kmax, rho=0.25, K=64):
    th = 2 * np.pi * np.arange(K) / K
    eps = rho * np.exp(1j * th)
    vals = np.array([f(e) for e in eps])
    return np.array([np.mean(vals * eps ** (-k)) for k in range(kmin, kmax + 1)])


def run(topo, pt, omin, omax, z, n=4093, m=8, lam=0.5, r=3, seed=5, strategy="iterated"):
    prob = OI.make_problem(topo, pt, omin, omax, strategy)
    sh = W.shifts(seed, m)
    mean, err, Q, per, fails = OI.integrate(prob, n, z, sh, lam, r)
    return mean, err, fails, prob


def close(mean, err, ref, nsig=5.0, floor=1e-12):
    return np.all(np.abs(mean - ref) <= nsig * err + floor * (1 + np.abs(ref)))


@pytest.mark.parametrize("strategy", ["iterated", "geometric"])
def test_massless_bubble_all_orders(z4093, strategy):
    p2 = -2.0
    mean, err, fails, _ = run(W.bubble(False), dict(pp1=p2), -1, 2, z4093, strategy=strategy)
    ref = laurent(lambda e: sp.gamma(e) * sp.gamma(1 - e) ** 2 / sp.gamma(2 - 2 * e) * (-p2) ** (-e), -1, 2)
    assert close(mean, err, ref), (mean, ref, err)
    assert np.max(np.abs(mean - ref)) < 1e-9


@pytest.mark.parametrize("strategy", ["iterated", "geometric"])
def test_massive_bubble_above_threshold_deformed(z4093, strategy):
    p2 = 5.0
    mean, err, fails, prob = run(W.bubble(True), dict(pp1=p2, msq=1.0), -1, 0, z4093, lam=0.5, strategy=strategy)
    assert all(s.kind == OI.KIND_DEFORM for s in prob.sectors) and fails == 0
    b = cmath.sqrt(1 - 4 / complex(p2, 1e-300))
    ref = np.array([1.0, -GAMMA_E + 2 - b * cmath.log((b + 1) / (b - 1))])
    assert close(mean, err, ref) and np.max(np.abs(mean - ref)) < 1e-9, (mean, ref)


@pytest.mark.parametrize("s", [-3.0, 5.0, 12.0])
def test_massive_triangle(z4093, s):
    mean, err, fails, prob = run(W.triangle_massive(), dict(pp3=s, msq=1.0), 0, 0, z4093, lam=0.5)
    b = cmath.sqrt(1 - 4 / complex(s, 1e-300))
    ref = -1 / (2 * s) * cmath.log((b - 1) / (b + 1)) ** 2
    assert fails == 0
    assert close(mean, err, np.array([ref])) and abs(mean[0] - ref) < 1e-7, (mean, ref)


def massless_box_closed(s, t):
    def f(e):
        cg = sp.gamma(1 + e) * sp.gamma(1 - e) ** 2 / sp.gamma(1 - 2 * e)
        return cg / (s * t) * (2 / e ** 2 * ((-s + 0j) ** (-e) + (-t + 0j) ** (-e))
                               - cmath.log(s / t) ** 2 - math.pi ** 2) * e ** 2
    return laurent(f, 0, 2)


@pytest.mark.parametrize("strategy", ["iterated", "hepp", "geometric"])
def test_massless_box_config0(z4093, strategy):
    cfg = W.CONFIG0
    mean, err, fails, prob = run(cfg.topology, {**cfg.point, **LEGS0}, -2, 0, z4093, lam=0.0, strategy=strategy)
    assert len(prob.sectors) == {"iterated": 12, "hepp": 32, "geometric": 12}[strategy]
    ref = massless_box_closed(-3.0, -2.0)
    assert abs(ref[0] - 2.0 / 3.0) < 1e-14  # 4/(st)
    assert close(mean, err, ref) and np.max(np.abs(mean - ref)) < 1e-7, (mean, ref, err)


def test_massive_box_lambda_and_strategy_independence(z4093):
    cfg = W.CONFIG1
    pt = {**cfg.point, **LEGS0}
    res = [run(cfg.topology, pt, 0, 0, z4093, m=16, lam=lam) for lam in (0.5, 0.25, 0.125)]
    res.append(run(cfg.topology, pt, 0, 0, z4093, m=16, lam=0.5, strategy="hepp"))
    assert len(res[-1][3].sectors) == 24 and len(res[0][3].sectors) == 4
    res.append(run(cfg.topology, pt, 0, 0, z4093, m=16, lam=0.5, strategy="geometric"))
    assert len(res[-1][3].sectors) == 4
    for mean, err, fails, _ in res:
        assert fails == 0
    m0, e0 = res[0][0], res[0][1]
    for mean, err, _, _ in res[1:]:
        assert np.abs(mean - m0) <= 5 * np.hypot(err, e0), (mean, m0)
    assert abs(m0[0]) > 0.1 and e0[0] < 1e-4 * abs(m0[0])


def test_below_threshold_deformed_equals_undeformed_and_cubature(z4093):
    topo, pt = W.box(True), dict(s=3.0, t=-1.5, msq=1.0, **LEGS0)
    mean_d, err_d, fails, prob = run(topo, pt, 0, 0, z4093, lam=0.5)
    assert any(s.kind == OI.KIND_DEFORM for s in prob.sectors) and fails == 0
    mean_u, err_u, _, _ = run(topo, pt, 0, 0, z4093, lam=0.0)
    assert abs(mean_d[0] - mean_u[0]) <= 5 * math.hypot(err_d[0], err_u[0]) + 1e-12
    assert abs(mean_u[0].imag) < 1e-12

    def integrand(x3, x2, x1):
        x4 = 1 - x1 - x2 - x3
        return 1.0 / (1.0 - 3.0 * x1 * x3 + 1.5 * x2 * x4) ** 2

    ref, _ = si.tplquad(integrand, 0, 1, 0, lambda x1: 1 - x1, 0, lambda x1, x2: 1 - x1 - x2, epsabs=1e-13,
                        epsrel=1e-11)
    assert abs(mean_u[0].real - ref) < 1e-8 * ref
    assert abs(mean_d[0] - ref) <= 5 * err_d[0] + 1e-12


def test_error_estimate_coverage():
    """Eq. (20) is an unbiased estimate of the mean-square error: over many independent shift sets the exact
    value lies within 2 estimated standard errors about as often as a Student-t with m-1 dof predicts."""
    topo, pt = W.triangle_massive(), dict(pp3=-3.0, msq=1.0)
    prob = OI.make_problem(topo, pt, 0, 0)
    b = math.sqrt(1 + 4 / 3.0)
    exact = -1 / (2 * -3.0) * math.log((b - 1) / (b + 1)) ** 2
    n, m = 31, 16
    z = OL.cbc_plain(n, 2)
    hits = 0
    trials = 200
    for seed in range(trials):
        mean, err, _, _, _ = OI.integrate(prob, n, z, W.shifts(1000 + seed, m), 0.0, 1, nthreads=1)
        hits += abs(mean[0].real - exact) <= 2 * err[0]
    # t_15: P(|T| < 2) = 0.936
    assert 0.87 <= hits / trials <= 0.985, hits


@pytest.mark.slow
def test_two_loop_lambda_independence():
    z = OL.cbc_plain(1021, 6)
    cfg = W.CONFIG2
    prob = OI.make_problem(cfg.topology, {**cfg.point, **LEGS0}, -2, 0)
    sh = W.shifts(9, 16)
    lams, halv = OI.adapt_lambda(prob, 1021, z, sh, 0.5, 3)
    m1, e1, _, _, f1 = OI.integrate(prob, 1021, z, sh, lams, 3)
    m2, e2, _, _, f2 = OI.integrate(prob, 1021, z, W.shifts(10, 16), [0.5 * x for x in lams], 3)
    assert f1 == 0 and f2 == 0
    assert np.all(np.abs(m1 - m2) <= 5 * np.hypot(e1, e2))


@pytest.mark.parametrize("cfg", [W.CONFIG2, W.CONFIG3], ids=["planar", "nonplanar"])
def test_two_loop_strategy_independence_geometric_vs_iterated(cfg):
    """The physical two-loop double boxes (deformed sectors, poles to eps^-2) from the geometric and the iterated
    decompositions (46 vs 46 and 56 vs 48 sectors, different sector polynomials) must give the same Laurent
    coefficients within the combined errors."""
    n = 2039
    z = OL.cbc_plain(n, 6)
    pt = {**cfg.point, **LEGS0}
    res = []
    for strategy, seed in (("iterated", 21), ("geometric", 22)):
        prob = OI.make_problem(cfg.topology, pt, -2, 0, strategy)
        sh = W.shifts(seed, 16)
        lams, _ = OI.adapt_lambda(prob, n, z, sh, 0.5, 3)
        mean, err, _, _, fails = OI.integrate(prob, n, z, sh, lams, 3)
        assert fails == 0
        res.append((mean, err, len(prob.sectors)))
    (m1, e1, n1), (m2, e2, n2) = res
    assert (n1, n2) == ((46, 46) if cfg is W.CONFIG2 else (48, 56))
    assert np.all(np.abs(m1 - m2) <= 5 * np.hypot(e1, e2)), (m1, m2, e1, e2)
    assert np.all(e1 < 0.25 * np.abs(m1))   # the comparison has teeth: every order is resolved from zero at 4 sigma
