"""Pins for the Taylor-subtraction oracle (oracle/taylor.py): Eq. (11) of Sec. II for endpoint exponents
alpha_j <= -1 of any order, the groundwork for integrals with squared propagators.

* On sectors with alpha = -1 only it must reproduce the C oracle on the same lattice points (the established
  p = 0 path), to rounding.
* Massless bubbles with raised propagator powers have the closed form
      I(nu1, nu2) = (-p^2)^{D/2-nu1-nu2} Gamma(nu1+nu2-D/2) Gamma(D/2-nu1) Gamma(D/2-nu2)
                    / (Gamma(nu1) Gamma(nu2) Gamma(D-nu1-nu2)),
  and (3,1), (4,1), (3,2), (3,3) give sectors with alpha = -2 and -3: every Laurent coefficient from eps^-2 to
  eps^2 must match.
* The massless box with one squared propagator has alpha = -2 sectors, up to two singular variables, under both
  decompositions, which share no sector: the two totals must agree.
"""
import dataclasses

import numpy as np
import pytest
from scipy import special as sp

import workloads as W
from oracle import integrate as OI
from oracle import lattice as OL
from oracle import sectors as OS
from oracle import taylor as TT

MASSLESS_LEGS = ("pp1", "pp2", "pp3", "pp4")


def with_nu(topo, nus):
    return dataclasses.replace(topo, props=tuple(dataclasses.replace(p, nu=n) for p, n in zip(topo.props, nus)))


def laurent(f, kmin, kmax, rho=0.25, K=64):
    th = 2 * np.pi * np.arange(K) / K
    eps = rho * np.exp(1j * th)
    vals = np.array([f(e) for e in eps])
    return np.array([np.mean(vals * eps ** (-k)) for k in range(kmin, kmax + 1)])


def test_alpha_minus_one_sectors_reproduce_the_c_oracle():
    cfg = W.CONFIG0
    prob = OI.make_problem(cfg.topology, cfg.point, -2, 0)
    n = 1021
    z = OL.cbc_plain(n, 6)
    sh = W.shifts(3, 2)
    for sec in prob.sectors:
        ours = TT.lattice_sums(sec, prob.e4, n, z, sh, 3, prob.kmax)
        ref, _, _, l1c = OI.lattice_sums(sec, prob.e4, n, z, sh, 0.0, 3, prob.kmax, with_scale=True)
        assert np.all(np.abs(ours - ref.real) <= 1e-12 * np.maximum(l1c, 1e-300)), (sec.A, ours, ref)


@pytest.mark.parametrize("nus", [(2, 1), (3, 1), (4, 1), (3, 2), (3, 3)])
def test_raised_power_bubbles_match_the_closed_form(nus):
    p2 = -2.0
    topo = with_nu(W.bubble(False), nus)
    secs = OS.decompose(topo, (), "iterated", allow_higher_poles=True)
    assert min(min(s.A) for s in secs) == -(max(nus) - 1)
    prob = OI.make_problem(topo, dict(pp1=p2), -2, 2, sectors=secs)
    n = 4093
    mean, err = TT.integrate(prob, n, OL.cbc_plain(n, 6), W.shifts(5, 8), 3)
    v1, v2 = nus

    def closed(e):
        h = 2 - e
        return ((-p2) ** (h - v1 - v2) * sp.gamma(v1 + v2 - h) * sp.gamma(h - v1) * sp.gamma(h - v2)
                / (sp.gamma(v1) * sp.gamma(v2) * sp.gamma(2 * h - v1 - v2)))

    ref = laurent(closed, -2, 2)
    assert np.all(np.abs(mean - ref) <= 5 * err + 1e-12 * (1 + np.abs(ref))), (mean, ref, err)


def test_squared_propagator_box_is_independent_of_the_decomposition():
    topo = W.box(False)
    dotted = with_nu(topo, (2, 1, 1, 1))
    pt = dict(s=-3.0, t=-2.0, **{k: 0.0 for k in MASSLESS_LEGS})
    n = 1021
    z = OL.cbc_plain(n, 6)
    res = []
    for strategy, seed in (("iterated", 1), ("geometric", 2)):
        secs = OS.decompose(dotted, MASSLESS_LEGS, strategy, allow_higher_poles=True)
        assert min(min(s.A) for s in secs) == -2 and max(sum(a <= -1 for a in s.A) for s in secs) == 2
        prob = OI.make_problem(dotted, pt, -2, 0, sectors=secs)
        res.append(TT.integrate(prob, n, z, W.shifts(seed, 4), 3))
    (m1, e1), (m2, e2) = res
    assert np.all(np.abs(m1 - m2) <= 5 * np.hypot(e1, e2)), (m1, m2, e1, e2)
    assert np.all(e1 < 1e-5 * np.abs(m1))
