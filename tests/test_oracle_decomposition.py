"""Pins for the oracle's sector decomposition (paper Sec. II, Eqs. 3-9).

* the massless box splits into 4 primary x 3 = 12 sectors, with the exponents of Eq. (9);
* the massless bubble's sectors carry t^{-eps} (alpha = 0, beta = -1) and (1+t)^{-2+2eps};
* the sum over sectors of the (finite) undecomposed integrand equals a direct adaptive cubature of the
  Feynman-parameter integral over the simplex (Eq. 2), for the Euclidean massive box and triangle;
* each leaf polynomial has a nonzero constant term (the factorised form of Eqs. 7-8);
* geometric strategy: its simplicial cones tile the space of log x (every random direction lies inside exactly
  one of them), its sectors sum to the simplex integral like the iterated ones, and it terminates (with
  exponents >= -1) on the massless double box, where the iterated strategy does not.
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


@pytest.mark.parametrize("strategy", ["iterated", "hepp", "geometric"])
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


@pytest.mark.parametrize("strategy", ["iterated", "geometric"])
@pytest.mark.parametrize("case", ["box", "triangle"])
def test_sectors_sum_to_simplex_integral(case, strategy):
    if case == "box":
        topo, pt = W.box(True), dict(s=-3.0, t=-2.0, msq=1.0)
    else:
        topo, pt = W.triangle_massive(), dict(pp3=-3.0, msq=1.0)
    prob = OI.make_problem(topo, pt, 0, 0, strategy)
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


def _cone_generators(sec):
    """Generator rows m_i of a geometric sector (x_j = prod_i y_i^(-m_ij))."""
    assert sec.label[0] == "geometric"
    return np.array(sec.label[2], dtype=float)


@pytest.mark.parametrize("topo,zero", [(W.box(False), MASSLESS_LEGS), (W.box(True), MASSLESS_LEGS),
                                       (W.double_box_planar(False), ("pp2", "pp3")),
                                       (W.double_box_nonplanar(True), MASSLESS_LEGS)],
                         ids=["massless_box", "massive_box", "massless_dbox_2offshell", "nonplanar_dbox"])
def test_geometric_cones_tile_log_space(topo, zero):
    """The sectors' cones must cover R^(N-1) without overlap: a random direction u = log x lies in the interior
    of exactly one cone, u = -sum_i s_i m_i with all s_i > 0 (brute force over all cones).  A missing facet of
    the Newton polytope or a wrong triangulation leaves gaps or double cover; and each cone must be a unit of
    Jacobian |det m| = D."""
    secs = sd.decompose(topo, zero, "geometric")
    rng = np.random.default_rng(11)
    gens = [_cone_generators(s) for s in secs]
    for s, g in zip(secs, gens):
        assert abs(abs(np.linalg.det(g)) - float(s.D)) < 1e-9
    for u in rng.standard_normal((300, gens[0].shape[1])):
        inside = 0
        for g in gens:
            coef = np.linalg.solve(g.T, -u)
            inside += bool(np.all(coef > 1e-12))
        assert inside == 1


def test_alpha_below_minus_one_is_rejected_by_both_strategies():
    """A squared propagator of the massless box gives a sector exponent alpha = -2, which needs Taylor
    subtraction beyond Eq. (11) with p = 0; both strategies must refuse it rather than mis-integrate."""
    import dataclasses
    topo = W.box(False)
    dotted = dataclasses.replace(topo, props=(dataclasses.replace(topo.props[0], nu=2),) + topo.props[1:])
    for strategy in ("iterated", "geometric"):
        with pytest.raises(sd.DecompositionError, match="alpha=-2"):
            sd.decompose(dotted, MASSLESS_LEGS, strategy)


def test_geometric_terminates_on_massless_double_box():
    topo = W.double_box_planar(False)
    with pytest.raises(sd.DecompositionError):
        sd.decompose(topo, ("pp2", "pp3"), "iterated", max_depth=25)
    secs = sd.decompose(topo, ("pp2", "pp3"), "geometric")
    assert len(secs) == 143
    assert max(len(s.singular) for s in secs) == 4 and min(min(s.A) for s in secs) == -1
    for s in secs:
        assert (0,) * 6 in s.U and (0,) * 6 in s.F
        assert all(min(e) >= 0 for e in s.U) and all(min(e) >= 0 for e in s.F)
