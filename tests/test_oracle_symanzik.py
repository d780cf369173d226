"""Pins for the oracle's Symanzik polynomials (paper Sec. II, Eq. 2): textbook forms, homogeneity, and the
graph (spanning tree / 2-forest) construction against the momentum-representation construction."""
from fractions import Fraction

import pytest

import workloads as W
from oracle import feynman as fy

TOPOS = [W.bubble(False), W.bubble(True), W.triangle_massive(), W.box(False), W.box(True),
         W.double_box_planar(False), W.double_box_planar(True), W.double_box_nonplanar(False),
         W.double_box_nonplanar(True)]


def num(poly, **vals):
    return fy.substitute_invariants(poly, {k: Fraction(v) for k, v in vals.items()})


def test_bubble_textbook():
    # F = -p^2 x1 x2 + (x1 + x2)(x1 m1^2 + x2 m2^2) with m1 = m2 = m
    U, F = fy.symanzik_momentum(W.bubble(True))
    assert num(U) == {(1, 0): 1, (0, 1): 1}
    assert num(F, pp1=7, msq=3) == {(1, 1): -7 + 6, (2, 0): 3, (0, 2): 3}


def test_massless_box_textbook():
    # F = -s x1 x3 - t x2 x4 for massless legs, U = x1 + x2 + x3 + x4
    U, F = fy.symanzik_momentum(W.box(False))
    assert num(U) == {(1, 0, 0, 0): 1, (0, 1, 0, 0): 1, (0, 0, 1, 0): 1, (0, 0, 0, 1): 1}
    assert num(F, s=5, t=-3, pp1=0, pp2=0, pp3=0, pp4=0) == {(1, 0, 1, 0): -5, (0, 1, 0, 1): 3}


def test_massive_box_is_massless_plus_U_sum_m2x():
    _, F0 = fy.symanzik_momentum(W.box(False))
    U, F = fy.symanzik_momentum(W.box(True))
    vals = dict(s=5, t=-3, pp1=0, pp2=0, pp3=0, pp4=0)
    expect = fy.p_add(F0, fy.p_mul(U, {(1, 0, 0, 0): {"msq": 1}, (0, 1, 0, 0): {"msq": 1},
                                         (0, 0, 1, 0): {"msq": 1}, (0, 0, 0, 1): {"msq": 1}}))
    assert num(F, msq=2, **vals) == num(expect, msq=2, **vals)


@pytest.mark.parametrize("topo", TOPOS, ids=lambda t: t.name)
def test_homogeneity(topo):
    U, F = fy.symanzik_momentum(topo)
    assert all(sum(e) == topo.loops for e in U)
    assert all(sum(e) == topo.loops + 1 for e in F)
    # U is linear in every Feynman parameter (a sum over trees)
    assert all(max(e) <= 1 for e in U)


@pytest.mark.parametrize("topo", TOPOS, ids=lambda t: t.name)
def test_graph_construction_matches_momentum(topo):
    Um, Fm = fy.symanzik_momentum(topo)
    Ug, Fg = fy.symanzik_graph(topo)
    assert Um == Ug
    assert Fm == Fg


def test_double_box_U_term_count():
    # planar double box: 3x3 products of the two outer loops plus 6 terms with the rung = 15 spanning trees
    U, _ = fy.symanzik_momentum(W.double_box_planar(False))
    assert len(U) == 15
