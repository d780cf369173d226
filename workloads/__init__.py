"""Integral definitions and seeded synthetic inputs shared by the oracle and the GPU path.

This module holds *data only*: the loop integrals of the form of the paper's Eq. (1) (propagator momenta as
integer combinations of loop momenta k_l and independent external momenta p_e, internal masses, powers nu_j),
the kinematic points, the lattice/shift parameters of the five workloads, and a seeded generator of random
shift vectors.  It contains none of the method's arithmetic (no Feynman parametrisation, no sector
decomposition, no integrand, no lattice rule): both the oracle and the product derive everything from these
definitions independently.

Conventions (all momenta incoming, sum p = 0):
  * propagator j is 1/(-q_j^2 + m_j^2 - i0)^{nu_j}, measure d^Dk/(i pi^{D/2}), D = 4 - 2 eps
    (the convention of the paper's examples, Eqs. (23), (25), (27));
  * 4-point kinematics use independent p1, p2, p3 (p4 = -p1-p2-p3) and invariants
    s = (p1+p2)^2, t = (p2+p3)^2, pp_i = p_i^2; u = pp1+pp2+pp3+pp4 - s - t;
  * masses are named invariants (e.g. "msq" = M^2) so that coefficients of the Symanzik polynomials are
    linear forms in the invariants.

Graphs (vertex lists per edge and the vertex each external momentum enters) are given alongside the momentum
routing; tests use them for the spanning-tree / 2-forest cross-check of U and F.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from fractions import Fraction
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

F = Fraction
LinearForm = Dict[str, Fraction]  # invariant name -> coefficient ("" would be a constant; unused)


@dataclass(frozen=True)
class Propagator:
    k: Tuple[int, ...]          # coefficients of the loop momenta k_1..k_L
    p: Tuple[int, ...]          # coefficients of the independent external momenta p_1..p_E
    mass: Optional[str] = None  # name of the invariant holding m_j^2, or None for a massless line
    nu: int = 1                 # propagator power


@dataclass(frozen=True)
class Topology:
    name: str
    loops: int
    n_ext: int                                  # number of independent external momenta E
    props: Tuple[Propagator, ...]
    invariants: Tuple[str, ...]                 # ordered invariant basis of the kinematics vector
    gram: Tuple[Tuple[Tuple[Tuple[str, Fraction], ...], ...], ...]  # gram[e][f] = linear form (name, coef)
    # graph description (for cross-checks): edge j joins (tail, head); ext_at[e] = vertex where the e-th
    # external momentum enters (including the dependent one, last)
    edges: Tuple[Tuple[int, int], ...] = ()
    ext_at: Tuple[int, ...] = ()

    @property
    def n_props(self) -> int:
        return len(self.props)

    def gram_form(self, e: int, f: int) -> LinearForm:
        return {k: F(v) for k, v in self.gram[e][f]}


def _lf(**kw) -> Tuple[Tuple[str, Fraction], ...]:
    return tuple((k, F(v)) for k, v in kw.items() if v != 0)


def _gram_2pt():
    return ((_lf(pp1=1),),)


def _gram_3pt():
    # p3 = -p1-p2: p1.p2 = (pp3 - pp1 - pp2)/2
    h = F(1, 2)
    p12 = _lf(pp3=h, pp1=-h, pp2=-h)
    return ((_lf(pp1=1), p12), (p12, _lf(pp2=1)))


def _gram_4pt():
    h = F(1, 2)
    p12 = _lf(s=h, pp1=-h, pp2=-h)
    p23 = _lf(t=h, pp2=-h, pp3=-h)
    p13 = _lf(pp2=h, pp4=h, s=-h, t=-h)  # (u - pp1 - pp3)/2 with u = sum pp - s - t
    return ((_lf(pp1=1), p12, p13), (p12, _lf(pp2=1), p23), (p13, p23, _lf(pp3=1)))


INV_2PT = ("pp1",)
INV_3PT = ("pp1", "pp2", "pp3")
INV_4PT = ("s", "t", "pp1", "pp2", "pp3", "pp4")


def bubble(massive: bool) -> Topology:
    m = "msq" if massive else None
    inv = INV_2PT + (("msq",) if massive else ())
    return Topology(
        name="bubble_m" if massive else "bubble_0", loops=1, n_ext=1,
        props=(Propagator((1,), (0,), m), Propagator((1,), (1,), m)),
        invariants=inv, gram=_gram_2pt(),
        edges=((1, 0), (0, 1)), ext_at=(0, 1))


def triangle_massive() -> Topology:
    """Triangle with three internal lines of mass^2 'msq'; legs p1, p2 and p3 = -p1-p2 (pp3 = s)."""
    m = "msq"
    return Topology(
        name="triangle_m", loops=1, n_ext=2,
        props=(Propagator((1,), (0, 0), m), Propagator((1,), (1, 0), m), Propagator((1,), (1, 1), m)),
        invariants=INV_3PT + ("msq",), gram=_gram_3pt(),
        # e1: v3->v1 (k), e2: v1->v2 (k+p1), e3: v2->v3 (k+p1+p2); p1 at v1, p2 at v2, p3 at v3
        edges=((2, 0), (0, 1), (1, 2)), ext_at=(0, 1, 2))


def box(massive: bool) -> Topology:
    """One-loop box: q = k, k+p1, k+p1+p2, k+p1+p2+p3 (F = -s x1 x3 - t x2 x4 + ... when legs are massless)."""
    m = "msq" if massive else None
    inv = INV_4PT + (("msq",) if massive else ())
    return Topology(
        name="box_m" if massive else "box_0", loops=1, n_ext=3,
        props=(Propagator((1,), (0, 0, 0), m), Propagator((1,), (1, 0, 0), m),
               Propagator((1,), (1, 1, 0), m), Propagator((1,), (1, 1, 1), m)),
        invariants=inv, gram=_gram_4pt(),
        # e1: v4->v1, e2: v1->v2, e3: v2->v3, e4: v3->v4; p_i enters at v_i
        edges=((3, 0), (0, 1), (1, 2), (2, 3)), ext_at=(0, 1, 2, 3))


def double_box_planar(massive: bool = True) -> Topology:
    """Planar double box with the routing of the paper's Eq. (25), outgoing p3 rewritten as incoming.

    Lines 4..7 (the right loop and the rung) carry mass^2 'msq' when massive.
    q = k1, k1-p1, k1+p2, k1-k2-p1, k2, k1-k2+p2+p3, k1-k2+p2.
    """
    m = "msq" if massive else None
    P = Propagator
    props = (P((1, 0), (0, 0, 0)), P((1, 0), (-1, 0, 0)), P((1, 0), (0, 1, 0)),
             P((1, -1), (-1, 0, 0), m), P((0, 1), (0, 0, 0), m),
             P((1, -1), (0, 1, 1), m), P((1, -1), (0, 1, 0), m))
    inv = INV_4PT + (("msq",) if massive else ())
    # vertices A=0(p1) B=1(p2) C=2 D=3 E=4(p3) F=5(p4)
    edges = ((0, 1), (3, 0), (1, 2), (5, 3), (2, 3), (4, 5), (2, 4))
    return Topology(name="dbox_planar" + ("_m" if massive else "_0"), loops=2, n_ext=3, props=props,
                    invariants=inv, gram=_gram_4pt(), edges=edges, ext_at=(0, 1, 4, 5))


def double_box_nonplanar(massive: bool = True) -> Topology:
    """Non-planar (crossed) double box with the routing of the paper's Eq. (27), outgoing p3, p4 rewritten as
    incoming.  q = k1, k1+p1, k1-p2, k1-k2+p1, k2, k2-p1-p2-p3, k1-k2+p1+p3; lines 4..7 massive."""
    m = "msq" if massive else None
    P = Propagator
    props = (P((1, 0), (0, 0, 0)), P((1, 0), (1, 0, 0)), P((1, 0), (0, -1, 0)),
             P((1, -1), (1, 0, 0), m), P((0, 1), (0, 0, 0), m),
             P((0, 1), (-1, -1, -1), m), P((1, -1), (1, 0, 1), m))
    inv = INV_4PT + (("msq",) if massive else ())
    # vertices A=0(p1) B=1(p2) C=2 D=3(p3) E=4(p4) F=5
    edges = ((1, 0), (0, 2), (5, 1), (2, 3), (2, 4), (4, 5), (3, 5))
    return Topology(name="dbox_nonplanar" + ("_m" if massive else "_0"), loops=2, n_ext=3, props=props,
                    invariants=inv, gram=_gram_4pt(), edges=edges, ext_at=(0, 1, 3, 4))


def kinematics(topo: Topology, **values: float) -> np.ndarray:
    """Kinematics vector in the topology's invariant order; unspecified invariants (external masses) are 0."""
    unknown = set(values) - set(topo.invariants)
    if unknown:
        raise KeyError(f"unknown invariants {sorted(unknown)} for {topo.name}")
    return np.array([float(values.get(n, 0.0)) for n in topo.invariants], dtype=np.float64)


@dataclass(frozen=True)
class Workload:
    """One benchmark / parity configuration."""
    name: str
    topology: Topology
    point: Dict[str, float]            # kinematic point
    order_min: int                     # lowest Laurent order wanted
    order_max: int                     # highest Laurent order wanted
    n_shifts: int
    lattice_log2: Tuple[int, ...]      # lattice sizes: largest prime below 2**k for k in this tuple
    transform_r: int = 3               # Korobov periodising transform order
    lam: float = 0.5                   # contour-deformation parameter lambda
    rel_tol: float = 1e-3
    seed: int = 0
    strategy: str = "iterated"         # sector decomposition strategy ("iterated" or "geometric")

    @property
    def kin(self) -> np.ndarray:
        return kinematics(self.topology, **self.point)


CONFIG0 = Workload("massless_box_euclid", box(False), dict(s=-3.0, t=-2.0), -2, 0, 8, (16,), 3, 0.0)
CONFIG1 = Workload("massive_box_physical", box(True), dict(s=5.0, t=-1.5, msq=1.0), 0, 0, 16,
                   tuple(range(16, 25)), 3, 0.5)
CONFIG2 = Workload("planar_dbox_physical", double_box_planar(True), dict(s=6.0, t=-2.0, msq=1.0), -2, 0, 16,
                   tuple(range(16, 27)), 3, 0.5)
CONFIG3 = Workload("nonplanar_dbox_physical", double_box_nonplanar(True), dict(s=6.0, t=-2.0, msq=1.0), -2, 0,
                   16, tuple(range(16, 27)), 3, 0.5)
CONFIGS = (CONFIG0, CONFIG1, CONFIG2, CONFIG3)

# The kinematic point of the paper's two-loop examples in the physical region (Sec. IV, gg -> HH): p1^2 = p2^2
# = 0, p3^2 = p4^2 = M_H^2, s = 160000 GeV^2, t = -6000 GeV^2, in units of M_t = 172 GeV (M_t^2 = 1 on the four
# massive lines); M_H = 125 GeV.
M_T_GEV, M_H_GEV = 172.0, 125.0
PAPER_HH_POINT = dict(s=160000.0 / M_T_GEV ** 2, t=-6000.0 / M_T_GEV ** 2, pp3=(M_H_GEV / M_T_GEV) ** 2,
                      pp4=(M_H_GEV / M_T_GEV) ** 2, msq=1.0)


def shifts(seed: int, m: int, dim: int = 6) -> np.ndarray:
    """m random shift vectors, uniform in [0,1)^dim, from numpy's PCG64 seeded by `seed` (paper Sec. III,
    step 1 of the shifted-lattice algorithm draws them; here they are passed in as inputs)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.random((m, dim), dtype=np.float64)


def serving_arrivals(n_requests: int, rate_per_s: float = 50.0, seed: int = 0):
    """Poisson arrival stream for the serving workload: (arrival_time_s, config_index, s, t) tuples with
    s ~ U[4.5, 12], t ~ U[-4, -0.5] and the config drawn uniformly from the four integrals."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_per_s, size=n_requests)
    times = np.cumsum(gaps)
    cfg = rng.integers(0, 4, size=n_requests)
    s = rng.uniform(4.5, 12.0, size=n_requests)
    t = rng.uniform(-4.0, -0.5, size=n_requests)
    return [(float(a), int(c), float(x), float(y)) for a, c, x, y in zip(times, cfg, s, t)]


# The Euclidean points of the paper's Table 2 (Sec. IV): the massless planar double box with two off-shell legs,
# s = t = u = -2/3 (so that pp1 + pp2 + pp3 + pp4 = -2), one point per pair of off-shell legs.
PAPER_IB_POINTS = {
    "-1,0,0,-1": dict(s=-2.0 / 3.0, t=-2.0 / 3.0, pp1=-1.0, pp4=-1.0),
    "0,-1,0,-1": dict(s=-2.0 / 3.0, t=-2.0 / 3.0, pp2=-1.0, pp4=-1.0),
    "0,0,-1,-1": dict(s=-2.0 / 3.0, t=-2.0 / 3.0, pp3=-1.0, pp4=-1.0),
}

# Table 2's first point as a benchmark workload (the iterated strategy does not terminate for this integral).
PAPER_IB = Workload("massless_dbox_euclid_table2", double_box_planar(False), PAPER_IB_POINTS["-1,0,0,-1"], -4, 0,
                    16, tuple(range(16, 27)), 3, 0.0, strategy="geometric")

# The paper's one-loop example I_A (Sec. IV, gg -> HH box with four top-quark lines): on-shell gluons
# p1^2 = p2^2 = 0, Higgs legs p3^2 = p4^2 = M_H^2 (outgoing), t = (p2 - p3)^2 = -6000 GeV^2 fixed and a scan of
# s = (p1 + p2)^2 from 70000 to 500000 GeV^2.  Its propagators k, k+p1, k+p1-p4, k-p2 are box(True) with the
# incoming legs (q1, q2, q3, q4) = (p1, -p4, -p3, p2), so box(True)'s s = (q1+q2)^2 is the paper's t, its
# t = (q2+q3)^2 the paper's s, and pp2 = pp3 = M_H^2.  Units M_t = 1.  The paper's measure d^Dk/(2 pi)^D makes
# I_A = i/(16 pi^2) I at eps^0 (in GeV^-4 after dividing by M_t^4).
PAPER_IA_T_GEV2 = -6000.0
PAPER_IA_S_RANGE_GEV2 = (70000.0, 500000.0)


def paper_ia_point(s_gev2: float) -> Dict[str, float]:
    """Kinematic point of box(True) for the paper's I_A at s = s_gev2 (GeV^2)."""
    mh2 = (M_H_GEV / M_T_GEV) ** 2
    return dict(s=PAPER_IA_T_GEV2 / M_T_GEV ** 2, t=s_gev2 / M_T_GEV ** 2, pp2=mh2, pp3=mh2, msq=1.0)
