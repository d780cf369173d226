"""Sector decomposition in exact arithmetic (oracle; test use only).

Paper Sec. II.
  * Primary sectors, Eqs. (3)-(6): in sector l set x_l = 1 and x_j = t_j (j != l); the delta function and
    homogeneity of U (degree L) and F (degree L+1) remove x_l, leaving the integrand of Eq. (6) on [0,1]^{N-1}
    with t_j^{nu_j - 1}.
  * Iterated decomposition, Eqs. (7)-(9): while U_l or F_l (after pulling out their monomial factors) vanish
    at t = 0, pick a set S' of variables on which one of them vanishes identically and split the sector into
    |S'| subsectors t_j -> t_k t_j (j in S' \\ {k}, Jacobian t_k^{|S'|-1}).  S' is the smallest such set,
    ties broken by the lexicographically smallest index tuple.  A depth cap turns non-termination into an
    error.  The geometric strategy that the paper prefers (Sec. II, after Eq. 9) is not used.
  * Exponents, Eq. (9): each leaf is D * prod_j t_j^{A_j + B_j eps} * Ut^{eU(eps)} / Ft^{eF(eps)} with
    eU = N_nu - (L+1)(2 - eps), eF = N_nu - L(2 - eps); the monomials pulled out of U and F are folded into
    A and B.  Ut and Ft keep their constant term (they are C(1+H) and C'(1+H') of Eqs. (7)-(8)).
  * Hepp sectors: a second strategy (all N! orderings of the x_j, each ordering mapped to the cube and then
    refined by the same iteration) used to test that the total does not depend on the decomposition.

Coefficients stay exact linear forms in the kinematic invariants (oracle.feynman), so a table is valid for every
kinematic point of its zero pattern.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from fractions import Fraction
from itertools import combinations, permutations
from typing import Dict, List, Tuple

from . import feynman as fy


class DecompositionError(RuntimeError):
    pass


@dataclass
class Sector:
    label: Tuple                       # provenance (primary index / ordering, then split choices)
    A: List[int]                       # integer part of the exponent of t_j
    B: List[int]                       # eps part of the exponent of t_j
    U: Dict[Tuple[int, ...], dict]     # Ut: exps -> linear form
    F: Dict[Tuple[int, ...], dict]     # Ft
    D: Fraction = Fraction(1)

    @property
    def dim(self) -> int:
        return len(self.A)

    @property
    def singular(self) -> List[int]:
        return [j for j, a in enumerate(self.A) if a == -1]


def drop_zero_invariants(poly, zero: set):
    """Remove invariants that vanish in the kinematic class (e.g. massless external legs)."""
    out = {}
    for k, lf in poly.items():
        lf2 = {n: c for n, c in lf.items() if n not in zero}
        if lf2:
            out[k] = lf2
    return out


def _min_exps(poly, s):
    return [min(e[j] for e in poly) for j in range(s)]


def _divide_monomial(poly, b):
    return {tuple(x - y for x, y in zip(e, b)): c for e, c in poly.items()}


def _has_constant(poly, s):
    return (0,) * s in poly


def _vanishes_on(poly, S):
    """True when every term of poly contains at least one variable of S (poly|_{t_S = 0} == 0)."""
    return all(any(e[j] > 0 for j in S) for e in poly)


def _substitute(poly, S, k):
    """t_j -> t_k t_j for j in S \\ {k}: exponent e_k gains sum_{j in S\\{k}} e_j."""
    out = {}
    for e, c in poly.items():
        e2 = list(e)
        e2[k] += sum(e[j] for j in S if j != k)
        e2 = tuple(e2)
        if e2 in out:  # the map is injective; a collision would mean a bug
            raise DecompositionError("monomial collision in substitution")
        out[e2] = c
    return out


def _iterate(sec: Sector, eU, eF, depth, max_depth, out):
    s = sec.dim
    bU, bF = _min_exps(sec.U, s), _min_exps(sec.F, s)
    U, F = _divide_monomial(sec.U, bU), _divide_monomial(sec.F, bF)
    A = [a + bu * eU[0] - bf * eF[0] for a, bu, bf in zip(sec.A, bU, bF)]
    B = [b + bu * eU[1] - bf * eF[1] for b, bu, bf in zip(sec.B, bU, bF)]
    if _has_constant(U, s) and _has_constant(F, s):
        out.append(Sector(sec.label, A, B, U, F, sec.D))
        return
    if depth >= max_depth:
        raise DecompositionError(f"iterated decomposition exceeded depth {max_depth} in sector {sec.label}")
    chosen = None
    for size in range(1, s + 1):
        for S in combinations(range(s), size):
            if _vanishes_on(U, S) or _vanishes_on(F, S):
                chosen = S
                break
        if chosen:
            break
    for k in chosen:
        A2, B2 = list(A), list(B)
        A2[k] += sum(A[j] for j in chosen if j != k) + len(chosen) - 1
        B2[k] += sum(B[j] for j in chosen if j != k)
        sub = Sector(sec.label + ((chosen, k),), A2, B2, _substitute(U, chosen, k), _substitute(F, chosen, k),
                     sec.D)
        _iterate(sub, eU, eF, depth + 1, max_depth, out)


def exponents_eU_eF(n_nu: int, loops: int):
    """(eU0, eU1), (eF0, eF1) with U^{eU0 + eU1 eps} / F^{eF0 + eF1 eps}, D = 4 - 2 eps (Eq. 2)."""
    return (n_nu - 2 * (loops + 1), loops + 1), (n_nu - 2 * loops, loops)


def primary_sectors(U, F, nu: List[int]):
    """Eqs. (3)-(6): x_l = 1, x_j = t_j; returns unrefined sectors with A_j = nu_j - 1."""
    n = len(nu)
    secs = []
    for l in range(n):
        keep = [j for j in range(n) if j != l]

        def restrict(poly):
            out = {}
            for e, c in poly.items():
                e2 = tuple(e[j] for j in keep)
                if e2 in out:
                    raise DecompositionError("polynomial is not homogeneous")
                out[e2] = c
            return out

        secs.append(Sector((l,), [nu[j] - 1 for j in keep], [0] * (n - 1), restrict(U), restrict(F)))
    return secs


def hepp_sectors(U, F, nu: List[int]):
    """All orderings x_{p0} >= x_{p1} >= ... : x_{p0} = 1, x_{pk} = u_1 ... u_k (k >= 1), Jacobian
    prod_i u_i^{N-1-i}; variables are u_1..u_{N-1}."""
    n = len(nu)
    secs = []
    for perm in permutations(range(n)):
        def mapped(poly):
            out = {}
            for e, c in poly.items():
                u = tuple(sum(e[perm[k]] for k in range(i, n)) for i in range(1, n))
                if u in out:
                    raise DecompositionError("collision in Hepp map")
                out[u] = c
            return out

        A = [sum(nu[perm[k]] - 1 for k in range(i, n)) + (n - 1 - i) for i in range(1, n)]
        secs.append(Sector(("hepp",) + perm, A, [0] * (n - 1), mapped(U), mapped(F)))
    return secs


def decompose(topo, zero_invariants=(), strategy="iterated", max_depth=40):
    """Leaf sectors of `topo` for the kinematic class in which `zero_invariants` vanish."""
    U, F = fy.symanzik_momentum(topo)
    zero = set(zero_invariants)
    U = drop_zero_invariants(U, zero)
    F = drop_zero_invariants(F, zero)
    nu = [p.nu for p in topo.props]
    eU, eF = exponents_eU_eF(sum(nu), topo.loops)
    if strategy == "iterated":
        start = primary_sectors(U, F, nu)
    elif strategy == "hepp":
        start = hepp_sectors(U, F, nu)
    else:
        raise ValueError(strategy)
    leaves: List[Sector] = []
    for sec in start:
        _iterate(sec, eU, eF, 0, max_depth, leaves)
    for sec in leaves:
        for a, b in zip(sec.A, sec.B):
            if a <= -2:
                raise DecompositionError(f"exponent alpha={a} <= -2 needs higher Taylor subtraction")
            if a == -1 and b == 0:
                raise DecompositionError("unregulated endpoint singularity (alpha=-1, beta=0)")
    return leaves


def zero_invariants_of(topo, point: Dict[str, float]):
    return tuple(n for n in topo.invariants if float(point.get(n, 0.0)) == 0.0)


def canonical(sectors, values=None):
    """Order-independent description of a decomposition, for exact comparison between implementations:
    a sorted tuple of (A, B, sorted Ut terms, sorted Ft terms) with exact coefficients."""
    def poly_key(poly):
        return tuple(sorted((e, tuple(sorted(lf.items()))) for e, lf in poly.items()))

    return tuple(sorted((tuple(s.A), tuple(s.B), poly_key(s.U), poly_key(s.F)) for s in sectors))
