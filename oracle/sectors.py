"""Sector decomposition in exact arithmetic (oracle; test use only).

Paper Sec. II.
  * Primary sectors, Eqs. (3)-(6): in sector l set x_l = 1 and x_j = t_j (j != l); the delta function and
    homogeneity of U (degree L) and F (degree L+1) remove x_l, leaving the integrand of Eq. (6) on [0,1]^{N-1}
    with t_j^{nu_j - 1}.
  * Iterated decomposition, Eqs. (7)-(9): while U_l or F_l (after pulling out their monomial factors) vanish
    at t = 0, pick a set S' of variables on which one of them vanishes identically and split the sector into
    |S'| subsectors t_j -> t_k t_j (j in S' \\ {k}, Jacobian t_k^{|S'|-1}).  S' is the smallest such set,
    ties broken by the lexicographically smallest index tuple.  A depth cap turns non-termination into an
    error.
  * Geometric decomposition (the strategy the paper prefers, Sec. II after Eq. 9; Kaneko and Ueda): by the
    Cheng-Wu theorem the delta function may keep x_N = 1 alone, leaving x_1..x_{N-1} in (0, inf).  In the
    logarithms u_j = log x_j, the normal fan of the Newton polytope of U F (exponents of x_1..x_{N-1}) covers
    R^{N-1}; on a simplicial cone with integer generators m_1..m_{N-1} (u = -sum_i m_i log y_i, y in (0,1]) every
    monomial x^v becomes prod_i y_i^{-<m_i, v>}, and the term v* of U (of F) maximising <m, .> over the whole
    cone is the same for all of it, so U = prod_i y_i^{-<m_i, vU*>} Ut(y) with Ut(0) = c_{vU*} != 0.  The
    measure prod_j x_j^{nu_j - 1} dx_j becomes |det m| prod_i y_i^{-<m_i, nu> - 1} dy_i.  Cones of the fan with
    more generators than the dimension are split by the pulling triangulation.  Ordering rules that fix the
    sector list: facets are named by their primitive outer normals, vertices are visited in lexicographic
    order, a vertex cone's generators are listed lexicographically, the pulling apex is the first generator,
    the facets of a cone are visited in lexicographic order of their generator index tuples, and a sector's
    variables follow its generators' lexicographic order.  scipy's convex hull only proposes the polytope's
    facets; each is rebuilt and checked in exact arithmetic.
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
from math import gcd
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


# ---------------------------------------------------------------- geometric strategy: exact linear algebra
def _q_rank(rows) -> int:
    """Rank of a list of rational vectors (Gaussian elimination in Fractions)."""
    A = [[Fraction(x) for x in r] for r in rows]
    rank, ncol = 0, len(A[0]) if A else 0
    for c in range(ncol):
        p = next((i for i in range(rank, len(A)) if A[i][c] != 0), None)
        if p is None:
            continue
        A[rank], A[p] = A[p], A[rank]
        for i in range(rank + 1, len(A)):
            f = A[i][c] / A[rank][c]
            if f:
                A[i] = [a - f * b for a, b in zip(A[i], A[rank])]
        rank += 1
    return rank


def _q_det(rows) -> Fraction:
    A = [[Fraction(x) for x in r] for r in rows]
    n, det = len(A), Fraction(1)
    for c in range(n):
        p = next((i for i in range(c, n) if A[i][c] != 0), None)
        if p is None:
            return Fraction(0)
        if p != c:
            A[c], A[p] = A[p], A[c]
            det = -det
        det *= A[c][c]
        for i in range(c + 1, n):
            f = A[i][c] / A[c][c]
            if f:
                A[i] = [a - f * b for a, b in zip(A[i], A[c])]
    return det


def _cross(rows):
    """Generalised cross product of k-1 vectors in Q^k: the form x -> det(rows; x), by cofactors."""
    k = len(rows) + 1
    return [(-1) ** (k - 1 + j) * _q_det([[r[c] for c in range(k) if c != j] for r in rows]) for j in range(k)]


def _primitive(v):
    den = 1
    for x in v:
        den = den * Fraction(x).denominator // gcd(den, Fraction(x).denominator)
    w = [int(Fraction(x) * den) for x in v]
    g = 0
    for x in w:
        g = gcd(g, abs(x))
    return tuple(x // g for x in w)


def _independent(vectors, want):
    """Indices of the first `want` linearly independent vectors (greedy, in order)."""
    chosen = []
    for i, v in enumerate(vectors):
        if _q_rank([vectors[j] for j in chosen] + [v]) == len(chosen) + 1:
            chosen.append(i)
            if len(chosen) == want:
                break
    return chosen


def _polytope_facets(points):
    """[(primitive outer normal m, h)] with <m, p> <= h on all points, equality on a facet."""
    import numpy as np
    from scipy.spatial import ConvexHull

    d = len(points[0])
    if d == 1:
        return [((-1,), -min(p[0] for p in points)), ((1,), max(p[0] for p in points))]
    hull = ConvexHull(np.array(points, dtype=float))
    out = {}
    for eq in hull.equations:
        on = [p for p in points if abs(sum(a * b for a, b in zip(p, eq[:-1])) + eq[-1]) <= 1e-7]
        diffs = [[a - b for a, b in zip(p, on[0])] for p in on[1:]]
        basis = _independent(diffs, d - 1)
        if len(basis) != d - 1 or _q_rank(diffs) != d - 1:
            raise DecompositionError("degenerate facet")
        m = _primitive(_cross([diffs[i] for i in basis]))
        if sum(a * b for a, b in zip(m, eq[:-1])) < 0:
            m = tuple(-x for x in m)
        h = sum(a * b for a, b in zip(m, on[0]))
        vals = [sum(a * b for a, b in zip(m, p)) for p in points]
        if max(vals) != h or sorted(p for p, v in zip(points, vals) if v == h) != sorted(on):
            raise DecompositionError("inexact facet")
        out[m] = h
    return sorted(out.items())


def _facets_of_cone(gens, idx, dim):
    """Facets of the dim-dimensional cone spanned by gens[idx] (sorted tuples of indices), found in coordinates
    of a basis of its span: the cofactor form of every dim - 1 independent generators must have one sign."""
    basis = [idx[i] for i in _independent([gens[i] for i in idx], dim)]
    # coordinates c with gens[i] = sum_b c_b gens[basis[b]]: solve by Cramer's rule on `dim` independent rows
    cols = _independent([[gens[b][j] for b in basis] for j in range(len(gens[0]))], dim)
    Bm = [[gens[b][j] for b in basis] for j in cols]            # dim x dim, invertible
    detB = _q_det(Bm)

    def coords(g):
        rhs = [g[j] for j in cols]
        return [_q_det([[rhs[r] if c == b else Bm[r][c] for c in range(dim)] for r in range(dim)]) / detB
                for b in range(dim)]

    C = {i: coords(gens[i]) for i in idx}
    found = set()
    for comb in combinations(idx, dim - 1):
        if _q_rank([C[i] for i in comb]) != dim - 1:
            continue
        form = _cross([C[i] for i in comb])
        vals = {i: sum(a * b for a, b in zip(form, C[i])) for i in idx}
        if all(v >= 0 for v in vals.values()) or all(v <= 0 for v in vals.values()):
            found.add(tuple(i for i in idx if vals[i] == 0))
    return sorted(found)


def _pulling(gens, idx, dim):
    if len(idx) == dim:
        return [tuple(idx)]
    out = []
    for face in _facets_of_cone(gens, idx, dim):
        if idx[0] not in face:
            out += [(idx[0],) + c for c in _pulling(gens, list(face), dim - 1)]
    return out


def geometric_sectors(U, F, nu: List[int], eU, eF):
    """Sectors of the geometric strategy (module docstring), final: Ut and Ft have nonzero constant terms."""
    n = len(nu)
    d = n - 1
    for poly in (U, F):
        if len({sum(e) for e in poly}) != 1:
            raise DecompositionError("polynomial is not homogeneous")
    points = sorted({tuple(a + b for a, b in zip(eu[:d], ef[:d])) for eu in U for ef in F})
    facets = _polytope_facets(points)
    secs = []
    for p in points:
        gens = sorted(m for m, h in facets if sum(a * b for a, b in zip(m, p)) == h)
        if len(gens) < d or _q_rank(gens) != d:
            continue
        for cone in _pulling(gens, list(range(len(gens))), d):
            ms = [gens[i] for i in sorted(cone)]
            D = abs(_q_det(ms))
            new, shift = [], []
            for poly in (U, F):
                pair = {e: [sum(m[j] * e[j] for j in range(d)) for m in ms] for e in poly}
                top = [max(v[i] for v in pair.values()) for i in range(d)]
                if sum(1 for v in pair.values() if v == top) != 1:
                    raise DecompositionError("cone not inside one vertex's normal cone")
                new.append({tuple(t - x for t, x in zip(top, v)): poly[e] for e, v in pair.items()})
                shift.append([-t for t in top])
            A = [-sum(m[j] * nu[j] for j in range(d)) - 1 + shift[0][i] * eU[0] - shift[1][i] * eF[0]
                 for i, m in enumerate(ms)]
            B = [shift[0][i] * eU[1] - shift[1][i] * eF[1] for i in range(d)]
            secs.append(Sector(("geometric", p, tuple(ms)), A, B, new[0], new[1], D))
    return secs


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


def decompose(topo, zero_invariants=(), strategy="iterated", max_depth=40, allow_higher_poles=False):
    """Leaf sectors of `topo` for the kinematic class in which `zero_invariants` vanish.  Exponents alpha <= -2
    are refused unless allow_higher_poles (for the Taylor-subtraction oracle, oracle.taylor)."""
    U, F = fy.symanzik_momentum(topo)
    zero = set(zero_invariants)
    U = drop_zero_invariants(U, zero)
    F = drop_zero_invariants(F, zero)
    nu = [p.nu for p in topo.props]
    eU, eF = exponents_eU_eF(sum(nu), topo.loops)
    leaves: List[Sector] = []
    if strategy == "geometric":
        leaves = geometric_sectors(U, F, nu, eU, eF)
        start = []
    elif strategy == "iterated":
        start = primary_sectors(U, F, nu)
    elif strategy == "hepp":
        start = hepp_sectors(U, F, nu)
    else:
        raise ValueError(strategy)
    for sec in start:
        _iterate(sec, eU, eF, 0, max_depth, leaves)
    for sec in leaves:
        for a, b in zip(sec.A, sec.B):
            if a <= -2 and not allow_higher_poles:
                raise DecompositionError(f"exponent alpha={a} <= -2 needs higher Taylor subtraction")
            if a <= -1 and b == 0:
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
