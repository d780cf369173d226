"""Symanzik polynomials U and F of a loop integral, in exact rational arithmetic (oracle; test use only).

Paper Sec. II, Eq. (2): after Feynman parametrisation the integral is a projective integral of
U^{N_nu-(L+1)D/2} / F^{N_nu-LD/2}; U and F follow "from the momentum representation, or ... the topology of
the Feynman graph".  Both constructions are written here; tests check that they agree.

Momentum representation.  With D_j = -q_j^2 + m_j^2 and q_j = sum_a A_ja k_a + r_j (r_j a combination of the
external momenta):
    sum_j x_j (q_j^2 - m_j^2) = sum_ab M_ab k_a.k_b + 2 sum_a k_a.Q_a + J,
    M_ab = sum_j x_j A_ja A_jb,  Q_a = sum_j x_j A_ja r_j,  J = sum_j x_j (r_j^2 - m_j^2),
    U = det M,   F = sum_ab adj(M)_ab Q_a.Q_b - J det M.
For the massless bubble this gives U = x1+x2, F = -p^2 x1 x2 (positive for Euclidean p^2 < 0).

Polynomials are dicts {exponent tuple: LinearForm}; a LinearForm is a dict {invariant name: Fraction},
with the key "1" for a pure number.
"""
from __future__ import annotations

from fractions import Fraction
from itertools import combinations
from typing import Dict, List, Tuple

ONE = "1"


# ---------------------------------------------------------------- linear forms in the invariants
def lf_const(c) -> Dict[str, Fraction]:
    c = Fraction(c)
    return {} if c == 0 else {ONE: c}


def lf_add(a, b):
    out = dict(a)
    for k, v in b.items():
        out[k] = out.get(k, Fraction(0)) + v
        if out[k] == 0:
            del out[k]
    return out


def lf_scale(a, c):
    c = Fraction(c)
    return {} if c == 0 else {k: v * c for k, v in a.items()}


def lf_is_const(a) -> bool:
    return all(k == ONE for k in a)


def lf_mul(a, b):
    """Product of two linear forms, defined only when one of them is a pure number."""
    if lf_is_const(a):
        return lf_scale(b, a.get(ONE, Fraction(0)))
    if lf_is_const(b):
        return lf_scale(a, b.get(ONE, Fraction(0)))
    raise ValueError("product of two non-constant linear forms is not linear")


def lf_eval(a, values: Dict[str, float]) -> float:
    return float(sum(float(v) * (1.0 if k == ONE else float(values[k])) for k, v in a.items()))


# ---------------------------------------------------------------- sparse polynomials in x_1..x_n
def p_zero():
    return {}


def p_var(n, j, coef=1):
    e = [0] * n
    e[j] = 1
    return {tuple(e): lf_const(coef)} if coef != 0 else {}


def p_const(n, lf):
    return {(0,) * n: dict(lf)} if lf else {}


def p_add(a, b):
    out = {k: dict(v) for k, v in a.items()}
    for k, v in b.items():
        s = lf_add(out.get(k, {}), v)
        if s:
            out[k] = s
        elif k in out:
            del out[k]
    return out


def p_scale(a, c):
    return {k: lf_scale(v, c) for k, v in a.items() if c != 0}


def p_mul(a, b):
    out = {}
    for ka, va in a.items():
        for kb, vb in b.items():
            k = tuple(x + y for x, y in zip(ka, kb))
            s = lf_add(out.get(k, {}), lf_mul(va, vb))
            if s:
                out[k] = s
            elif k in out:
                del out[k]
    return out


def p_mul_lf(a, lf):
    out = {}
    for k, v in a.items():
        s = lf_mul(v, lf)
        if s:
            out[k] = s
    return out


def p_det(M):
    """Determinant by Laplace expansion along the first row (L <= 3 here)."""
    n = len(M)
    if n == 1:
        return M[0][0]
    acc = {}
    for c in range(n):
        minor = [[M[r][cc] for cc in range(n) if cc != c] for r in range(1, n)]
        term = p_mul(M[0][c], p_det(minor))
        acc = p_add(acc, term if c % 2 == 0 else p_scale(term, -1))
    return acc


def p_adj(M):
    n = len(M)
    if n == 1:
        return [[p_const(len(next(iter(M[0][0]))) if M[0][0] else 0, lf_const(1))]]
    adj = [[None] * n for _ in range(n)]
    for r in range(n):
        for c in range(n):
            minor = [[M[i][j] for j in range(n) if j != r] for i in range(n) if i != c]
            d = p_det(minor)
            adj[r][c] = d if (r + c) % 2 == 0 else p_scale(d, -1)
    return adj


# ---------------------------------------------------------------- U, F from the momentum representation
def symanzik_momentum(topo):
    """(U, F) of `topo` (a workloads.Topology) as exact polynomials in x_1..x_N."""
    n, L, E = topo.n_props, topo.loops, topo.n_ext
    x = [p_var(n, j) for j in range(n)]
    M = [[p_zero() for _ in range(L)] for _ in range(L)]
    Q = [[p_zero() for _ in range(E)] for _ in range(L)]  # Q[a][e]: coefficient polynomial of p_e in Q_a
    J = p_zero()
    for j, pr in enumerate(topo.props):
        for a in range(L):
            for b in range(L):
                c = pr.k[a] * pr.k[b]
                if c:
                    M[a][b] = p_add(M[a][b], p_scale(x[j], c))
            for e in range(E):
                c = pr.k[a] * pr.p[e]
                if c:
                    Q[a][e] = p_add(Q[a][e], p_scale(x[j], c))
        r2 = {}
        for e in range(E):
            for f in range(E):
                c = pr.p[e] * pr.p[f]
                if c:
                    r2 = lf_add(r2, lf_scale(topo.gram_form(e, f), c))
        if pr.mass is not None:
            r2 = lf_add(r2, {pr.mass: Fraction(-1)})
        J = p_add(J, p_mul_lf(x[j], r2))
    U = p_det(M)
    adj = p_adj(M) if L > 1 else [[p_const(n, lf_const(1))]]
    F = p_zero()
    for a in range(L):
        for b in range(L):
            for e in range(E):
                for f in range(E):
                    poly = p_mul(p_mul(adj[a][b], Q[a][e]), Q[b][f])
                    if poly:
                        F = p_add(F, p_mul_lf(poly, topo.gram_form(e, f)))
    F = p_add(F, p_scale(p_mul(J, U), -1))
    return U, F


# ---------------------------------------------------------------- U, F from the graph
def _components(n_vertices, edges):
    parent = list(range(n_vertices))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for u, v in edges:
        parent[find(u)] = find(v)
    return [find(v) for v in range(n_vertices)]


def symanzik_graph(topo):
    """(U, F) from spanning trees and spanning 2-forests (Kirchhoff; Bogner-Weinzierl):
        U = sum_{trees T} prod_{e not in T} x_e,
        F = sum_{2-forests (T1,T2)} prod_{e not in T1 u T2} x_e * (-(P_{T1})^2) + U sum_e x_e m_e^2,
    with P_{T1} the external momentum flowing into T1 (all momenta incoming)."""
    n = topo.n_props
    nv = 1 + max(max(e) for e in topo.edges)
    E = topo.n_ext
    # incoming external momenta per vertex as coefficient vectors over p_1..p_E (the last leg is -sum)
    ext_vec = [[0] * E for _ in range(nv)]
    for leg, v in enumerate(topo.ext_at):
        if leg < E:
            ext_vec[v][leg] += 1
        else:
            for e in range(E):
                ext_vec[v][e] -= 1
    U = p_zero()
    F0 = p_zero()
    L = topo.loops
    for cut in combinations(range(n), L):
        kept = [topo.edges[e] for e in range(n) if e not in cut]
        comp = _components(nv, kept)
        if len(set(comp)) == 1:
            mono = [0] * n
            for e in cut:
                mono[e] = 1
            U = p_add(U, {tuple(mono): lf_const(1)})
    for cut in combinations(range(n), L + 1):
        kept = [topo.edges[e] for e in range(n) if e not in cut]
        comp = _components(nv, kept)
        roots = sorted(set(comp))
        if len(roots) != 2:
            continue
        # forest condition: a spanning 2-forest has exactly nv-2 edges and no cycle
        if len(kept) != nv - 2:
            continue
        P = [0] * E
        for v in range(nv):
            if comp[v] == roots[0]:
                for e in range(E):
                    P[e] += ext_vec[v][e]
        P2 = {}
        for e in range(E):
            for f in range(E):
                c = P[e] * P[f]
                if c:
                    P2 = lf_add(P2, lf_scale(topo.gram_form(e, f), c))
        mono = [0] * n
        for e in cut:
            mono[e] = 1
        if P2:
            F0 = p_add(F0, {tuple(mono): lf_scale(P2, -1)})
    mass = p_zero()
    for j, pr in enumerate(topo.props):
        if pr.mass is not None:
            mono = [0] * n
            mono[j] = 1
            mass = p_add(mass, {tuple(mono): {pr.mass: Fraction(1)}})
    F = p_add(F0, p_mul(U, mass))
    return U, F


def substitute_invariants(poly, values: Dict[str, Fraction]):
    """Replace the invariants by exact numbers; returns {exps: Fraction} without zero terms."""
    out = {}
    for k, lf in poly.items():
        v = sum((c * (Fraction(1) if name == ONE else Fraction(values[name])) for name, c in lf.items()),
                Fraction(0))
        if v != 0:
            out[k] = v
    return out
