"""Sector-table compiler: loop integral -> Symanzik polynomials -> sector decomposition -> binary sector table.

This is the host-side front end of the library (offline, not on the GPU hot path).  It turns an integral of the
form of the paper's Eq. (1) into the table that `qmc_prepare` / `qmc_load_sectors` read:

  * Feynman parametrisation (Sec. II, Eq. 2):  sum_j x_j (q_j^2 - m_j^2) = k^T M k + 2 k.Q + J gives
    U = det M and F = Q^T adj(M) Q - J det M (propagators -q^2 + m^2, all momenta incoming);
  * primary sectors (Eqs. 3-6): x_l = 1, the remaining x_j become t_j in [0,1], monomial t_j^{nu_j-1};
  * iterated decomposition (Eqs. 7-9): while U or F fails to have a nonzero constant term after its monomial
    factor is pulled out, take the smallest variable set S (lexicographically first) on which one of them
    vanishes identically and split into |S| subsectors t_j -> t_k t_j (j in S, j != k), Jacobian t_k^{|S|-1};
  * or the geometric decomposition the paper prefers (Sec. II, after Eq. 9; Kaneko and Ueda): x_N = 1, the other
    x_j range over (0, inf), and the normal fan of the Newton polytope of U F, triangulated into unimodular or
    simplicial cones, splits that range into sectors x_j = prod_i y_i^{-m_ij} (m_i the cone's generators),
    y in (0, 1]^{N-1}, on each of which U and F factorise with a nonzero constant term;
  * exponents of Eq. (9): prod_j t_j^{A_j + B_j eps} with A, B collecting nu_j - 1, the Jacobians and the
    monomials of U^{eU0 + eU1 eps} / F^{eF0 + eF1 eps}, eU = N_nu - (L+1)(2 - eps), eF = N_nu - L(2 - eps).

Polynomials are numpy arrays: exponents int32[T, n] and coefficients float64[T, 1 + K], column 0 a pure number
and column 1 + k the coefficient of kinematic invariant k, so one table serves every kinematic point of its
zero pattern.  All coefficients that arise are dyadic rationals and exact in float64.

Binary table (little-endian, 8-byte aligned), read by csrc/qmc_prepare.cpp:
  header   "QMCSEC01", int32 version, n_sectors, dim, loops, n_props, n_nu, n_inv, eU0, eU1, eF0, eF1,
           header_bytes, 2 x int32 reserved; int32 nu[n_props] (padded to 8 bytes); char names[n_inv][16]
  sector   int32 nU, nF; int32 A[dim], B[dim] (padded to 8 bytes); double D;
           nU terms then nF terms, each: uint8 e[8]; double c[1 + n_inv]
"""
from __future__ import annotations

import math
import struct
from dataclasses import dataclass
from fractions import Fraction
from itertools import combinations, permutations
from typing import List, Sequence, Tuple

import numpy as np

MAGIC = b"QMCSEC01"
VERSION = 1
MAX_DIM = 6


class TableError(RuntimeError):
    pass


# ------------------------------------------------------------------------------------------- polynomials
@dataclass
class Poly:
    e: np.ndarray  # int32 [T, n]
    c: np.ndarray  # float64 [T, 1 + K]

    @staticmethod
    def zero(n, K):
        return Poly(np.zeros((0, n), np.int32), np.zeros((0, 1 + K)))

    @staticmethod
    def monomial(n, K, j, value=1.0):
        e = np.zeros((1, n), np.int32)
        if j is not None:
            e[0, j] = 1
        c = np.zeros((1, 1 + K))
        c[0, 0] = value
        return Poly(e, c)

    def simplified(self) -> "Poly":
        if len(self.e) == 0:
            return self
        keys, inv = np.unique(self.e, axis=0, return_inverse=True)
        c = np.zeros((len(keys), self.c.shape[1]))
        np.add.at(c, inv.ravel(), self.c)
        keep = np.any(c != 0.0, axis=1)
        return Poly(keys[keep].astype(np.int32), c[keep])

    def __add__(self, o):
        return Poly(np.vstack([self.e, o.e]), np.vstack([self.c, o.c])).simplified()

    def scaled(self, s: float):
        return Poly(self.e.copy(), self.c * s).simplified()

    def __mul__(self, o):
        if len(self.e) == 0 or len(o.e) == 0:
            return Poly.zero(self.e.shape[1], self.c.shape[1] - 1)
        a_num = not np.any(self.c[:, 1:])
        b_num = not np.any(o.c[:, 1:])
        if not (a_num or b_num):
            raise TableError("product of two kinematics-dependent polynomials")
        e = (self.e[:, None, :] + o.e[None, :, :]).reshape(-1, self.e.shape[1])
        if a_num:
            c = (self.c[:, None, 0:1] * o.c[None, :, :]).reshape(-1, o.c.shape[1])
        else:
            c = (self.c[:, None, :] * o.c[None, :, 0:1]).reshape(-1, self.c.shape[1])
        return Poly(e, c).simplified()

    def with_form(self, form: np.ndarray):
        """Multiply a pure-number polynomial by a linear form (vector over 1 + K)."""
        if np.any(self.c[:, 1:]):
            raise TableError("expected a pure-number polynomial")
        return Poly(self.e.copy(), self.c[:, 0:1] * form[None, :]).simplified()


def _det(M):
    L = len(M)
    n, K = M[0][0].e.shape[1], M[0][0].c.shape[1] - 1
    acc = Poly.zero(n, K)
    for perm in permutations(range(L)):
        sign = 1.0
        for i in range(L):
            for j in range(i + 1, L):
                if perm[i] > perm[j]:
                    sign = -sign
        term = Poly.monomial(n, K, None, sign)
        for i in range(L):
            term = term * M[i][perm[i]]
        acc = acc + term
    return acc


def symanzik(topo) -> Tuple[Poly, Poly]:
    """U, F of a workloads.Topology-like object (fields loops, n_ext, props, invariants, gram_form)."""
    n, L, E, K = len(topo.props), topo.loops, topo.n_ext, len(topo.invariants)
    col = {name: 1 + i for i, name in enumerate(topo.invariants)}

    def form(lf):
        v = np.zeros(1 + K)
        for name, coef in lf.items():
            v[col[name]] += float(coef)
        return v

    G = [[form(topo.gram_form(e, f)) for f in range(E)] for e in range(E)]
    M = [[Poly.zero(n, K) for _ in range(L)] for _ in range(L)]
    Q = [[Poly.zero(n, K) for _ in range(E)] for _ in range(L)]
    J = Poly.zero(n, K)
    for j, pr in enumerate(topo.props):
        xj = Poly.monomial(n, K, j)
        for a in range(L):
            for b in range(L):
                if pr.k[a] * pr.k[b]:
                    M[a][b] = M[a][b] + xj.scaled(pr.k[a] * pr.k[b])
            for e in range(E):
                if pr.k[a] * pr.p[e]:
                    Q[a][e] = Q[a][e] + xj.scaled(pr.k[a] * pr.p[e])
        r2 = np.zeros(1 + K)
        for e in range(E):
            for f in range(E):
                r2 += pr.p[e] * pr.p[f] * G[e][f]
        if pr.mass is not None:
            r2[col[pr.mass]] -= 1.0
        if np.any(r2):
            J = J + xj.with_form(r2)
    U = _det(M)
    if L == 1:
        adj = [[Poly.monomial(n, K, None)]]
    else:
        adj = [[None] * L for _ in range(L)]
        for r in range(L):
            for c in range(L):
                minor = [[M[i][j] for j in range(L) if j != r] for i in range(L) if i != c]
                adj[r][c] = _det(minor).scaled(1.0 if (r + c) % 2 == 0 else -1.0)
    F = Poly.zero(n, K)
    for a in range(L):
        for b in range(L):
            for e in range(E):
                for f in range(E):
                    p = adj[a][b] * Q[a][e] * Q[b][f]
                    if len(p.e):
                        F = F + p.with_form(G[e][f])
    F = F + (J * U).scaled(-1.0)
    return U, F


# ------------------------------------------------------------------------------------------- decomposition
@dataclass
class SectorRecord:
    A: np.ndarray      # int32 [dim]
    B: np.ndarray      # int32 [dim]
    U: Poly
    F: Poly
    D: float = 1.0


def _leaves(U0: Poly, F0: Poly, A0, B0, eU, eF, max_depth: int) -> List[SectorRecord]:
    out: List[SectorRecord] = []
    stack = [(U0, F0, np.array(A0, np.int64), np.array(B0, np.int64), 0)]
    while stack:
        U, F, A, B, depth = stack.pop()
        s = U.e.shape[1]
        bU, bF = U.e.min(axis=0), F.e.min(axis=0)
        U = Poly(U.e - bU, U.c)
        F = Poly(F.e - bF, F.c)
        A = A + bU * eU[0] - bF * eF[0]
        B = B + bU * eU[1] - bF * eF[1]
        const_U = np.any(np.all(U.e == 0, axis=1))
        const_F = np.any(np.all(F.e == 0, axis=1))
        if const_U and const_F:
            out.append(SectorRecord(A.astype(np.int32), B.astype(np.int32), U, F))
            continue
        if depth >= max_depth:
            raise TableError(f"iterated decomposition did not terminate within depth {max_depth}")
        chosen = None
        for size in range(1, s + 1):
            for S in combinations(range(s), size):
                cols = list(S)
                if np.all(np.any(U.e[:, cols] > 0, axis=1)) or np.all(np.any(F.e[:, cols] > 0, axis=1)):
                    chosen = cols
                    break
            if chosen is not None:
                break
        children = []
        for k in chosen:
            others = [j for j in chosen if j != k]
            Ue, Fe = U.e.copy(), F.e.copy()
            Ue[:, k] += U.e[:, others].sum(axis=1)
            Fe[:, k] += F.e[:, others].sum(axis=1)
            A2, B2 = A.copy(), B.copy()
            A2[k] += A[others].sum() + len(others)
            B2[k] += B[others].sum()
            children.append((Poly(Ue, U.c), Poly(Fe, F.c), A2, B2, depth + 1))
        stack.extend(reversed(children))  # depth-first, in the order of the split variables
    return out


# ------------------------------------------------------------------------------------------- geometric strategy
# Ordering rules (they fix the table, sector by sector):
#   * facets of the Newton polytope are identified by their primitive integer outer normals m (<m, p> <= h);
#   * vertices are taken in lexicographic order of their exponent vectors; a vertex's normal cone is spanned by
#     the normals of the facets through it, listed in lexicographic order;
#   * a cone with more generators than its dimension is split by the pulling triangulation from its first
#     generator: the cone over each facet not containing it (facets in lexicographic order of their generator
#     index tuples), recursively;
#   * the variables y_1..y_{N-1} of a sector follow its generators in lexicographic order.


def _null_basis(rows: np.ndarray, d: int) -> List[np.ndarray]:
    """Primitive integer basis of {x in Q^d : rows x = 0}, one vector per free column of the exact reduced row
    echelon form.  Its length is d - rank(rows)."""
    R = [[Fraction(int(v)) for v in r] for r in np.asarray(rows).reshape(-1, d)]
    piv: List[int] = []
    for c in range(d):
        r = len(piv)
        p = next((i for i in range(r, len(R)) if R[i][c] != 0), None)
        if p is None:
            continue
        R[r], R[p] = R[p], R[r]
        lead = R[r][c]
        R[r] = [v / lead for v in R[r]]
        for i in range(len(R)):
            if i != r and R[i][c] != 0:
                f = R[i][c]
                R[i] = [a - f * b for a, b in zip(R[i], R[r])]
        piv.append(c)
    out = []
    for f in [c for c in range(d) if c not in piv]:
        v = [Fraction(0)] * d
        v[f] = Fraction(1)
        for i, c in enumerate(piv):
            v[c] = -R[i][f]
        scale = math.lcm(*(x.denominator for x in v))
        w = np.array([int(x * scale) for x in v], np.int64)
        out.append(w // np.gcd.reduce(np.abs(w)))
    return out


def _int_det(M: np.ndarray) -> int:
    """Exact determinant of a small integer matrix (fraction-free Bareiss elimination)."""
    A = [[int(v) for v in r] for r in M]
    n, sign, prev = len(A), 1, 1
    for k in range(n - 1):
        if A[k][k] == 0:
            p = next((i for i in range(k + 1, n) if A[i][k] != 0), None)
            if p is None:
                return 0
            A[k], A[p] = A[p], A[k]
            sign = -sign
        for i in range(k + 1, n):
            for j in range(k + 1, n):
                A[i][j] = (A[i][j] * A[k][k] - A[i][k] * A[k][j]) // prev
        prev = A[k][k]
    return sign * A[n - 1][n - 1]


def _cone_facets(G: np.ndarray, idx: List[int], dim: int) -> List[Tuple[int, ...]]:
    """Facets of the dim-dimensional cone spanned by the rows G[idx], as sorted tuples of the generator indices
    they contain.  A facet is the zero set of a linear form that vanishes on dim - 1 independent generators and
    has one sign on all of them."""
    d = G.shape[1]
    found = set()
    for comb in combinations(idx, dim - 1):
        ns = _null_basis(G[list(comb)], d)
        if d - len(ns) != dim - 1:
            continue
        vals = next(v for v in (G[idx] @ b for b in ns) if np.any(v))  # the form, up to sign, on span(G[idx])
        if np.all(vals >= 0) or np.all(vals <= 0):
            found.add(tuple(i for i, x in zip(idx, vals) if x == 0))
    return sorted(found)


def _pulling_triangulation(G: np.ndarray, idx: List[int], dim: int) -> List[Tuple[int, ...]]:
    """Simplicial cones (generator index tuples) of the pulling triangulation of cone(G[idx]) from G[idx[0]]."""
    if len(idx) == dim:
        return [tuple(idx)]
    apex = idx[0]
    cones: List[Tuple[int, ...]] = []
    for face in _cone_facets(G, idx, dim):
        if apex not in face:
            cones.extend((apex,) + c for c in _pulling_triangulation(G, list(face), dim - 1))
    return cones


def _newton_facets(pts: np.ndarray) -> List[Tuple[Tuple[int, ...], int]]:
    """Facets (primitive outer normal m, h = max_p <m, p>) of the convex hull of integer points spanning R^d.
    scipy's Quickhull proposes the supporting hyperplanes; each is rebuilt exactly from the points on it and
    checked to bound all points with a point set of affine rank d - 1."""
    from scipy.spatial import ConvexHull

    d = pts.shape[1]
    if d == 1:  # an interval: its two end points
        return [((-1,), -int(pts[:, 0].min())), ((1,), int(pts[:, 0].max()))]
    hull = ConvexHull(pts.astype(np.float64))
    facets = {}
    for eq in hull.equations:
        on = np.flatnonzero(np.abs(pts @ eq[:-1] + eq[-1]) <= 1e-7)
        ns = _null_basis(pts[on[1:]] - pts[on[0]], d) if len(on) >= d else []
        if len(ns) != 1:
            raise TableError("degenerate facet of the Newton polytope")
        m = ns[0] if float(ns[0] @ eq[:-1]) > 0 else -ns[0]
        h = int(pts[on[0]] @ m)
        vals = pts @ m
        if np.any(vals > h) or not np.array_equal(np.flatnonzero(vals == h), on):
            raise TableError("inexact facet of the Newton polytope")
        facets[tuple(int(x) for x in m)] = h
    return sorted(facets.items())


def _geometric_leaves(U: Poly, F: Poly, nu: Sequence[int], eU, eF) -> List[SectorRecord]:
    """Sectors of the geometric strategy for U, F in N variables (x_N = 1)."""
    n = U.e.shape[1]
    d = n - 1
    if len(np.unique(U.e.sum(axis=1))) != 1 or len(np.unique(F.e.sum(axis=1))) != 1:
        raise TableError("Symanzik polynomial is not homogeneous")
    Ue, Fe = U.e[:, :d].astype(np.int64), F.e[:, :d].astype(np.int64)
    pts = np.unique((Ue[:, None, :] + Fe[None, :, :]).reshape(-1, d), axis=0)
    facets = _newton_facets(pts)
    NM = np.array([m for m, _ in facets], np.int64)
    H = np.array([h for _, h in facets], np.int64)
    nu_d = np.array(nu[:d], np.int64)
    out: List[SectorRecord] = []
    for p in pts:  # lexicographic (np.unique sorts rows)
        G = NM[(NM @ p) == H]
        if len(G) < d or len(_null_basis(G, d)) != 0:
            continue  # p is not a vertex
        for cone in _pulling_triangulation(G, list(range(len(G))), d):
            M = G[sorted(cone)]
            det = abs(_int_det(M))
            if det == 0:
                raise TableError("degenerate cone in the triangulation")
            polys, b = [], []
            for P, E in ((U, Ue), (F, Fe)):
                ev = E @ M.T                       # <m_i, v> for every term v
                top = ev.max(axis=0)
                if np.count_nonzero(np.all(ev == top, axis=1)) != 1:
                    raise TableError("cone is not inside the normal cone of one vertex")
                polys.append(Poly((top - ev).astype(np.int32), P.c.copy()).simplified())
                b.append(-top)
            A = -(M @ nu_d) - 1 + b[0] * eU[0] - b[1] * eF[0]
            B = b[0] * eU[1] - b[1] * eF[1]
            out.append(SectorRecord(A.astype(np.int32), B.astype(np.int32), polys[0], polys[1], float(det)))
    return out


def decompose(topo, zero_invariants: Sequence[str] = (), max_depth: int = 40, strategy: str = "iterated",
              allow_higher_poles: bool = False) -> Tuple[List[SectorRecord], dict]:
    """Leaf sectors of the iterated (default) or geometric decomposition and the integral's metadata.  Exponents
    alpha <= -2 (Taylor subtraction beyond Eq. 11 with p = 0) are refused unless allow_higher_poles; the binary
    table carries them, and qmc_prepare answers QMC_ERR_UNSUPPORTED."""
    U, F = symanzik(topo)
    K = len(topo.invariants)
    for name in zero_invariants:
        if name in topo.invariants:
            idx = 1 + topo.invariants.index(name)
            U.c[:, idx] = 0.0
            F.c[:, idx] = 0.0
    U, F = U.simplified(), F.simplified()
    nu = [p.nu for p in topo.props]
    n, L = len(nu), topo.loops
    n_nu = sum(nu)
    eU = (n_nu - 2 * (L + 1), L + 1)
    eF = (n_nu - 2 * L, L)
    leaves: List[SectorRecord] = []
    if strategy == "geometric":
        leaves = _geometric_leaves(U, F, nu, eU, eF)
    elif strategy != "iterated":
        raise ValueError(f"unknown decomposition strategy {strategy!r}")
    for l in range(n if strategy == "iterated" else 0):
        keep = [j for j in range(n) if j != l]
        Ul = Poly(U.e[:, keep], U.c)
        Fl = Poly(F.e[:, keep], F.c)
        if len(np.unique(Ul.e, axis=0)) != len(Ul.e) or len(np.unique(Fl.e, axis=0)) != len(Fl.e):
            raise TableError("Symanzik polynomial is not homogeneous")
        A0 = [nu[j] - 1 for j in keep]
        leaves.extend(_leaves(Ul, Fl, A0, [0] * (n - 1), eU, eF, max_depth))
    for s in leaves:
        if np.any(s.A <= -2) and not allow_higher_poles:
            raise TableError("exponent alpha <= -2 needs higher-order subtraction (not supported)")
        if np.any((s.A <= -1) & (s.B == 0)):
            raise TableError("unregulated endpoint singularity (alpha = -1, beta = 0)")
    meta = dict(dim=n - 1, loops=L, nu=nu, n_nu=n_nu, eU=eU, eF=eF, invariants=tuple(topo.invariants))
    return leaves, meta


# ------------------------------------------------------------------------------------------- binary table
def _pad8(b: bytes) -> bytes:
    return b + b"\0" * ((-len(b)) % 8)


def write_table(leaves: List[SectorRecord], meta: dict) -> bytes:
    dim, K = meta["dim"], len(meta["invariants"])
    if dim > MAX_DIM:
        raise TableError(f"sector dimension {dim} exceeds {MAX_DIM}")
    nu = meta["nu"]
    names = b"".join(nm.encode()[:15].ljust(16, b"\0") for nm in meta["invariants"])
    nu_block = _pad8(struct.pack(f"<{len(nu)}i", *nu))
    header_bytes = 64 + len(nu_block) + len(names)
    head = MAGIC + struct.pack("<14i", VERSION, len(leaves), dim, meta["loops"], len(nu), meta["n_nu"], K,
                               meta["eU"][0], meta["eU"][1], meta["eF"][0], meta["eF"][1], header_bytes, 0, 0)
    parts = [head, nu_block, names]
    for s in leaves:
        parts.append(struct.pack("<2i", len(s.U.e), len(s.F.e)))
        parts.append(_pad8(struct.pack(f"<{2 * dim}i", *[int(a) for a in s.A], *[int(b) for b in s.B])))
        parts.append(struct.pack("<d", s.D))
        for P in (s.U, s.F):
            for e, c in zip(P.e, P.c):
                if np.any(e < 0) or np.any(e > 255):
                    raise TableError("exponent out of range")
                parts.append(bytes(list(int(v) for v in e) + [0] * (8 - dim)))
                parts.append(struct.pack(f"<{1 + K}d", *c))
    return b"".join(parts)


def read_table(blob: bytes):
    """Parse a table back into (meta, [SectorRecord]) -- for inspection and tests."""
    if blob[:8] != MAGIC:
        raise TableError("bad magic")
    v = struct.unpack_from("<14i", blob, 8)
    version, ns, dim, loops, nprops, n_nu, K, eU0, eU1, eF0, eF1, hb = v[:12]
    nu = list(struct.unpack_from(f"<{nprops}i", blob, 64))
    off = 64 + len(_pad8(b"\0" * 4 * nprops))
    names = tuple(blob[off + 16 * i: off + 16 * (i + 1)].rstrip(b"\0").decode() for i in range(K))
    off = hb
    leaves = []
    for _ in range(ns):
        nU, nF = struct.unpack_from("<2i", blob, off)
        off += 8
        AB = struct.unpack_from(f"<{2 * dim}i", blob, off)
        off += len(_pad8(b"\0" * 8 * dim))
        (D,) = struct.unpack_from("<d", blob, off)
        off += 8
        polys = []
        for cnt in (nU, nF):
            e = np.zeros((cnt, dim), np.int32)
            c = np.zeros((cnt, 1 + K))
            for t in range(cnt):
                e[t] = list(blob[off: off + dim])
                off += 8
                c[t] = struct.unpack_from(f"<{1 + K}d", blob, off)
                off += 8 * (1 + K)
            polys.append(Poly(e, c))
        leaves.append(SectorRecord(np.array(AB[:dim], np.int32), np.array(AB[dim:], np.int32), polys[0], polys[1], D))
    meta = dict(dim=dim, loops=loops, nu=nu, n_nu=n_nu, eU=(eU0, eU1), eF=(eF0, eF1), invariants=names)
    return meta, leaves


def compile_integral(topo, zero_invariants: Sequence[str] = (), strategy: str = "iterated",
                     allow_higher_poles: bool = False) -> bytes:
    """Sector table (bytes) of `topo` for the kinematic class in which `zero_invariants` vanish."""
    leaves, meta = decompose(topo, zero_invariants, strategy=strategy, allow_higher_poles=allow_higher_poles)
    return write_table(leaves, meta)


def zero_invariants_of(topo, point) -> Tuple[str, ...]:
    return tuple(n for n in topo.invariants if float(point.get(n, 0.0)) == 0.0)
