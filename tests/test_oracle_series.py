"""Pin for the oracle's per-point integrand (paper Sec. II, Eqs. 10-12 and 14; Sec. III, Eq. 21).

The oracle expands everything in eps as truncated Laurent series.  Here the same sector integrand is evaluated
*unexpanded* at finite complex eps (complex powers, the subtraction of Eq. 11 applied to actual function
values, a Jacobian of the deformation z(t) of Eq. 14 taken by an exact 5-point finite difference, the transform
phi_r obtained by integrating c_r u^r (1-u)^r with numpy's polynomial class), and its Laurent coefficients are
extracted by the trapezoidal rule on a circle |eps| = rho (a contour integral, exponentially accurate).  A wrong
sign, a dropped term or a wrong truncation in the series arithmetic fails this test.
"""
import cmath
import math

import numpy as np
import pytest

import workloads as W
from oracle import integrate as OI

MASSLESS_LEGS = dict(pp1=0.0, pp2=0.0, pp3=0.0, pp4=0.0)


def phi_poly(r):
    c = math.factorial(2 * r + 1) / math.factorial(r) ** 2
    dens = np.polynomial.Polynomial([0, 1]) ** r * np.polynomial.Polynomial([1, -1]) ** r * c
    return dens.integ(lbnd=0.0), dens


def unexpanded(sec, e4, x, lam, r, eps):
    d = sec.dim
    ph, dph = phi_poly(r)
    t = np.array([ph(v) for v in x])
    tm = np.array([ph(1.0 - v) for v in x])
    w = float(np.prod([dph(v) for v in x]))

    def poly(c, ex, z):
        return sum(cc * np.prod([z[j] ** ex[a, j] for j in range(d)]) for a, cc in enumerate(c))

    def grad(tt):
        g = np.zeros(d)
        for a, cc in enumerate(sec.cF):
            for j in range(d):
                e = sec.xF[a, j]
                if e:
                    ex = sec.xF[a].copy()
                    ex[j] -= 1
                    g[j] += cc * e * np.prod([tt[k] ** ex[k] for k in range(d)])
        return g

    def zmap(tt):
        g = grad(tt)
        return np.array([tt[j] - 1j * lam * tt[j] * (1 - tt[j]) * g[j] for j in range(d)]), g

    def log_f(v):  # log(F - i0)
        if v.imag == 0.0 and v.real < 0:
            return math.log(-v.real) - 1j * math.pi
        return cmath.log(v)

    sing = [j for j in range(d) if sec.A[j] == -1]

    def G(Y):
        tt = np.array([0.0 if j in Y else t[j] for j in range(d)])
        if sec.kind == 2:
            z, g = zmap(tt)
            h = 1e-2
            J = np.zeros((d, d), dtype=complex)
            for k in range(d):
                cols = []
                for s_ in (-2, -1, 1, 2):
                    tp = tt.copy()
                    tp[k] += s_ * h
                    cols.append(zmap(tp)[0])
                J[:, k] = (cols[0] - 8 * cols[1] + 8 * cols[2] - cols[3]) / (12 * h)
            detJ = np.linalg.det(J)
            q = np.array([1 - 1j * lam * (1 - tt[j]) * g[j] for j in range(d)])
        else:
            z, detJ, q = tt.astype(complex), 1.0, np.ones(d, dtype=complex)
        U = poly(sec.cU, sec.xU, z)
        Fv = poly(sec.cF, sec.xF, z)
        val = sec.D * detJ * cmath.exp((e4[0] + e4[1] * eps) * cmath.log(U) - (e4[2] + e4[3] * eps) * log_f(Fv))
        for j in range(d):
            a = sec.A[j] + sec.B[j] * eps
            if sec.A[j] != -1:
                val *= cmath.exp(a * math.log(tt[j])) if tt[j] > 0 else (1.0 if sec.A[j] == 0 else 0.0)
            val *= cmath.exp(a * cmath.log(q[j]))
        return val

    def sub(i, Y):
        if i == len(sing):
            return G(Y)
        j = sing[i]
        a = sub(i + 1, Y)
        b = sub(i + 1, Y | {j})
        return cmath.exp((-1 + sec.B[j] * eps) * math.log(t[j])) * (a - b) + b / (sec.B[j] * eps)

    return w * sub(0, frozenset())


def laurent_by_contour(f, kmin, kmax, rho=0.2, K=64):
    th = 2 * np.pi * np.arange(K) / K
    eps = rho * np.exp(1j * th)
    vals = np.array([f(e) for e in eps])
    return np.array([np.mean(vals * eps ** (-k)) for k in range(kmin, kmax + 1)])


CASES = [
    ("massless_box", W.box(False), dict(s=-3.0, t=-2.0, **MASSLESS_LEGS), 0.0, 0, 2),
    ("massive_box_deformed", W.box(True), dict(s=5.0, t=-1.5, msq=1.0, **MASSLESS_LEGS), 0.5, 2, 3),
    ("triangle_deformed", W.triangle_massive(), dict(pp3=5.0, msq=1.0), 0.4, 2, 1),
    ("bubble_negative_F", W.bubble(False), dict(pp1=2.0), 0.0, 2, 3),
    ("planar_dbox", W.double_box_planar(True), dict(s=6.0, t=-2.0, msq=1.0, **MASSLESS_LEGS), 0.25, 0, 3),
]


@pytest.mark.parametrize("name,topo,pt,lam,kmax,r", CASES, ids=[c[0] for c in CASES])
def test_point_series_matches_unexpanded(name, topo, pt, lam, kmax, r):
    prob = OI.make_problem(topo, pt, -4, kmax)
    rng = np.random.default_rng(17)
    # pick the sectors with the most singular variables (and a deformed one when available)
    nsec, npts = (2, 1) if prob.sectors[0].dim > 3 else (3, 2)
    secs = sorted(range(len(prob.sectors)), key=lambda i: -prob.sectors[i].sigma)[:nsec]
    for i in secs:
        sec = prob.sectors[i]
        for _ in range(npts):
            x = rng.uniform(0.05, 0.95, size=sec.dim)
            ser, fail = OI.point_series(sec, prob.e4, x, lam, r, kmax)
            ref = laurent_by_contour(lambda e: unexpanded(sec, prob.e4, x, lam, r, e), -sec.sigma, kmax)
            scale = np.max(np.abs(ref))
            assert np.max(np.abs(ser - ref)) <= 1e-10 * scale, (name, i, ser, ref)
