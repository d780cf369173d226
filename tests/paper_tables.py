"""Printed Laurent coefficients of the paper's two-loop examples (tests/golden/paper_tables_3_4.txt for the
physical region, tests/golden/paper_table_2.txt for the Euclidean one) and the conversion of a result to the
paper's normalisation I = exp(-2 eps gamma_E) s^(-3-2 eps) sum_i P_i eps^-i ((-s) in place of s when s < 0)."""
import math
import os

import numpy as np

GAMMA_E = 0.5772156649015329
HERE = os.path.dirname(os.path.abspath(__file__))


def golden():
    """{(integral, method): {i: (P_i complex, error re, error im)}}"""
    out = {}
    for line in open(os.path.join(HERE, "golden", "paper_tables_3_4.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        name, i, method, re_, ere, im_, eim = line.split()
        out.setdefault((name, method), {})[int(i)] = (complex(float(re_), float(im_)), float(ere), float(eim))
    return out


def to_paper(c, e, s):
    """c[k], e[k]: coefficients of eps^(k-2), k = 0, 1, 2 (complex) and their errors (complex: re and im errors,
    or real: one error for both).  Returns {2: (P_2, err re, err im), 1: ..., 0: ...}; errors add linearly."""
    a = 2.0 * (GAMMA_E + math.log(s))
    w = [[1.0], [a, 1.0], [a * a / 2.0, a, 1.0]]  # P_{2-k} = s^3 sum_q w[k][q] c[q]
    er = np.real(e) if np.iscomplexobj(e) else np.asarray(e, float)
    ei = np.imag(e) if np.iscomplexobj(e) else np.asarray(e, float)
    out = {}
    for k in range(3):
        P = s ** 3 * sum(w[k][q] * c[q] for q in range(k + 1))
        out[2 - k] = (P, s ** 3 * sum(abs(w[k][q]) * er[q] for q in range(k + 1)),
                      s ** 3 * sum(abs(w[k][q]) * ei[q] for q in range(k + 1)))
    return out


def agrees(ours, printed, nsig):
    """ours/printed: (P, err re, err im); within nsig combined standard errors in both parts"""
    (p, er, ei), (q, fr, fi) = ours, printed
    return abs(p.real - q.real) <= nsig * math.hypot(er, fr) and abs(p.imag - q.imag) <= nsig * math.hypot(ei, fi)


def golden_table2():
    """{(column tag, method): {i: (P_i, error)}} of Table 2 (real coefficients)."""
    out = {}
    for line in open(os.path.join(HERE, "golden", "paper_table_2.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        tag, i, method, val, err = line.split()
        out.setdefault((tag, method), {})[int(i)] = (float(val), float(err))
    return out


def to_paper_euclid(c, e, s):
    """c[k], e[k]: real coefficients of eps^(k-4), k = 0..4, and their errors, at s < 0.  Returns
    {4 - k: (P_{4-k}, error)} for P(eps) = exp(2 eps gamma_E) (-s)^(3 + 2 eps) I(eps); errors add linearly."""
    a = 2.0 * (GAMMA_E + math.log(-s))
    out = {}
    for k in range(5):
        w = [a ** (k - q) / math.factorial(k - q) for q in range(k + 1)]
        out[4 - k] = ((-s) ** 3 * sum(w[q] * c[q] for q in range(k + 1)),
                      (-s) ** 3 * sum(abs(w[q]) * e[q] for q in range(k + 1)))
    return out


def agrees_real(ours, printed, nsig, floor=1e-12):
    """ours/printed: (P, error); within nsig combined errors (plus an absolute floor for exact zeros)."""
    return abs(ours[0] - printed[0]) <= nsig * math.hypot(ours[1], printed[1]) + floor
