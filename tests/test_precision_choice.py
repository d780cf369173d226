"""qmc_choose_precision on the host (no GPU): the per-sector choice between FP32, FP32 with FP64 islands at a level
and FP64 for a mixed pass, from synthetic probe outputs.  The rule as the header states it is restated here (option
errors from the island bins, costs with FP64 counted 30 times, the per-order limits budget * |T_k| from the sums),
and the library's choice must
* bound each order's FP32 bias by the sectors' summed statistics (each sector's |signed mean|, three standard
  errors of the sum, capped by the mean |e|);
* meet every order's limit (on random instances, including ones where options tie in some slots -- the case where
  a rounding of used - e0 + e1 once made every change look worse and sent all sectors to FP64);
* cost no more than 1.5x the brute-force optimum over the sectors that carry error;
* take, without an estimate, each sector's cheapest option within its own magnitude;
* never take an option with a non-finite error, and keep class-2 sectors (alpha <= -2) in FP64."""
import dataclasses
import itertools

import numpy as np
import pytest

import workloads as W
from oracle import integrate as OI
from oracle import sectors as OS
from paper_1508_02512_gb300 import _native as N
from paper_1508_02512_gb300 import api
from paper_1508_02512_gb300 import tables as T

BINS = N.QMC_ISLAND_BINS
NOPT = N.QMC_ISLAND_LEVELS + 2  # FP32, islands L = 0..5, FP64
FP64_COST = 30.0
BOX_POINT = dict(s=-3.0, t=-2.0, pp1=0.0, pp2=0.0, pp3=0.0, pp4=0.0)


@pytest.fixture(scope="module")
def box():
    topo = W.box(False)
    blob = T.compile_integral(topo, T.zero_invariants_of(topo, BOX_POINT))
    return api.prepare(blob, W.kinematics(topo, **BOX_POINT), -2, 0)


def call(prep, probe, bins, n_sample, rel_tol, budget, sums=None, n_sector=None, m=0):
    ns = prep.info.n_sectors
    codes = np.full(ns, -7, dtype=np.int32)
    counts = np.zeros(2, dtype=np.int32)
    probe = np.ascontiguousarray(probe, dtype=np.float64)
    bins = np.ascontiguousarray(bins, dtype=np.float64)
    sp = nsp = None
    if sums is not None:
        sums = np.ascontiguousarray(sums, dtype=np.float64)
        n_sector = np.ascontiguousarray(n_sector, dtype=np.int64)
        sp, nsp = sums.ctypes.data, n_sector.ctypes.data
    rc = N.lib().qmc_choose_precision(prep.packed, m, nsp, sp, probe.ctypes.data, bins.ctypes.data, n_sample,
                                      rel_tol, budget, codes.ctypes.data, counts.ctypes.data)
    return rc, codes, counts


def option_of(code):
    return NOPT - 1 if code == 0 else (0 if code == 1 else code - 1)


def restated(prep, bins, n_sample):
    """per sector and option: the FP32 bins' statistics per slot (mean |e|, |mean e|, 0, sum |e|^2 / n^2) and the
    cost, as the header defines them"""
    ns, sl = prep.info.n_sectors, prep.info.n_slots
    stats = np.zeros((ns, NOPT, sl, 4))
    cost = np.zeros((ns, NOPT))
    for s in range(ns):
        fl = max(prep.sector(s).flops, 1.0)
        for q in range(NOPT):
            top = -1 if q == NOPT - 1 else (BINS - 1 if q == 0 else q - 1)
            v = bins[s, : top + 1, 1:].reshape(top + 1, sl, 4).sum(axis=0)
            stats[s, q, :, 0] = v[:, 0] / n_sample
            stats[s, q, :, 1] = np.hypot(v[:, 1], v[:, 2]) / n_sample  # |mean e|: no cancellation between sectors
            stats[s, q, :, 3] = v[:, 3] / n_sample ** 2
            island = bins[s, top + 1:, 0].sum() / n_sample
            cost[s, q] = fl * (FP64_COST if q == NOPT - 1 else 1.0 + FP64_COST * island)
    return stats, cost


def bound(t):
    """the bias bound of summed statistics (last axis: mean |e|, mean e re, im, variance)"""
    return np.minimum(t[..., 0], np.hypot(t[..., 1], t[..., 2]) + 3.0 * np.sqrt(np.maximum(t[..., 3], 0.0)))


def limits(prep, sums, n_sector, m, budget):
    ns, sl = prep.info.n_sectors, prep.info.n_slots
    sig = [prep.sector(s).sigma for s in range(ns)]
    K = sl + max(sig)
    Tk = np.zeros(K, dtype=complex)
    for s in range(ns):
        for o in range(sl):
            Tk[o - sig[s] + max(sig)] += (sums[s, :, o, 0] + 1j * sums[s, :, o, 1]).sum() / (m * n_sector[s])
    return budget * np.maximum(np.abs(Tk), 1e-6 * np.abs(Tk).max()), sig


def used(prep, stats, picks, sig, K):
    """per order: the bias bound of the chosen options' statistics summed over sectors"""
    t = np.zeros((K, 4))
    for s, q in enumerate(picks):
        for o in range(prep.info.n_slots):
            t[o - sig[s] + max(sig)] += stats[s, q, o]
    return bound(t)


def instance(prep, rng, active, n_sample=4096, m=4, n=1021):
    """errors only in the active sectors, decreasing away from the faces (higher bins carry more)"""
    ns, sl = prep.info.n_sectors, prep.info.n_slots
    counts = rng.multinomial(n_sample, np.array([0.55, 0.25, 0.1, 0.05, 0.03, 0.015, 0.005]), size=ns)
    bins = np.zeros((ns, BINS, 1 + 4 * sl))
    bins[:, :, 0] = counts
    for s in active:
        scale = 10.0 ** rng.uniform(-7, -4)
        for o in range(sl):
            prof = 10.0 ** (rng.uniform(0.0, 1.5) * np.arange(BINS)) * rng.uniform(0.2, 1.0, BINS)
            if rng.uniform() < 0.3:  # ties: this slot's error lies in bin 0 only, the same for every FP32 option
                prof[1:] = 0.0
            absum = scale * prof / prof.sum() * n_sample
            bias = rng.uniform(-1.0, 1.0, (BINS, 2)) * absum[:, None] * rng.uniform(0.0, 1.0)
            bins[s, :, 1 + 4 * o] = absum
            bins[s, :, 2 + 4 * o] = bias[:, 0]
            bins[s, :, 3 + 4 * o] = bias[:, 1]
            bins[s, :, 4 + 4 * o] = absum ** 2 / np.maximum(counts[s], 1) * rng.uniform(1.0, 30.0, BINS)
    probe = np.zeros((ns, sl, 4))
    probe[:, :, 0] = n_sample * 1.0
    probe[:, :, 1] = bins[:, :, 1::4].sum(axis=1)
    sums = rng.normal(0.0, 1.0, (ns, m, sl, 2)) * n
    return probe, bins, sums, np.full(ns, n, dtype=np.int64), m


def test_random_instances_meet_every_limit_near_the_optimum(box):
    prep = box
    ns = prep.info.n_sectors
    rng = np.random.default_rng(7)
    ratios = []
    for trial in range(60):
        active = sorted(rng.choice(ns, 3, replace=False))
        probe, bins, sums, nsec, m = instance(prep, rng, active)
        budget_frac, rel_tol = 0.1, 10.0 ** rng.uniform(-5, -3)
        rc, codes, counts = call(prep, probe, bins, 4096, rel_tol, budget_frac, sums, nsec, m)
        assert rc == 0
        assert set(codes.tolist()) <= set(range(0, 2 + N.QMC_ISLAND_LEVELS))
        stats, cost = restated(prep, bins, 4096)
        lim, sig = limits(prep, sums, nsec, m, budget_frac * rel_tol)
        K = len(lim)
        picks = [option_of(c) for c in codes]
        assert np.all(used(prep, stats, picks, sig, K) <= lim * (1 + 1e-9)), trial
        assert counts[0] == int((codes == 0).sum()) and counts[1] == int((codes >= 2).sum())
        # brute force over the active sectors (the others carry no error: FP32, their cheapest option)
        base = [0] * ns
        best = np.inf
        for combo in itertools.product(range(NOPT), repeat=len(active)):
            pk = list(base)
            for s, q in zip(active, combo):
                pk[s] = q
            if np.all(used(prep, stats, pk, sig, K) <= lim):
                best = min(best, sum(cost[s, q] for s, q in enumerate(pk)))
        got = sum(cost[s, q] for s, q in enumerate(picks))
        ratios.append(got / best)
    print(f"greedy cost / optimum over 60 instances: mean {np.mean(ratios):.3f}, max {np.max(ratios):.3f}")
    assert np.max(ratios) <= 1.5 and np.mean(ratios) <= 1.1


def test_without_estimate_each_sector_is_held_to_its_own_magnitude(box):
    prep = box
    ns, sl = prep.info.n_sectors, prep.info.n_slots
    rng = np.random.default_rng(3)
    probe, bins, _, _, _ = instance(prep, rng, list(range(ns)))
    rel_tol, frac = 1e-4, 0.1
    rc, codes, _ = call(prep, probe, bins, 4096, rel_tol, frac)
    assert rc == 0
    stats, cost = restated(prep, bins, 4096)
    own = probe[:, :, 0] / 4096
    for s in range(ns):
        fits = [q for q in range(NOPT) if np.all(bound(stats[s, q]) <= frac * rel_tol * own[s])]
        want = min(fits, key=lambda q: (cost[s, q], q))
        assert option_of(codes[s]) == want or cost[s, option_of(codes[s])] == cost[s, want]


def test_non_finite_errors_and_class2_sectors_go_to_safe_options(box):
    prep = box
    ns, sl = prep.info.n_sectors, prep.info.n_slots
    rng = np.random.default_rng(5)
    probe, bins, sums, nsec, m = instance(prep, rng, [0, 1])
    bins[0, 4, 1] = np.inf   # an FP32 overflow at points of bin 4: only islands at levels 0..3 or FP64 avoid it
    bins[1, 0, 1 + 4 * 2] = np.nan   # a NaN away from the faces: only FP64 avoids it
    rc, codes, _ = call(prep, probe, bins, 4096, 1e-3, 10.0, sums, nsec, m)
    assert rc == 0
    assert codes[0] in (0, 2, 3, 4, 5) and codes[1] == 0
    # alpha <= -2 (class 2): FP64 whatever the errors
    topo = dataclasses.replace(W.bubble(False), props=tuple(dataclasses.replace(p, nu=v) for p, v in
                                                            zip(W.bubble(False).props, (3, 1))))
    blob = T.compile_integral(topo, (), allow_higher_poles=True)
    p2 = api.prepare(blob, W.kinematics(topo, pp1=-2.0), -2, 2)
    n2, s2 = p2.info.n_sectors, p2.info.n_slots
    pr2 = np.ones((n2, s2, 4))
    b2 = np.zeros((n2, BINS, 1 + 4 * s2))
    b2[:, 0, 0] = 4096
    rc, codes, counts = call(p2, pr2, b2, 4096, 1e-3, 0.1)
    prob = OI.make_problem(topo, dict(pp1=-2.0), -2, 2,
                           sectors=OS.decompose(topo, (), "iterated", allow_higher_poles=True))
    cls2 = np.array([int(sec.A.min()) <= -2 for sec in prob.sectors])
    assert rc == 0 and cls2.any() and np.all(codes[cls2] == 0) and np.all(codes[~cls2] == 1)


def test_argument_errors(box):
    prep = box
    ns, sl = prep.info.n_sectors, prep.info.n_slots
    probe = np.zeros((ns, sl, 4))
    bins = np.zeros((ns, BINS, 1 + 4 * sl))
    codes = np.zeros(ns, dtype=np.int32)
    L = N.lib()
    assert L.qmc_choose_precision(None, 0, None, None, probe.ctypes.data, bins.ctypes.data, 1, 1e-3, 0.1,
                                  codes.ctypes.data, None) == N.QMC_ERR_ARG
    assert L.qmc_choose_precision(prep.packed, 0, None, None, probe.ctypes.data, None, 1, 1e-3, 0.1,
                                  codes.ctypes.data, None) == N.QMC_ERR_ARG
    assert L.qmc_choose_precision(prep.packed, 0, None, None, probe.ctypes.data, bins.ctypes.data, 0, 1e-3, 0.1,
                                  codes.ctypes.data, None) == N.QMC_ERR_ARG
    sums = np.zeros((ns, 2, sl, 2))
    assert L.qmc_choose_precision(prep.packed, 2, None, sums.ctypes.data, probe.ctypes.data, bins.ctypes.data, 1,
                                  1e-3, 0.1, codes.ctypes.data, None) == N.QMC_ERR_ARG
    nz = np.zeros(ns, dtype=np.int64)
    assert L.qmc_choose_precision(prep.packed, 2, nz.ctypes.data, sums.ctypes.data, probe.ctypes.data,
                                  bins.ctypes.data, 1, 1e-3, 0.1, codes.ctypes.data, None) == N.QMC_ERR_ARG
    assert L.qmc_choose_precision(prep.packed, 0, None, None, probe.ctypes.data, bins.ctypes.data, 1, -1.0, 0.1,
                                  codes.ctypes.data, None) == N.QMC_ERR_ARG
