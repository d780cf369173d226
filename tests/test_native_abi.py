"""CPU checks of the product side: the C-ABI library loads and exports every symbol include/qmcfi.h declares; the
host-only entry points (table validation, packing, prefactor, combination) agree with the oracle; the table
compiler and the fast CBC reproduce the oracle's decomposition and CBC exactly (integer data, bit for bit)."""
import ctypes
import os
import re
from fractions import Fraction

import numpy as np
import pytest

import workloads as W
from oracle import integrate as OI
from oracle import lattice as OL
from oracle import sectors as OS
from paper_1508_02512_gb300 import _native as N
from paper_1508_02512_gb300 import api
from paper_1508_02512_gb300 import lattice as PL
from paper_1508_02512_gb300 import tables as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LEGS0 = dict(pp1=0.0, pp2=0.0, pp3=0.0, pp4=0.0)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1508_02512_gb300 import build
    build.build()
    N.lib()


def header_functions():
    txt = open(os.path.join(ROOT, "include", "qmcfi.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(qmc_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported_and_bound():
    names = header_functions()
    assert len(names) >= 15
    L = N.lib()
    for nm in names:
        assert hasattr(L, nm), nm
        assert nm in N.PROTOTYPES, f"{nm} has no Python binding"
    assert set(N.PROTOTYPES) == set(names)


def test_strerror_and_version():
    assert N.strerror(0) == "ok"
    assert "table" in N.strerror(N.QMC_ERR_TABLE)
    assert N.lib().qmc_version() >= 100


def canon_product(leaves, meta):
    names = meta["invariants"]

    def pk(P):
        return tuple(sorted((tuple(int(v) for v in e),
                             tuple(sorted((names[k - 1] if k else "1", Fraction(float(c[k])))
                                          for k in range(len(c)) if c[k] != 0)))
                            for e, c in zip(P.e, P.c)))

    return tuple(sorted((tuple(int(a) for a in s.A), tuple(int(b) for b in s.B), pk(s.U), pk(s.F)) for s in leaves))


@pytest.mark.parametrize("cfg", W.CONFIGS, ids=lambda c: c.name)
def test_table_compiler_matches_oracle_decomposition(cfg):
    blob = T.compile_integral(cfg.topology, T.zero_invariants_of(cfg.topology, cfg.point))
    meta, leaves = T.read_table(blob)
    mine = canon_product(leaves, meta)
    ref = OS.canonical(OS.decompose(cfg.topology, OS.zero_invariants_of(cfg.topology, cfg.point)))
    assert mine == ref


GEOMETRIC_CASES = [(c.topology, T.zero_invariants_of(c.topology, c.point), c.name) for c in W.CONFIGS] + [
    (W.double_box_planar(False), T.zero_invariants_of(W.double_box_planar(False), W.PAPER_IB_POINTS["0,-1,0,-1"]),
     "massless_dbox_table2")]


@pytest.mark.parametrize("topo,zero,name", GEOMETRIC_CASES, ids=[c[2] for c in GEOMETRIC_CASES])
def test_geometric_table_matches_oracle_sector_by_sector(topo, zero, name):
    """The geometric strategy, written twice (product: integer elimination; oracle: rational cofactors), must give
    the same sectors in the same order: exponents, Jacobian D and both polynomials."""
    meta, leaves = T.read_table(T.compile_integral(topo, zero, strategy="geometric"))
    ref = OS.decompose(topo, zero, "geometric")
    assert len(leaves) == len(ref)
    for a, b in zip(leaves, ref):
        assert canon_product([a], meta) == OS.canonical([b])
        assert a.D == float(b.D)


def test_table_compiler_rejects_alpha_minus_two():
    """The massless box with a squared propagator has alpha = -2 sectors (Taylor subtraction beyond Eq. 11 with
    p = 0): the table compiler refuses it under both strategies."""
    import dataclasses
    topo = W.box(False)
    dotted = dataclasses.replace(topo, props=(dataclasses.replace(topo.props[0], nu=2),) + topo.props[1:])
    for strategy in ("iterated", "geometric"):
        with pytest.raises(T.TableError, match="alpha <= -2"):
            T.compile_integral(dotted, ("pp1", "pp2", "pp3", "pp4"), strategy=strategy)


def test_squared_propagator_tables_match_the_oracle_and_prepare_takes_them():
    """With allow_higher_poles the table compiler writes the alpha = -2 sectors of the squared-propagator box,
    sector for sector equal to the oracle's (which integrates them with oracle.taylor); qmc_prepare takes them
    (undeformed: Taylor subtraction of Eq. 11 with p > 0 in the class-2 kernel) and counts them as such."""
    import dataclasses
    topo = W.box(False)
    dotted = dataclasses.replace(topo, props=(dataclasses.replace(topo.props[0], nu=2),) + topo.props[1:])
    zero = ("pp1", "pp2", "pp3", "pp4")
    for strategy in ("iterated", "geometric"):
        blob = T.compile_integral(dotted, zero, strategy=strategy, allow_higher_poles=True)
        meta, leaves = T.read_table(blob)
        ref = OS.decompose(dotted, zero, strategy, allow_higher_poles=True)
        assert canon_product(leaves, meta) == OS.canonical(ref)
        assert min(int(s.A.min()) for s in leaves) == -2
        prep = api.prepare(blob, W.kinematics(dotted, s=-3.0, t=-2.0), -2, 0)
        # class-2 sectors are sorted last; their sigma counts every variable with alpha <= -1
        higher = [k for k, s in enumerate(leaves) if int(s.A.min()) <= -2]
        for k in higher:
            assert prep.sector(k).sigma == int((leaves[k].A <= -1).sum())
        assert 0 < len(higher) < len(leaves)
        # the physical region (deformed sectors) stays refused for alpha <= -2
        assert _prep_status(blob, W.kinematics(dotted, s=3.0, t=-2.0)) == N.QMC_ERR_UNSUPPORTED


def test_symanzik_matches_oracle_for_all_topologies():
    from oracle import feynman as fy
    for topo in (W.bubble(True), W.triangle_massive(), W.box(True), W.double_box_planar(True),
                 W.double_box_nonplanar(True)):
        U, F = T.symanzik(topo)
        Uo, Fo = fy.symanzik_momentum(topo)
        names = topo.invariants

        def conv(P):
            return {tuple(int(v) for v in e): {(names[k - 1] if k else "1"): Fraction(float(c[k]))
                                               for k in range(len(c)) if c[k] != 0} for e, c in zip(P.e, P.c)}

        assert conv(U) == Uo and conv(F) == Fo


@pytest.mark.parametrize("n", [101, 1009, 1021, 2039, 4093])
def test_fast_cbc_matches_oracle_cbc(n):
    assert PL.fast_cbc(n) == OL.cbc_plain(n, 6)


def test_builtin_lattices():
    lat = api.builtin_lattices()
    assert [n for n, _ in lat] == [OL.prime_below(1 << k) for k in range(10, 10 + len(lat))]
    for n, z in lat[:3]:
        assert z == OL.cbc_plain(n, 6)
    # the criterion decreases along the ladder
    e = [OL.cbc_error2(n, z) for n, z in lat[:6]]
    assert all(a > b for a, b in zip(e, e[1:]))


@pytest.mark.parametrize("cfg", W.CONFIGS, ids=lambda c: c.name)
def test_prepare_matches_oracle(cfg):
    blob = T.compile_integral(cfg.topology, T.zero_invariants_of(cfg.topology, cfg.point))
    prep = api.prepare(blob, cfg.kin, cfg.order_min, cfg.order_max)
    prob = OI.make_problem(cfg.topology, cfg.point, cfg.order_min, cfg.order_max)
    assert prep.info.n_sectors == len(prob.sectors)
    assert prep.info.pre_low == prob.pre_low
    k = min(prep.info.n_pre, 6)
    assert np.allclose(list(prep.info.pre)[:k], prob.pre[:k], rtol=1e-14, atol=1e-15)
    for s, sec in enumerate(prob.sectors):
        d = prep.sector(s)
        assert (d.kind, d.sigma) == (sec.kind, sec.sigma)
    assert prep.info.flops_per_eval > 0


def test_prepare_geometric_table_with_four_poles():
    """qmc_prepare on the geometric table of the massless double box (Table 2): sector kinds, singular-variable
    counts up to four, five series slots for eps^-4..eps^0, and the prefactor Gamma(3 + 2 eps)."""
    topo, pt = W.double_box_planar(False), W.PAPER_IB_POINTS["-1,0,0,-1"]
    blob = T.compile_integral(topo, T.zero_invariants_of(topo, pt), strategy="geometric")
    prep = api.prepare(blob, W.kinematics(topo, **pt), -4, 0)
    prob = OI.make_problem(topo, pt, -4, 0, "geometric")
    assert prep.info.n_sectors == len(prob.sectors) == 143
    assert prep.info.max_sigma == 4 and prep.info.n_slots == 5 and prep.info.pre_low == prob.pre_low == 0
    assert np.allclose(list(prep.info.pre)[:5], prob.pre[:5], rtol=1e-14, atol=1e-15)
    for s, sec in enumerate(prob.sectors):
        d = prep.sector(s)
        assert (d.kind, d.sigma) == (sec.kind, sec.sigma) == (0, sec.sigma)


def test_prefactor_with_pole_matches_oracle():
    blob = T.compile_integral(W.bubble(False), ())
    prep = api.prepare(blob, np.array([-2.0]), -1, 3)
    prob = OI.make_problem(W.bubble(False), dict(pp1=-2.0), -1, 3)
    assert prep.info.pre_low == prob.pre_low == -1
    assert np.allclose(list(prep.info.pre)[:6], prob.pre[:6], rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("cfg", [W.CONFIG0, W.CONFIG1], ids=lambda c: c.name)
def test_combine_matches_oracle(cfg):
    """qmc_combine and the oracle's combination agree on the same (synthetic) per-sector sums."""
    blob = T.compile_integral(cfg.topology, T.zero_invariants_of(cfg.topology, cfg.point))
    prep = api.prepare(blob, cfg.kin, cfg.order_min, cfg.order_max)
    prob = OI.make_problem(cfg.topology, cfg.point, cfg.order_min, cfg.order_max)
    m, n = 6, 1021
    rng = np.random.default_rng(1)
    slots = prep.info.n_slots
    sums = np.zeros((prep.info.n_sectors, m, slots, 2))
    per = []
    for s, sec in enumerate(prob.sectors):
        nout = prob.kmax + sec.sigma + 1
        v = rng.normal(size=(m, nout)) + 1j * rng.normal(size=(m, nout))
        per.append(v)
        sums[s, :, :nout, 0] = v.real
        sums[s, :, :nout, 1] = v.imag
    p = api.make_pass(n, [1] * 6, m)
    Q, mean, err = api.combine(prep, p, sums)
    Qo = OI.combine(prob, per, n)
    mo, eo = OI.mean_and_error(Qo)
    assert np.allclose(Q, Qo, rtol=1e-13, atol=1e-15)
    assert np.allclose(mean, mo, rtol=1e-13, atol=1e-15)
    assert np.allclose(np.hypot(err[:, 0], err[:, 1]), eo, rtol=1e-12)


@pytest.mark.parametrize("cfg", [W.CONFIG0, W.CONFIG1], ids=lambda c: c.name)
def test_combine_sectors_matches_oracle_with_per_sector_lattices(cfg):
    """Sectors from lattices of different sizes: each sector's sum enters Eq. 19 with its own 1/n_s, so the oracle's
    single-n combination of the rescaled sums n/n_s * v_s gives the same totals."""
    blob = T.compile_integral(cfg.topology, T.zero_invariants_of(cfg.topology, cfg.point))
    prep = api.prepare(blob, cfg.kin, cfg.order_min, cfg.order_max)
    prob = OI.make_problem(cfg.topology, cfg.point, cfg.order_min, cfg.order_max)
    m, n = 5, 1021
    rng = np.random.default_rng(2)
    slots = prep.info.n_slots
    ladder = [1021, 2039, 4093, 8191]
    n_s = [ladder[s % len(ladder)] for s in range(prep.info.n_sectors)]
    sums = np.zeros((prep.info.n_sectors, m, slots, 2))
    per = []
    for s, sec in enumerate(prob.sectors):
        nout = prob.kmax + sec.sigma + 1
        v = rng.normal(size=(m, nout)) + 1j * rng.normal(size=(m, nout))
        per.append(v * (n / n_s[s]))
        sums[s, :, :nout, 0] = v.real
        sums[s, :, :nout, 1] = v.imag
    Q, mean, err = api.combine_sectors(prep, m, n_s, sums)
    Qo = OI.combine(prob, per, n)
    mo, eo = OI.mean_and_error(Qo)
    assert np.allclose(Q, Qo, rtol=1e-13, atol=1e-15)
    assert np.allclose(mean, mo, rtol=1e-13, atol=1e-15)
    assert np.allclose(np.hypot(err[:, 0], err[:, 1]), eo, rtol=1e-12)
    # equal sizes reduce to qmc_combine
    Q2, mean2, _ = api.combine_sectors(prep, m, [n] * prep.info.n_sectors, sums)
    Q3, mean3, _ = api.combine(prep, api.make_pass(n, [1] * 6, m), sums)
    assert np.array_equal(Q2, Q3) and np.array_equal(mean2, mean3)


def _prep_status(blob, kin, omin=0, omax=0):
    inv = np.ascontiguousarray(np.asarray(kin, dtype=np.float64))
    info = N.qmc_info()
    return N.lib().qmc_prepare(blob, len(blob), inv.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(inv), omin,
                               omax, None, 0, ctypes.byref(info))


def test_prepare_rejects_malformed_tables():
    cfg = W.CONFIG1
    blob = T.compile_integral(cfg.topology, T.zero_invariants_of(cfg.topology, cfg.point))
    kin = cfg.kin
    assert _prep_status(blob, kin) == 0
    assert _prep_status(b"XXXXXXXX" + blob[8:], kin) == N.QMC_ERR_TABLE          # bad magic
    assert _prep_status(blob[:-8], kin) == N.QMC_ERR_TABLE                         # truncated
    assert _prep_status(blob + b"\0" * 8, kin) == N.QMC_ERR_TABLE                  # trailing bytes
    assert _prep_status(blob, kin[:-1]) == N.QMC_ERR_ARG                           # wrong invariant count
    assert _prep_status(blob, kin, 0, 9) == N.QMC_ERR_ARG                          # too many orders
    meta, leaves = T.read_table(blob)
    bad = [T.SectorRecord(s.A.copy(), s.B.copy(), s.U, s.F, s.D) for s in leaves]
    bad[0].A[0], bad[0].B[0] = -2, -1                                      # alpha <= -2 in a deformed sector
    assert _prep_status(T.write_table(bad, meta), kin) == N.QMC_ERR_UNSUPPORTED
    bad[0].A[0] = -4                                                               # beyond alpha = -3
    assert _prep_status(T.write_table(bad, meta), kin) == N.QMC_ERR_UNSUPPORTED
    bad[0].B[0] = 0                                                                # alpha <= -2 unregulated
    assert _prep_status(T.write_table(bad, meta), kin) in (N.QMC_ERR_UNSUPPORTED, N.QMC_ERR_TABLE)
    bad[0].A[0] = -1
    bad[0].B[0] = 0                                                                # unregulated pole
    assert _prep_status(T.write_table(bad, meta), kin) == N.QMC_ERR_TABLE
    # kinematics that make the constant term of F vanish: msq = 0 for the massive box
    k2 = kin.copy()
    k2[list(cfg.topology.invariants).index("msq")] = 0.0
    assert _prep_status(blob, k2) == N.QMC_ERR_KINEMATICS
    nan = kin.copy()
    nan[0] = np.nan
    assert _prep_status(blob, nan) == N.QMC_ERR_ARG


def test_pass_validation_on_host():
    cfg = W.CONFIG1
    blob = T.compile_integral(cfg.topology, T.zero_invariants_of(cfg.topology, cfg.point))
    prep = api.prepare(blob, cfg.kin, 0, 0)
    good = api.make_pass(1021, [1, 2, 3, 4, 5, 6], 4)
    assert api.scratch_bytes(prep, good) > 0
    for bad in (api.make_pass(1, [1] * 6, 4), api.make_pass(1021, [0, 1, 1, 1, 1, 1], 4),
                api.make_pass(1021, [1] * 6, 0), api.make_pass(1021, [1] * 6, 4, transform_r=7),
                api.make_pass(1021, [1] * 6, 4, block=48), api.make_pass(1021, [1] * 6, 4, points_per_thread=65),
                api.make_pass(1021, [1] * 6, 4, evaluator=3)):
        assert api.scratch_bytes(prep, bad) == 0


def test_generated_fp32_passes_of_six_dimensional_sectors_take_at_most_128_threads():
    cfg = W.CONFIG2
    blob = T.compile_integral(cfg.topology, T.zero_invariants_of(cfg.topology, cfg.point))
    prep = api.prepare(blob, cfg.kin, cfg.order_min, cfg.order_max)
    z = [1, 2, 3, 4, 5, 6]
    for block, ok in ((128, True), (256, False)):
        gen = api.make_pass(1021, z, 4, precision=N.QMC_PREC_MIXED, block=block)
        assert (api.scratch_bytes(prep, gen) > 0) == ok
    for ev, prec in ((N.QMC_EVAL_TABLE, N.QMC_PREC_MIXED), (N.QMC_EVAL_AUTO, N.QMC_PREC_FP64)):
        assert api.scratch_bytes(prep, api.make_pass(1021, z, 4, precision=prec, block=256, evaluator=ev)) > 0
