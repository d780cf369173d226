"""FP32 passes with the generated evaluator (straight-line code per family, compiled with NVRTC at run time):
sums against the FP64 oracle on the same points, agreement with the table evaluator, the two-loop planar
double box, and the per-family module cache."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import integrate as OI  # noqa: E402
from oracle import lattice as OL  # noqa: E402
from paper_1508_02512_gb300 import _native as N  # noqa: E402
from paper_1508_02512_gb300 import api  # noqa: E402
from paper_1508_02512_gb300 import tables as T  # noqa: E402

LEGS0 = dict(pp1=0.0, pp2=0.0, pp3=0.0, pp4=0.0)
# FP32 evaluation error bound relative to the summed term magnitudes (as for the table evaluator)
MIXED_L1_BOUND = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def setup(cfg):
    blob = T.compile_integral(cfg.topology, T.zero_invariants_of(cfg.topology, cfg.point))
    prep = api.prepare(blob, cfg.kin, cfg.order_min, cfg.order_max)
    return prep, api.DeviceIntegral(prep)


def run(dev, p, shifts, lams):
    sh = torch.tensor(np.asarray(shifts, dtype=np.float64), device="cuda")
    lam = torch.tensor(np.asarray(lams, dtype=np.float64), device="cuda")
    sums, fails = dev.outputs(p)
    dev.eval_sums(p, sh, lam, sums, fails)
    torch.cuda.synchronize()
    s = sums.cpu().numpy()
    return s[..., 0] + 1j * s[..., 1], fails.cpu().numpy()


# a sector stays in FP32 while the probe finds sum |v32 - v64| <= 0.1 * rel_tol * sum |v64| (rel_tol = 1e-3)
PROBE_BUDGET = 1e-4


def probe_keeps(prep, dev, p, shifts, lams):
    """Sectors the FP32/FP64 probe (qmc_probe_precision, every point of the first shift when n <= 4096) keeps in
    FP32 at rel_tol 1e-3."""
    import ctypes
    ns, slots = prep.info.n_sectors, prep.info.n_slots
    out = torch.zeros((ns, slots, 4), dtype=torch.float64, device="cuda")
    sh = torch.tensor(np.asarray(shifts, dtype=np.float64), device="cuda")
    lam = torch.tensor(np.asarray(lams, dtype=np.float64), device="cuda")
    assert N.lib().qmc_probe_precision(prep.packed, dev.dpacked.data_ptr(), ctypes.byref(p), sh.data_ptr(),
                                       lam.data_ptr(), 4096, out.data_ptr(), None) == 0
    torch.cuda.synchronize()
    pr = out.cpu().numpy()
    return np.all(pr[:, :, 1] <= PROBE_BUDGET * pr[:, :, 0], axis=1)


def oracle_sums(cfg, n, z, shifts, lams):
    prob = OI.make_problem(cfg.topology, {**cfg.point, **LEGS0}, cfg.order_min, cfg.order_max)
    out = []
    for s, sec in enumerate(prob.sectors):
        o, l1, _, l1c = OI.lattice_sums(sec, prob.e4, n, z, shifts, lams[s], 3, prob.kmax, with_scale=True)
        out.append((o, l1c))
    return out


@pytest.mark.parametrize("cfg", [W.CONFIG0, W.CONFIG1, W.CONFIG2, W.CONFIG3], ids=lambda c: c.name)
def test_generated_sums_against_oracle_and_table_evaluator(cfg):
    prep, dev = setup(cfg)
    info = api.gen_compile(prep)
    print(f"{cfg.name}: generated evaluator compiled in {info.compile_ms:.0f} ms "
          f"({info.source_bytes} B source, {info.cubin_bytes} B cubin)")
    n = 1021 if cfg.topology.loops == 2 else 4093
    z = OL.cbc_plain(n, 6)
    shifts = W.shifts(23, 2 if cfg.topology.loops == 2 else 4)
    lams = [cfg.lam if cfg.lam > 0 else 0.0] * prep.info.n_sectors
    gen, _ = run(dev, api.make_pass(n, z, len(shifts), 3, precision=N.QMC_PREC_MIXED,
                                    evaluator=N.QMC_EVAL_GENERATED), shifts, lams)
    tab, _ = run(dev, api.make_pass(n, z, len(shifts), 3, precision=N.QMC_PREC_MIXED,
                                    evaluator=N.QMC_EVAL_TABLE), shifts, lams)
    keep = probe_keeps(prep, dev, api.make_pass(n, z, len(shifts), 3, precision=N.QMC_PREC_MIXED), shifts, lams)
    worst_gen = worst_tab = worst_diff = worst_kept = 0.0
    per_sector = []
    for s, (o, l1c) in enumerate(oracle_sums(cfg, n, z, shifts, lams)):
        k = o.shape[1]
        scale = np.maximum(l1c, 1e-300)
        eg = float((np.abs(gen[s, :, :k] - o) / scale).max())
        et = float((np.abs(tab[s, :, :k] - o) / scale).max())
        ed = float((np.abs(gen[s, :, :k] - tab[s, :, :k]) / scale).max())
        per_sector.append(eg)
        worst_gen, worst_tab, worst_diff = max(worst_gen, eg), max(worst_tab, et), max(worst_diff, ed)
        if keep[s]:
            worst_kept = max(worst_kept, eg)
    print(f"{cfg.name}: |gen-oracle|/mag {worst_gen:.2e} (sectors the probe keeps in FP32: {worst_kept:.2e}, "
          f"{int(keep.sum())}/{len(keep)})  |table-oracle|/mag {worst_tab:.2e}  |gen-table|/mag {worst_diff:.2e}  "
          f"per-sector median {np.median(per_sector):.2e}")
    if cfg.topology.loops == 1:
        # same products and FMAs per term, summed in another order: the two FP32 evaluators agree to FP32 rounding
        assert worst_diff <= MIXED_L1_BOUND
        assert worst_gen <= MIXED_L1_BOUND
    else:
        # two-loop sectors: the sectors the probe keeps in FP32 meet its budget (1e-4 of the summed magnitudes at
        # rel_tol 1e-3) on the probed first shift, every point of it sampled; the second shift is held to twice
        # that; the other sectors run in FP64
        assert worst_kept <= 2 * PROBE_BUDGET


def test_generated_module_is_cached_per_family():
    prep, dev = setup(W.CONFIG1)
    a = api.gen_compile(prep)
    kin2 = W.kinematics(W.CONFIG1.topology, **{**W.CONFIG1.point, "s": 7.0, "t": -2.0})
    blob = T.compile_integral(W.CONFIG1.topology, T.zero_invariants_of(W.CONFIG1.topology, W.CONFIG1.point))
    b = api.gen_compile(api.prepare(blob, kin2, 0, 0))
    assert b.cached == 1 and b.family == a.family


@pytest.mark.parametrize("cfg", [W.CONFIG0, W.CONFIG1, W.CONFIG2], ids=lambda c: c.name)
def test_generated_fp64_sums_match_oracle_to_1e12(cfg):
    prep, dev = setup(cfg)
    info = api.gen_compile(prep, precision=N.QMC_PREC_FP64)
    print(f"{cfg.name}: FP64 generated evaluator compiled in {info.compile_ms:.0f} ms")
    n = 1021 if cfg.topology.loops == 2 else 4093
    z = OL.cbc_plain(n, 6)
    shifts = W.shifts(29, 2 if cfg.topology.loops == 2 else 4)
    lams = [cfg.lam if cfg.lam > 0 else 0.0] * prep.info.n_sectors
    gen, gf = run(dev, api.make_pass(n, z, len(shifts), 3, evaluator=N.QMC_EVAL_GENERATED), shifts, lams)
    tab, tf = run(dev, api.make_pass(n, z, len(shifts), 3, evaluator=N.QMC_EVAL_TABLE), shifts, lams)
    assert np.array_equal(gf, tf)
    worst = 0.0
    for s, (o, l1c) in enumerate(oracle_sums(cfg, n, z, shifts, lams)):
        k = o.shape[1]
        worst = max(worst, float((np.abs(gen[s, :, :k] - o) / np.maximum(l1c, 1e-300)).max()))
    print(f"{cfg.name}: FP64 generated |gpu-oracle| / term magnitudes = {worst:.2e}")
    assert worst <= 1e-12


def test_generated_fp32_on_geometric_sectors_with_four_poles():
    """Mixed-precision (FP32) generated evaluation of the massless double box of Table 2 (geometric strategy,
    sectors with up to four singular variables) against the FP64 oracle, at the FP32 bound."""
    topo, pt = W.double_box_planar(False), W.PAPER_IB_POINTS["-1,0,0,-1"]
    blob = T.compile_integral(topo, T.zero_invariants_of(topo, pt), strategy="geometric")
    prep = api.prepare(blob, W.kinematics(topo, **pt), -4, 0)
    dev = api.DeviceIntegral(prep)
    n = 251
    z = OL.cbc_plain(n, 6)
    shifts = W.shifts(29, 2)
    lams = [0.0] * prep.info.n_sectors
    gen, fails = run(dev, api.make_pass(n, z, len(shifts), 3, precision=N.QMC_PREC_MIXED,
                                        evaluator=N.QMC_EVAL_GENERATED), shifts, lams)
    assert not fails.any()
    prob = OI.make_problem(topo, pt, -4, 0, "geometric")
    worst = 0.0
    for s, sec in enumerate(prob.sectors):
        o, l1, _, l1c = OI.lattice_sums(sec, prob.e4, n, z, shifts, 0.0, 3, prob.kmax, with_scale=True)
        k = o.shape[1]
        worst = max(worst, float((np.abs(gen[s, :, :k] - o) / np.maximum(l1c, 1e-300)).max()))
    print(f"massless double box, FP32 generated: worst |gen-oracle|/mag {worst:.2e}")
    assert worst < MIXED_L1_BOUND
