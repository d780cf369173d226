"""Mixed-precision path (FP32 evaluation, FP64 lattice arithmetic and accumulation, FP64 re-runs of sectors over
the FP32 budget): its error against the FP64 oracle is measured and bounded per order, the probe flags sectors
correctly, a mixed pass with FP64-forced sectors reproduces the FP64 kernel on those sectors, and integration to
1e-3 in mixed precision agrees with the closed form / the FP64 result."""
import ctypes
import math

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


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def setup(cfg):
    blob = T.compile_integral(cfg.topology, T.zero_invariants_of(cfg.topology, cfg.point))
    prep = api.prepare(blob, cfg.kin, cfg.order_min, cfg.order_max)
    return blob, prep, api.DeviceIntegral(prep)


def run_pass(dev, p, shifts, lams, prec=None):
    sh = torch.tensor(np.asarray(shifts, dtype=np.float64), device="cuda")
    lam = torch.tensor(np.asarray(lams, dtype=np.float64), device="cuda")
    keep = None
    if prec is not None:
        keep = torch.tensor(np.asarray(prec, dtype=np.int32), device="cuda")
        p.sector_precision = keep.data_ptr()
    sums, fails = dev.outputs(p)
    dev.eval_sums(p, sh, lam, sums, fails)
    torch.cuda.synchronize()
    p.sector_precision = None
    s = sums.cpu().numpy()
    return s[..., 0] + 1j * s[..., 1], fails.cpu().numpy()


# error budget of the FP32 evaluation, per order, relative to the summed magnitudes (L1): measured values are
# printed; the bound is what the mixed path promises for sectors it keeps in FP32
MIXED_L1_BOUND = 2e-5


@pytest.mark.parametrize("cfg", [W.CONFIG1, W.CONFIG0], ids=lambda c: c.name)
def test_mixed_sums_error_against_oracle(cfg):
    blob, prep, dev = setup(cfg)
    prob = OI.make_problem(cfg.topology, {**cfg.point, **LEGS0}, cfg.order_min, cfg.order_max)
    n = 4093
    z = OL.cbc_plain(n, 6)
    shifts = W.shifts(31, 4)
    lam = cfg.lam if cfg.lam > 0 else 0.0
    lams = [lam] * prep.info.n_sectors
    p = api.make_pass(n, z, 4, 3, precision=N.QMC_PREC_MIXED)
    sums, fails = run_pass(dev, p, shifts, lams)
    worst = np.zeros(prep.info.n_slots)
    for s, sec in enumerate(prob.sectors):
        o, l1, _, l1c = OI.lattice_sums(sec, prob.e4, n, z, shifts, lams[s], 3, prob.kmax, with_scale=True)
        rel = np.abs(sums[s, :, : o.shape[1]] - o) / np.maximum(l1c, 1e-300)
        worst[: o.shape[1]] = np.maximum(worst[: o.shape[1]], rel.max(axis=0))
    print(f"{cfg.name}: mixed |gpu-oracle| / term magnitudes per slot = {worst}")
    assert np.all(worst <= MIXED_L1_BOUND), worst


def test_probe_reports_fp32_discrepancy_and_forced_fp64_matches_fp64_kernel():
    cfg = W.CONFIG1
    blob, prep, dev = setup(cfg)
    ns, slots = prep.info.n_sectors, prep.info.n_slots
    n = 65521
    z = dict(api.builtin_lattices())[n]
    shifts = W.shifts(5, 8)
    lams = [0.5] * ns
    p = api.make_pass(n, z, 8, 3, precision=N.QMC_PREC_MIXED, points_per_thread=16)
    out = torch.zeros((ns, slots, 4), dtype=torch.float64, device="cuda")
    sh = torch.tensor(shifts, device="cuda")
    lam = torch.tensor(lams, device="cuda", dtype=torch.float64)
    rc = N.lib().qmc_probe_precision(prep.packed, dev.dpacked.data_ptr(), ctypes.byref(p), sh.data_ptr(),
                                     lam.data_ptr(), 4096, out.data_ptr(), None)
    assert rc == 0
    torch.cuda.synchronize()
    pr = out.cpu().numpy()
    rel = pr[:, 0, 1] / pr[:, 0, 0]
    print("probe sum|v32-v64|/sum|v64| per sector:", rel)
    assert np.all(pr[:, 0, 0] > 0) and np.all(rel < 1e-4) and np.all(rel > 0)
    # sectors 0 and 2 forced to FP64 inside a mixed pass equal the FP64 kernel with the same chunking
    mixed, _ = run_pass(dev, p, shifts, lams, prec=[0, 1, 0, 1])
    p64 = api.make_pass(n, z, 8, 3, precision=N.QMC_PREC_FP64, points_per_thread=16)
    ref, _ = run_pass(dev, p64, shifts, lams)
    assert np.array_equal(mixed[[0, 2]], ref[[0, 2]])
    assert not np.array_equal(mixed[[1, 3]], ref[[1, 3]])
    assert np.max(np.abs(mixed[[1, 3]] - ref[[1, 3]]) / np.abs(ref[[1, 3]])) < 1e-5


def test_mixed_integrate_massless_box_to_closed_form():
    from scipy import special as sp
    import cmath
    cfg = W.CONFIG0
    blob, prep, dev = setup(cfg)
    ctx = api.Context()
    iid = ctx.load_sectors(blob)
    ctx.set_kinematics(iid, cfg.kin, -2, 0)
    r = ctx.integrate(iid, rel_tol=1e-4, n_shifts=8, seed=3, precision=N.QMC_PREC_MIXED)
    assert r.status == 0
    val, err = api.result_arrays(r)

    def f(e):
        cg = sp.gamma(1 + e) * sp.gamma(1 - e) ** 2 / sp.gamma(1 - 2 * e)
        return cg / 6.0 * (2 / e ** 2 * (3.0 ** (-e) + 2.0 ** (-e)) - cmath.log(1.5) ** 2 - math.pi ** 2) * e ** 2

    th = 2 * np.pi * np.arange(64) / 64
    eps = 0.25 * np.exp(1j * th)
    vals = np.array([f(e) for e in eps])
    ref = np.array([np.mean(vals * eps ** (-k)) for k in range(3)])
    e = np.hypot(err[:, 0], err[:, 1])
    print("mixed massless box:", val, "closed form", ref, "err", e, "fp64 sectors", r.fp64_reruns)
    assert np.all(np.abs(val - ref) <= 5 * e + 2e-4 * np.abs(ref))
    ctx.close()


def test_fp32_overflow_missed_by_the_probe_reruns_the_sector_in_fp64():
    """The Euclidean massless box with s = -3e-20, t = -2: in the sectors where s multiplies the constant term of
    F, F is O(1e-20) near the faces where the t term vanishes, and F^-2 overflows FP32 there (largest float
    ~3.4e38) while FP64 holds it.  A probe of one point per sector misses those points, so FP32 sums come out
    non-finite; the integration moves those sectors to FP64 and evaluates the step again.  Its results stay finite
    and agree with the FP64 integration on the same lattices (both capped at n = 65521; this kinematics needs far
    larger lattices to converge).  With s and t scaled by 1e-160, F^-2 overflows FP64 as well and the integration
    stops with QMC_ERR_NONFINITE."""
    cfg = W.CONFIG0
    topo = cfg.topology
    blob = T.compile_integral(topo, T.zero_invariants_of(topo, cfg.point))

    def run(point, precision, **kw):
        ctx = api.Context()
        try:
            iid = ctx.load_sectors(blob)
            ctx.set_kinematics(iid, W.kinematics(topo, **point), -2, 0)
            return ctx.integrate(iid, rel_tol=1e-3, n_shifts=8, seed=3, precision=precision, max_n=65536, **kw)
        finally:
            ctx.close()

    pt = dict(s=-3e-20, t=-2.0)
    r64 = run(pt, N.QMC_PREC_FP64)
    r32 = run(pt, N.QMC_PREC_MIXED, probe_samples=1)
    assert r64.status in (0, N.QMC_ERR_NOT_CONVERGED) and r32.status == r64.status
    assert r64.nonfinite_sectors == 0 and r32.nonfinite_sectors > 0 and r32.fp64_reruns >= r32.nonfinite_sectors
    v64, e64 = api.result_arrays(r64)
    v32, e32 = api.result_arrays(r32)
    e = np.hypot(np.hypot(e64[:, 0], e64[:, 1]), np.hypot(e32[:, 0], e32[:, 1]))
    print(f"s = -3e-20: {r32.nonfinite_sectors} sectors came out non-finite in FP32 and ran again in FP64; "
          f"mixed {v32} vs FP64 {v64} (+- {e})")
    assert np.all(np.isfinite(v32)) and np.all(np.abs(v32 - v64) <= 5 * e + 1e-12 * np.abs(v64))
    with pytest.raises(N.QMCError) as info:
        run(dict(s=-3e-160, t=-2e-160), N.QMC_PREC_FP64)
    assert info.value.status == N.QMC_ERR_NONFINITE


def test_mixed_integrate_massive_box_matches_fp64():
    cfg = W.CONFIG1
    blob, prep, dev = setup(cfg)
    ctx = api.Context()
    iid = ctx.load_sectors(blob)
    ctx.set_kinematics(iid, cfg.kin, 0, 0)
    r64 = ctx.integrate(iid, rel_tol=1e-5, n_shifts=16, seed=4, precision=N.QMC_PREC_FP64)
    r32 = ctx.integrate(iid, rel_tol=1e-5, n_shifts=16, seed=4, precision=N.QMC_PREC_MIXED)
    assert r64.status == 0 and r32.status == 0
    v64, e64 = api.result_arrays(r64)
    v32, e32 = api.result_arrays(r32)
    print("massive box fp64", v64, "mixed", v32, "fp64 sectors in mixed", r32.fp64_reruns)
    assert abs(v32[0] - v64[0]) <= 5 * math.hypot(math.hypot(*e64[0]), math.hypot(*e32[0])) + 1e-5 * abs(v64[0])
    ctx.close()


# rel_tol 1e-3 with the library's default fp32_budget of 0.1: a sector stays in FP32 while its probe finds
# sum |v32 - v64| <= 1e-4 sum |v64| in every slot
PROBE_BUDGET = 1e-4


@pytest.mark.parametrize("cfg", [W.CONFIG2, W.CONFIG3], ids=lambda c: c.name)
def test_two_loop_mixed_sums_within_the_probe_budget(cfg):
    """Mixed (FP32, generated evaluator) sums of the two-loop double boxes against the FP64 oracle on identical
    points.  The probe samples every point of the first shift here (n <= 4096), so for each sector it keeps in
    FP32 the first shift's sums are guaranteed within the budget of its summed magnitudes per slot, and the second
    shift is held to twice that.  The error of every sector, kept or not, is printed per order."""
    blob, prep, dev = setup(cfg)
    api.gen_compile(prep)
    ns, slots = prep.info.n_sectors, prep.info.n_slots
    prob = OI.make_problem(cfg.topology, {**cfg.point, **LEGS0}, cfg.order_min, cfg.order_max)
    n = 1021
    z = OL.cbc_plain(n, 6)
    shifts = W.shifts(37, 2)
    lams = [cfg.lam] * ns
    p = api.make_pass(n, z, 2, 3, precision=N.QMC_PREC_MIXED, evaluator=N.QMC_EVAL_GENERATED)
    out = torch.zeros((ns, slots, 4), dtype=torch.float64, device="cuda")
    sh = torch.tensor(shifts, device="cuda")
    lam = torch.tensor(lams, device="cuda", dtype=torch.float64)
    assert N.lib().qmc_probe_precision(prep.packed, dev.dpacked.data_ptr(), ctypes.byref(p), sh.data_ptr(),
                                       lam.data_ptr(), 4096, out.data_ptr(), None) == 0
    torch.cuda.synchronize()
    pr = out.cpu().numpy()
    keep = np.all(pr[:, :, 1] <= PROBE_BUDGET * pr[:, :, 0], axis=1)
    sums, fails = run_pass(dev, p, shifts, lams)
    worst_kept = np.zeros(slots)
    worst_all = np.zeros(slots)
    for s, sec in enumerate(prob.sectors):
        o, l1, _, l1c = OI.lattice_sums(sec, prob.e4, n, z, shifts, lams[s], 3, prob.kmax, with_scale=True)
        k = o.shape[1]
        rel = np.abs(sums[s, :, :k] - o) / np.maximum(l1, 1e-300)
        worst_all[:k] = np.maximum(worst_all[:k], rel.max(axis=0))
        if keep[s]:
            worst_kept[:k] = np.maximum(worst_kept[:k], rel.max(axis=0))
            assert np.all(rel[0] <= PROBE_BUDGET * (1 + 1e-6)), (s, rel[0])
            assert np.all(rel[1] <= 2 * PROBE_BUDGET), (s, rel[1])
    print(f"{cfg.name}: {int(keep.sum())}/{ns} sectors kept in FP32; mixed |gpu-oracle| / sum|values| per slot: "
          f"kept {worst_kept}, all sectors {worst_all}")
    assert keep.sum() >= ns // 2
