"""GPU parity: the CUDA path (through the C ABI) against the oracle on identical inputs.

Both sides get the same integral definition (workloads), lattice size, generating vector, shifts and per-sector
lambda; each decomposes the integral itself (the two decompositions are checked equal, bit for bit, by a CPU
test).  Tolerance (FP64): per sector, shift and order, |GPU - oracle| <= 1e-12 * the summed magnitude of the terms
that the endpoint subtraction cancels (Sec. II, after Eq. 12: the subtracted remainder suffers from large
cancellation, and the kernel's regrouped subtraction rounds differently from the oracle's nested form); for
sectors without subtraction that scale is the plain L1 sum of the point values.  The plain ratio
|GPU - oracle| / sum_i |value_i| is reported beside it and bounded too: by 1e-12 where the two scales agree within
a factor 10, and by 1e-12 times their ratio elsewhere.

Sizes span several work items (blockDim * points_per_thread lattice points each) with a ragged last item; the
bench's full-size workload (massive box, n = 16777213, 16 shifts) is checked on sampled points, by determinism
across launch shapes, and by agreement with the oracle's estimate of the same integral within the errors.
"""
import math

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import integrate as OI  # noqa: E402
from oracle import lattice as OL  # noqa: E402
from paper_1508_02512_gb300 import api  # noqa: E402
from paper_1508_02512_gb300 import tables as T  # noqa: E402

LEGS0 = dict(pp1=0.0, pp2=0.0, pp3=0.0, pp4=0.0)
TOL = 1e-12
N_EVAL_TABLE, N_EVAL_GENERATED = 1, 2   # qmc_pass.evaluator: QMC_EVAL_TABLE, QMC_EVAL_GENERATED


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_02512_gb300 import _native
    _native.lib()


def setup_pair(topo, point, omin, omax, strategy="iterated"):
    blob = T.compile_integral(topo, T.zero_invariants_of(topo, point), strategy=strategy)
    kin = W.kinematics(topo, **point)
    prep = api.prepare(blob, kin, omin, omax)
    dev = api.DeviceIntegral(prep)
    prob = OI.make_problem(topo, point, omin, omax, strategy)
    assert prep.info.n_sectors == len(prob.sectors)
    return prep, dev, prob


def gpu_sums(dev, p, shifts, lams):
    sh = torch.tensor(np.asarray(shifts, dtype=np.float64), device="cuda")
    lam = torch.tensor(np.asarray(lams, dtype=np.float64), device="cuda")
    sums, fails = dev.outputs(p)
    dev.eval_sums(p, sh, lam, sums, fails)
    torch.cuda.synchronize()
    s = sums.cpu().numpy()
    return s[..., 0] + 1j * s[..., 1], fails.cpu().numpy()


def apply_kind1_phase(prep, prob, sums):
    """Kind-1 sectors (F < 0 everywhere) leave the factor exp(i pi eF(eps)) to the host; apply it here."""
    out = sums.copy()
    eF0, eF1 = prob.e4[2], prob.e4[3]
    slots = sums.shape[2]
    ph = np.array([(-1) ** eF0 * (1j * math.pi * eF1) ** k / math.factorial(k) for k in range(slots)])
    for s in range(prep.info.n_sectors):
        if prep.sector(s).kind == 1:
            for n in range(slots):
                out[s, :, n] = sum(ph[q] * sums[s, :, n - q] for q in range(n + 1))
    return out


def compare(prep, prob, sums, lams, n, z, shifts, r=3, tol=TOL):
    worst = plain = plain0 = 0.0
    for s, sec in enumerate(prob.sectors):
        d = prep.sector(s)
        assert d.kind == sec.kind and d.sigma == sec.sigma
        osum, l1, ofail, l1c = OI.lattice_sums(sec, prob.e4, n, z, shifts, lams[s], r, prob.kmax, with_scale=True)
        nout = osum.shape[1]
        g = sums[s, :, :nout]
        err = np.abs(g - osum)
        scale = np.maximum(l1c, 1e-300)
        worst = max(worst, float(np.max(err / scale)))
        assert np.all(err <= tol * scale + 1e-300), (s, float(np.max(err / scale)))
        # the plain ratio: against sum |values|, bounded by tol where the two scales agree within 10x, otherwise by
        # tol times their ratio (the terms that cancel set the rounding)
        l1p = np.maximum(l1, 1e-300)
        pr = err / l1p
        plain = max(plain, float(np.max(pr)))
        if sec.sigma == 0:
            plain0 = max(plain0, float(np.max(pr)))
        allowed = tol * np.where(scale <= 10 * l1p, 1.0, scale / l1p)
        assert np.all(pr <= allowed + 1e-300), (s, float(np.max(pr)))
        # slots beyond the sector's orders stay zero
        assert np.all(sums[s, :, nout:] == 0)
    return worst, plain, plain0


def report(worst):
    w, plain, plain0 = worst
    return (f"worst |gpu-oracle| / cancellation scale = {w:.2e}; / plain L1 = {plain:.2e} "
            f"(sectors without subtraction: {plain0:.2e})")


CASES = [
    # name, topology, point, orders, lambda, lattice size, block, points/thread
    ("massless_box", W.box(False), dict(s=-3.0, t=-2.0, **LEGS0), (-2, 0), 0.0, 4093, 128, 8),
    ("massive_box_phys", W.box(True), dict(s=5.0, t=-1.5, msq=1.0, **LEGS0), (0, 0), 0.5, 4093, 64, 3),
    ("massive_box_orders", W.box(True), dict(s=5.0, t=-1.5, msq=1.0, **LEGS0), (0, 2), 0.5, 2039, 96, 5),
    ("triangle_phys", W.triangle_massive(), dict(pp3=5.0, msq=1.0), (0, 1), 0.4, 1021, 32, 1),
    ("bubble_massive", W.bubble(True), dict(pp1=5.0, msq=1.0), (-1, 1), 0.5, 2039, 128, 7),
    ("massless_bubble", W.bubble(False), dict(pp1=-2.0), (-1, 2), 0.0, 1021, 64, 4),
    ("massless_bubble_negative_F", W.bubble(False), dict(pp1=2.0), (-1, 2), 0.0, 1021, 64, 4),
    ("planar_dbox", W.double_box_planar(True), dict(s=6.0, t=-2.0, msq=1.0, **LEGS0), (-2, 0), 0.25, 251, 64, 2),
    ("nonplanar_dbox", W.double_box_nonplanar(True), dict(s=6.0, t=-2.0, msq=1.0, **LEGS0), (-2, 0), 0.25, 251,
     128, 1),
    # the paper's gg -> HH point of Tables 3-4 (Sec. IV): Higgs-mass legs p3^2 = p4^2 = M_H^2, another zero pattern
    ("paper_IC_planar_hh", W.double_box_planar(True), W.PAPER_HH_POINT, (-2, 0), 0.25, 251, 64, 3),
    ("paper_ID_nonplanar_hh", W.double_box_nonplanar(True), W.PAPER_HH_POINT, (-2, 0), 0.25, 127, 128, 1),
]


@pytest.mark.parametrize("name,topo,pt,orders,lam,n,block,P", CASES, ids=[c[0] for c in CASES])
def test_sums_match_oracle(name, topo, pt, orders, lam, n, block, P):
    prep, dev, prob = setup_pair(topo, pt, *orders)
    z = OL.cbc_plain(n, 6)
    m = 5
    shifts = W.shifts(11, m)
    lams = [lam] * prep.info.n_sectors
    p = api.make_pass(n, z, m, 3, block=block, points_per_thread=P)
    sums, fails = gpu_sums(dev, p, shifts, lams)
    sums = apply_kind1_phase(prep, prob, sums)
    worst = compare(prep, prob, sums, lams, n, z, shifts)
    print(f"{name}: {report(worst)}")


GEOMETRIC_CASES = [
    # name, topology, point, orders, lambda, lattice size, block, points/thread
    ("massless_dbox_table2", W.double_box_planar(False), W.PAPER_IB_POINTS["-1,0,0,-1"], (-4, 0), 0.0, 251, 64, 2),
    ("massless_dbox_table2_col2", W.double_box_planar(False), W.PAPER_IB_POINTS["0,-1,0,-1"], (-4, 0), 0.0, 127,
     128, 1),
    ("planar_dbox", W.double_box_planar(True), dict(s=6.0, t=-2.0, msq=1.0, **LEGS0), (-2, 0), 0.25, 251, 64, 2),
]


@pytest.mark.parametrize("evaluator", [N_EVAL_TABLE, N_EVAL_GENERATED], ids=["table", "generated"])
@pytest.mark.parametrize("name,topo,pt,orders,lam,n,block,P", GEOMETRIC_CASES, ids=[c[0] for c in GEOMETRIC_CASES])
def test_geometric_sectors_match_oracle(name, topo, pt, orders, lam, n, block, P, evaluator):
    """Tables of the geometric strategy (poles to eps^-4 in the massless double box: up to 16 subtraction
    subsets per point, five series slots) through both FP64 evaluators."""
    prep, dev, prob = setup_pair(topo, pt, *orders, strategy="geometric")
    z = OL.cbc_plain(n, 6)
    shifts = W.shifts(13, 3)
    lams = [lam] * prep.info.n_sectors
    p = api.make_pass(n, z, len(shifts), 3, block=block, points_per_thread=P, evaluator=evaluator)
    sums, fails = gpu_sums(dev, p, shifts, lams)
    assert not fails.any()
    sums = apply_kind1_phase(prep, prob, sums)
    worst = compare(prep, prob, sums, lams, n, z, shifts)
    print(f"{name} ({'table' if evaluator == N_EVAL_TABLE else 'generated'}): {prep.info.n_sectors} sectors, "
          f"{report(worst)}")


def test_edge_single_shift_tiny_lattice_and_transforms():
    prep, dev, prob = setup_pair(W.box(False), dict(s=-3.0, t=-2.0, **LEGS0), -2, 0)
    for n, r in ((31, 0), (61, 1), (127, 2)):
        z = OL.cbc_plain(n, 6)
        shifts = W.shifts(3, 1)
        lams = [0.0] * prep.info.n_sectors
        p = api.make_pass(n, z, 1, r, block=32, points_per_thread=1)
        sums, _ = gpu_sums(dev, p, shifts, lams)
        compare(prep, prob, sums, lams, n, z, shifts, r=r)


def test_zero_shift_hits_the_origin():
    """Delta = 0 puts lattice point 0 on the corner of the cube, where the transform weight vanishes."""
    prep, dev, prob = setup_pair(W.box(True), dict(s=5.0, t=-1.5, msq=1.0, **LEGS0), 0, 0)
    n = 1021
    z = OL.cbc_plain(n, 6)
    shifts = np.zeros((2, 6))
    shifts[1] = W.shifts(4, 1)[0]
    lams = [0.5] * 4
    p = api.make_pass(n, z, 2, 3, block=64, points_per_thread=4)
    sums, _ = gpu_sums(dev, p, shifts, lams)
    compare(prep, prob, sums, lams, n, z, shifts)


def test_determinism_across_launch_shapes():
    prep, dev, prob = setup_pair(W.box(True), dict(s=5.0, t=-1.5, msq=1.0, **LEGS0), 0, 0)
    n = 65521
    z = api.builtin_lattices()[6][1]
    shifts = W.shifts(5, 16)
    lams = [0.5] * 4
    base = None
    for grid in (0, 1, 7, 300):
        p = api.make_pass(n, z, 16, 3, block=128, points_per_thread=8, grid=grid)
        sums, _ = gpu_sums(dev, p, shifts, lams)
        if base is None:
            base = sums
        assert np.array_equal(sums, base)


def test_full_size_bench_workload_sampled_points():
    """Massive box at the bench size n = 16777213 (16 shifts): per-point values at sampled lattice indices
    against the oracle, computed independently from (i, z, n, Delta)."""
    cfg = W.CONFIG1
    pt = {**cfg.point, **LEGS0}
    prep, dev, prob = setup_pair(cfg.topology, pt, 0, 0)
    lat = dict(api.builtin_lattices())
    n = OL.prime_below(1 << 24)
    z = lat[n]
    shifts = W.shifts(cfg.seed, 16)
    rng = np.random.default_rng(0)
    idx = np.concatenate([[0, 1, n - 1], rng.integers(0, n, size=509)]).astype(np.int64)
    p = api.make_pass(n, z, 16, 3)
    slots = prep.info.n_slots
    for s, sec in enumerate(prob.sectors):
        for k in (0, 7, 15):
            out = torch.zeros((len(idx), slots, 2), dtype=torch.float64, device="cuda")
            fl = torch.zeros(len(idx), dtype=torch.int32, device="cuda")
            dev.eval_points(s, p, torch.tensor(shifts[k], device="cuda"), 0.5, torch.tensor(idx, device="cuda"),
                            out, fl)
            torch.cuda.synchronize()
            g = out.cpu().numpy()
            g = g[..., 0] + 1j * g[..., 1]
            x = ((idx[:, None] * np.asarray(z[:3], dtype=np.int64)[None, :]) % n) / n + shifts[k][None, :3]
            x = np.where(x >= 1.0, x - 1.0, x)
            ref = np.array([OI.point_series(sec, prob.e4, x[j], 0.5, 3, prob.kmax)[0][0] for j in range(len(idx))])
            # 1e-12 of each value, with the sample's mean magnitude as floor (like the sums' L1 normalisation):
            # near-corner points carry a vanishing transform weight and are not judged relative to themselves
            floor = np.mean(np.abs(ref))
            bad = np.abs(g[:, 0] - ref) > 1e-12 * np.maximum(np.abs(ref), floor)
            assert not bad.any(), (s, k, idx[bad][:5], g[bad, 0][:5], ref[bad][:5])


def test_full_size_bench_workload_estimate():
    """The full-size pass estimates the same integral as the oracle at a smaller lattice (within errors), and
    the two sets of per-shift estimates are consistent with their stated errors."""
    cfg = W.CONFIG1
    pt = {**cfg.point, **LEGS0}
    prep, dev, prob = setup_pair(cfg.topology, pt, 0, 0)
    lat = dict(api.builtin_lattices())
    n = OL.prime_below(1 << 24)
    shifts = W.shifts(cfg.seed, 16)
    p = api.make_pass(n, lat[n], 16, 3)
    sums, fails = gpu_sums(dev, p, shifts, [0.5] * 4)
    assert fails.sum() == 0
    Q, mean, err = api.combine(prep, p, np.stack([sums.real, sums.imag], axis=-1))
    n_o = OL.prime_below(1 << 14)
    om, oe, _, _, of = OI.integrate(prob, n_o, lat[n_o], W.shifts(99, 16), 0.5, 3)
    e = math.hypot(err[0][0], err[0][1])
    assert abs(mean[0] - om[0]) <= 5 * math.hypot(e, oe[0])
    assert e < 1e-7 * abs(mean[0])


def test_context_integrate_massless_box_closed_form():
    from scipy import special as sp
    import cmath
    cfg = W.CONFIG0
    blob = T.compile_integral(cfg.topology, T.zero_invariants_of(cfg.topology, cfg.point))
    ctx = api.Context()
    iid = ctx.load_sectors(blob)
    ctx.set_kinematics(iid, cfg.kin, -2, 0)
    r = ctx.integrate(iid, rel_tol=1e-7, n_shifts=8, seed=1, lam=0.5, ladder_start=2)
    val, err = api.result_arrays(r)
    assert r.status == 0, r.status

    def f(e):
        cg = sp.gamma(1 + e) * sp.gamma(1 - e) ** 2 / sp.gamma(1 - 2 * e)
        return cg / 6.0 * (2 / e ** 2 * (3.0 ** (-e) + 2.0 ** (-e)) - cmath.log(1.5) ** 2 - math.pi ** 2) * e ** 2

    th = 2 * np.pi * np.arange(64) / 64
    eps = 0.25 * np.exp(1j * th)
    vals = np.array([f(e) for e in eps])
    ref = np.array([np.mean(vals * eps ** (-k)) for k in range(3)])
    e = np.hypot(err[:, 0], err[:, 1])
    assert np.all(np.abs(val - ref) <= 5 * e + 1e-10), (val, ref, e)
    ctx.close()


def test_context_integrate_massive_box_to_1e3():
    cfg = W.CONFIG1
    blob = T.compile_integral(cfg.topology, T.zero_invariants_of(cfg.topology, cfg.point))
    ctx = api.Context()
    iid = ctx.load_sectors(blob)
    ctx.set_kinematics(iid, cfg.kin, 0, 0)
    r = ctx.integrate(iid, rel_tol=1e-3, n_shifts=16, seed=3, lam=0.5, ladder_start=0)
    assert r.status == 0
    val, err = api.result_arrays(r)
    prob = OI.make_problem(cfg.topology, {**cfg.point, **LEGS0}, 0, 0)
    om, oe, _, _, _ = OI.integrate(prob, 4093, OL.cbc_plain(4093, 6), W.shifts(8, 16), 0.5, 3)
    assert abs(val[0] - om[0]) <= 5 * math.hypot(math.hypot(*err[0]), oe[0])
    assert math.hypot(*err[0]) <= 1e-3 * abs(val[0])
    ctx.close()
