"""FP64 islands of the mixed pass.  The endpoint subtraction of Eq. 11 cancels near the faces t_j = 0 of a
sector's singular variables (the remark after Eq. 12), and FP32 loses its digits there; a sector can stay in FP32
with its island points -- prod_j (k_j + 1) / n below 10^-(L+1) over the singular variables -- evaluated in FP64
(precision code 2 + L).

Checked here:
* the probe's island bins (qmc_probe_islands) count, bin by bin, exactly the sample points the criterion restated
  in numpy (tests/islands_ref.py) puts there, and their errors add up to the probe's own sum |v32 - v64|;
* passes with islands against the oracle on the same points: sectors without singular variables give the FP32
  pass bit for bit (they have no islands), every sector stays within the FP32 bound of the mixed path (a point
  dropped or counted twice moves a sum by ~1/n of it, far above that bound), and on the Table 2 sectors with three
  or four singular variables the islands lower the FP32 error of the sums;
* island passes are deterministic and independent of the launch shape;
* integration of a Table 2 point in mixed precision uses islands and agrees with FP64."""
import ctypes
import math

import numpy as np
import pytest

import islands_ref as R
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import integrate as OI  # noqa: E402
from oracle import lattice as OL  # noqa: E402
from paper_1508_02512_gb300 import _native as N  # noqa: E402
from paper_1508_02512_gb300 import api  # noqa: E402
from paper_1508_02512_gb300 import tables as T  # noqa: E402

LEGS0 = dict(pp1=0.0, pp2=0.0, pp3=0.0, pp4=0.0)
MIXED_L1_BOUND = 2e-5  # FP32 error bound of the mixed path relative to the summed term magnitudes (one loop)
TABLE2 = W.PAPER_IB_POINTS["-1,0,0,-1"]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def setup(topo, point, omin, omax, strategy="iterated"):
    blob = T.compile_integral(topo, T.zero_invariants_of(topo, point), strategy=strategy)
    prep = api.prepare(blob, W.kinematics(topo, **point), omin, omax)
    prob = OI.make_problem(topo, point, omin, omax, strategy)
    assert prep.info.n_sectors == len(prob.sectors)
    return prep, api.DeviceIntegral(prep), prob


def run_pass(dev, p, shifts, lams, codes):
    sh = torch.tensor(np.asarray(shifts, dtype=np.float64), device="cuda")
    lam = torch.tensor(np.asarray(lams, dtype=np.float64), device="cuda")
    c = torch.tensor(np.asarray(codes, dtype=np.int32), device="cuda")
    p.sector_precision = c.data_ptr()
    sums, fails = dev.outputs(p)
    dev.eval_sums(p, sh, lam, sums, fails)
    torch.cuda.synchronize()
    p.sector_precision = None
    s = sums.cpu().numpy()
    return s[..., 0] + 1j * s[..., 1], fails.cpu().numpy()


def kind1_phase(prep, prob, sums):
    """kind-1 sectors (F < 0) leave the factor exp(i pi eF(eps)) to the host"""
    out = sums.copy()
    eF0, eF1 = prob.e4[2], prob.e4[3]
    slots = sums.shape[2]
    ph = np.array([(-1) ** eF0 * (1j * math.pi * eF1) ** k / math.factorial(k) for k in range(slots)])
    for s in range(prep.info.n_sectors):
        if prep.sector(s).kind == 1:
            for n in range(slots):
                out[s, :, n] = sum(ph[q] * sums[s, :, n - q] for q in range(n + 1))
    return out


def test_probe_bins_count_the_islands_of_the_sample():
    prep, dev, prob = setup(W.double_box_planar(False), TABLE2, -4, 0, "geometric")
    ns, sl = prep.info.n_sectors, prep.info.n_slots
    n = 65521
    z = dict(api.builtin_lattices())[n]
    shifts = W.shifts(41, 2)
    lams = [0.0] * ns
    p = api.make_pass(n, z, len(shifts), 3, precision=N.QMC_PREC_MIXED)
    out = torch.zeros((ns, sl, 4), dtype=torch.float64, device="cuda")
    bins = torch.full((ns, R.BINS, 1 + 4 * sl), -1.0, dtype=torch.float64, device="cuda")
    sh = torch.tensor(np.asarray(shifts, dtype=np.float64), device="cuda")
    lam = torch.tensor(lams, dtype=torch.float64, device="cuda")
    n_sample = 4096
    assert N.lib().qmc_probe_islands(prep.packed, dev.dpacked.data_ptr(), ctypes.byref(p), sh.data_ptr(),
                                     lam.data_ptr(), n_sample, out.data_ptr(), bins.data_ptr(), None) == 0
    # a NULL bins buffer is refused
    assert N.lib().qmc_probe_islands(prep.packed, dev.dpacked.data_ptr(), ctypes.byref(p), sh.data_ptr(),
                                     lam.data_ptr(), n_sample, out.data_ptr(), None, None) == N.QMC_ERR_ARG
    torch.cuda.synchronize()
    pr, bn = out.cpu().numpy(), bins.cpu().numpy()
    stride = n // n_sample
    idx = np.arange(n_sample, dtype=np.uint64) * np.uint64(stride)
    frac_err = np.zeros((ns, R.BINS))
    for s, sec in enumerate(prob.sectors):
        mask = R.sing_mask(sec)
        k = R.shifted_indices(idx, n, z[: sec.dim], shifts[0][: sec.dim])
        want = np.bincount(R.bins(R.keys(k, mask, n)), minlength=R.BINS)
        assert np.array_equal(bn[s, :, 0], want.astype(np.float64)), (s, bn[s, :, 0], want)
        per = bn[s, :, 1:].reshape(R.BINS, sl, 4)  # sum |e|, sum e re, sum e im, sum |e|^2 per bin and slot
        assert np.allclose(per[:, :, 0].sum(axis=0), pr[s, :, 1], rtol=1e-12, atol=0.0)
        assert np.allclose(per[:, :, 1].sum(axis=0), pr[s, :, 2], rtol=1e-12, atol=1e-300)
        assert np.allclose(per[:, :, 2].sum(axis=0), pr[s, :, 3], rtol=1e-12, atol=1e-300)
        assert np.all(per[:, :, 3] >= per[:, :, 0] ** 2 / np.maximum(bn[s, :, 0:1], 1))  # Cauchy-Schwarz
        e = per[:, :, 0].sum(axis=1)
        frac_err[s] = np.cumsum(e) / max(e.sum(), 1e-300)
    heavy = [s for s, sec in enumerate(prob.sectors) if bin(R.sing_mask(sec)).count("1") == 4]
    print(f"{len(heavy)} four-pole sectors: median share of the FP32 error left outside the islands, levels "
          f"0..5: {np.round(np.median(frac_err[heavy][:, :R.LEVELS], axis=0), 3)}")


def error_per_sector(prep, prob, sums, lams, n, z, shifts):
    out = []
    for s, sec in enumerate(prob.sectors):
        o, l1, _, l1c = OI.lattice_sums(sec, prob.e4, n, z, shifts, lams[s], 3, prob.kmax, with_scale=True)
        k = o.shape[1]
        out.append(float((np.abs(sums[s, :, :k] - o) / np.maximum(l1c, 1e-300)).max()))
    return np.array(out)


CASES = [
    # name, topology, point, orders, strategy, lambda, n, shifts
    ("massless_box", W.box(False), dict(s=-3.0, t=-2.0, **LEGS0), (-2, 0), "iterated", 0.0, 4093, 3),
    ("massive_box", W.box(True), dict(s=5.0, t=-1.5, msq=1.0, **LEGS0), (0, 0), "iterated", 0.5, 4093, 3),
    ("table2", W.double_box_planar(False), TABLE2, (-4, 0), "geometric", 0.0, 251, 2),
]


@pytest.mark.parametrize("name,topo,pt,orders,strategy,lam,n,m", CASES, ids=[c[0] for c in CASES])
def test_island_passes_against_the_oracle(name, topo, pt, orders, strategy, lam, n, m):
    prep, dev, prob = setup(topo, pt, *orders, strategy)
    ns = prep.info.n_sectors
    z = OL.cbc_plain(n, 6)
    shifts = W.shifts(17, m)
    lams = [lam] * ns
    p = api.make_pass(n, z, m, 3, precision=N.QMC_PREC_MIXED, block=64, points_per_thread=4)
    masks = [R.sing_mask(sec) for sec in prob.sectors]
    res = {}
    for code in [1, 2, 4, 7, 0]:
        sums, fails = run_pass(dev, p, shifts, lams, [code] * ns)
        res[code] = (sums, fails)
    e = {c: error_per_sector(prep, prob, kind1_phase(prep, prob, res[c][0]), lams, n, z, shifts) for c in res}
    for c in (2, 4, 7):
        for s in range(ns):
            if masks[s] == 0:  # no singular variable: no islands, the FP32 pass bit for bit
                assert np.array_equal(res[c][0][s], res[1][0][s])
                assert np.array_equal(res[c][1][s], res[1][1][s])
    assert np.all(e[0] <= 1e-12)
    for c in (2, 4, 7):
        bound = MIXED_L1_BOUND if topo.loops == 1 else max(MIXED_L1_BOUND, 2.0 * float(e[1].max()))
        assert np.all(e[c] <= bound), (c, float(e[c].max()))
    print(f"{name}: worst |gpu-oracle|/term magnitudes: FP32 {e[1].max():.2e}, islands L=0 {e[2].max():.2e}, "
          f"L=2 {e[4].max():.2e}, L=5 {e[7].max():.2e}, FP64 {e[0].max():.2e}")
    heavy = [s for s in range(ns) if bin(masks[s]).count("1") >= 3]
    if heavy:
        # the islands take the cancellation-prone points: at level 0 (58-80 % of these sectors' points at n = 251)
        # the signed FP32 error of the sums falls by 1.5-7x per sector (the rest is rounding spread over every
        # point, measured here against the magnitude of the cancelling terms)
        assert e[2][heavy].sum() < 0.75 * e[1][heavy].sum()
        print(f"{name}: {len(heavy)} sectors with >= 3 singular variables: summed error FP32 "
              f"{e[1][heavy].sum():.2e}, islands L=0 {e[2][heavy].sum():.2e}, L=2 {e[4][heavy].sum():.2e}")


def test_island_pass_is_deterministic_across_launch_shapes():
    prep, dev, prob = setup(W.double_box_planar(False), TABLE2, -4, 0, "geometric")
    ns = prep.info.n_sectors
    n = 4093
    z = OL.cbc_plain(n, 6)
    shifts = W.shifts(3, 4)
    lams = [0.0] * ns
    codes = [(2 + s % 6) if s % 7 else (0 if s % 2 else 1) for s in range(ns)]
    a, fa = run_pass(dev, api.make_pass(n, z, 4, 3, precision=N.QMC_PREC_MIXED, block=128, points_per_thread=8),
                     shifts, lams, codes)
    b, fb = run_pass(dev, api.make_pass(n, z, 4, 3, precision=N.QMC_PREC_MIXED, block=128, points_per_thread=8,
                                        grid=7), shifts, lams, codes)
    c, _ = run_pass(dev, api.make_pass(n, z, 4, 3, precision=N.QMC_PREC_MIXED, block=128, points_per_thread=8),
                    shifts, lams, codes)
    assert np.array_equal(a, b) and np.array_equal(a, c) and np.array_equal(fa, fb)


def test_mixed_integration_with_islands_agrees_with_fp64():
    prep, dev, prob = setup(W.double_box_planar(False), TABLE2, -4, 0, "geometric")
    blob = T.compile_integral(W.double_box_planar(False), T.zero_invariants_of(W.double_box_planar(False), TABLE2),
                              strategy="geometric")
    ctx = api.Context()
    iid = ctx.load_sectors(blob)
    ctx.set_kinematics(iid, W.kinematics(W.double_box_planar(False), **TABLE2), -4, 0)
    out = {}
    for prec in (N.QMC_PREC_FP64, N.QMC_PREC_MIXED):
        r = ctx.integrate(iid, rel_tol=1e-4, n_shifts=16, seed=5, lam=0.0, precision=prec)
        assert r.status == 0
        val, err = api.result_arrays(r)
        out[prec] = (val, np.hypot(err[:, 0], err[:, 1]), r)
    ctx.close()
    (v64, e64, r64), (v32, e32, r32) = out[N.QMC_PREC_FP64], out[N.QMC_PREC_MIXED]
    print(f"Table 2 (-1,0,0,-1): FP64 {r64.seconds * 1e3:.0f} ms, mixed {r32.seconds * 1e3:.0f} ms with "
          f"{r32.fp64_reruns} FP64 sectors and {r32.island_sectors} sectors with FP64 islands of {prep.info.n_sectors}")
    assert r32.island_sectors > 0
    assert np.all(np.abs(v32 - v64) <= 5 * np.hypot(e32, e64) + 1e-12 * np.abs(v64))
