"""Per-sector lattice sizes: passes restricted to a subset of sectors (sector_active) write exactly those sectors'
sums, bit-identical to a full pass; qmc_integrate (by default) moves only the sectors that carry the
remaining error up the ladder, agrees with the closed form / the lock-step ladder within the errors, and the
serving loop returns the same result as qmc_integrate."""
import cmath
import ctypes
import math

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1508_02512_gb300 import _native as N  # noqa: E402
from paper_1508_02512_gb300 import api  # noqa: E402
from paper_1508_02512_gb300 import tables as T  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def table(cfg):
    return T.compile_integral(cfg.topology, T.zero_invariants_of(cfg.topology, cfg.point))


@pytest.mark.parametrize("precision", [N.QMC_PREC_FP64, N.QMC_PREC_MIXED], ids=["fp64", "mixed"])
def test_subset_pass_writes_only_its_sectors(precision):
    cfg = W.CONFIG0
    prep = api.prepare(table(cfg), cfg.kin, cfg.order_min, cfg.order_max)
    dev = api.DeviceIntegral(prep)
    n = 4093
    z = dict(api.builtin_lattices())[n]
    sh = torch.tensor(W.shifts(8, 4), device="cuda")
    lam = torch.zeros(prep.info.n_sectors, dtype=torch.float64, device="cuda")
    full = api.make_pass(n, z, 4, 3, precision=precision)
    ref, fref = dev.outputs(full)
    dev.eval_sums(full, sh, lam, ref, fref)
    mask = np.zeros(prep.info.n_sectors, dtype=np.int32)
    mask[[0, 3, 4, 5, 9, 11]] = 1
    sub = api.make_pass(n, z, 4, 3, precision=precision)
    sub.sector_active = mask.ctypes.data_as(ctypes.c_void_p)
    out, fout = dev.outputs(sub)
    out.fill_(7.0)
    fout.fill_(-1)
    dev.eval_sums(sub, sh, lam, out, fout)
    torch.cuda.synchronize()
    on = torch.tensor(mask.astype(bool), device="cuda")
    assert torch.equal(out[on], ref[on]) and torch.equal(fout[on], fref[on])
    assert bool((out[~on] == 7.0).all()) and bool((fout[~on] == -1).all())


def massless_box_reference():
    from scipy import special as sp

    def f(e):
        cg = sp.gamma(1 + e) * sp.gamma(1 - e) ** 2 / sp.gamma(1 - 2 * e)
        return cg / 6.0 * (2 / e ** 2 * (3.0 ** (-e) + 2.0 ** (-e)) - cmath.log(1.5) ** 2 - math.pi ** 2) * e ** 2

    th = 2 * np.pi * np.arange(64) / 64
    eps = 0.25 * np.exp(1j * th)
    vals = np.array([f(e) for e in eps])
    return np.array([np.mean(vals * eps ** (-k)) for k in range(3)])


@pytest.mark.parametrize("precision", [N.QMC_PREC_FP64, N.QMC_PREC_MIXED], ids=["fp64", "mixed"])
def test_adaptive_massless_box_to_closed_form(precision):
    cfg = W.CONFIG0
    ctx = api.Context()
    iid = ctx.load_sectors(table(cfg))
    ctx.set_kinematics(iid, cfg.kin, -2, 0)
    ref = massless_box_reference()
    res = {}
    tol = 1e-8 if precision == N.QMC_PREC_FP64 else 2e-6
    for adaptive in (0, 1):
        r = ctx.integrate(iid, rel_tol=tol, n_shifts=8, seed=5, precision=precision, lock_step=1 - adaptive)
        assert r.status == 0
        val, err = api.result_arrays(r)
        e = np.hypot(err[:, 0], err[:, 1])
        print(f"{'adaptive' if adaptive else 'lock-step'}: evals {r.evals} passes {r.passes} n_final {r.n_final}",
              val, e)
        assert np.all(np.abs(val - ref) <= 5 * e + (1e-9 if precision == N.QMC_PREC_FP64 else 2e-6) * np.abs(ref))
        res[adaptive] = r
    assert res[1].evals <= res[0].evals
    ctx.close()


def test_adaptive_two_loop_agrees_with_lock_step_and_evaluates_less():
    cfg = W.CONFIG2
    ctx = api.Context(0, 4 << 30)
    iid = ctx.load_sectors(table(cfg))
    ctx.set_kinematics(iid, cfg.kin, cfg.order_min, cfg.order_max)
    out = {}
    for adaptive in (0, 1):
        r = ctx.integrate(iid, rel_tol=1e-3, n_shifts=16, seed=9, lam=0.5, precision=N.QMC_PREC_MIXED,
                          lock_step=1 - adaptive, max_seconds=300)
        assert r.status == 0
        out[adaptive] = r
        print(f"planar {'adaptive' if adaptive else 'lock-step'}: {r.seconds:.3f} s, evals {r.evals:.3e}, "
              f"passes {r.passes}, n_final {r.n_final}")
    v0, e0 = api.result_arrays(out[0])
    v1, e1 = api.result_arrays(out[1])
    s = np.hypot(np.hypot(e0[:, 0], e0[:, 1]), np.hypot(e1[:, 0], e1[:, 1]))
    assert np.all(np.abs(v0 - v1) <= 5 * s)
    assert out[1].evals < out[0].evals
    ctx.close()


def test_serving_adaptive_equals_integrate():
    cfg = W.CONFIG1
    ctx = api.Context()
    iid = ctx.load_sectors(table(cfg))
    kw = dict(rel_tol=1e-5, n_shifts=16, seed=21, lam=0.5, precision=N.QMC_PREC_MIXED)
    rid = ctx.submit(iid, cfg.kin, 0, 0, **kw)
    rs = ctx.wait(rid)
    ctx.set_kinematics(iid, cfg.kin, 0, 0)
    ri = ctx.integrate(iid, **kw)
    assert rs.status == 0 and ri.status == 0
    vs, es = api.result_arrays(rs)
    vi, ei = api.result_arrays(ri)
    assert np.array_equal(vs, vi) and np.array_equal(es, ei) and rs.evals == ri.evals
    ctx.close()
