"""Batching and serving: qmc_eval_batch runs many passes in shared persistent launches with results identical to
running each alone; the serving loop (qmc_submit/qmc_poll/qmc_cancel) admits requests of uneven sector count and
dimension, overlaps their passes on the device, and returns for every request exactly the result it gives alone
(and that qmc_integrate gives with the same options)."""
import ctypes
import time

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


def point(cfg, **kw):
    return W.kinematics(cfg.topology, **{**cfg.point, **kw})


def test_batch_equals_alone_and_abort_flags_stop_their_passes():
    lat = dict(api.builtin_lattices())
    specs = [(W.CONFIG0, point(W.CONFIG0), -2, 0, 4093, 0.0, N.QMC_PREC_FP64),
             (W.CONFIG1, point(W.CONFIG1), 0, 0, 8191, 0.5, N.QMC_PREC_FP64),
             (W.CONFIG1, point(W.CONFIG1, s=7.0, t=-2.5), 0, 0, 2039, 0.5, N.QMC_PREC_FP64),
             (W.CONFIG0, point(W.CONFIG0, s=-5.0), -2, 0, 1021, 0.0, N.QMC_PREC_MIXED),
             (W.CONFIG2, point(W.CONFIG2), -2, 0, 1021, 0.25, N.QMC_PREC_FP64)]
    preps, devs, passes, ins, outs = [], [], [], [], []
    for k, (cfg, kin, omin, omax, n, lam, prec) in enumerate(specs):
        prep = api.prepare(table(cfg), kin, omin, omax)
        dev = api.DeviceIntegral(prep)
        p = api.make_pass(n, lat[n], 6, 3, precision=prec)
        sh = torch.tensor(W.shifts(40 + k, 6), device="cuda")
        lm = torch.full((prep.info.n_sectors,), lam, dtype=torch.float64, device="cuda")
        preps.append(prep)
        devs.append(dev)
        passes.append(p)
        ins.append((sh, lm))
        outs.append(dev.outputs(p))
    alone = []
    for prep, dev, p, (sh, lm), (sums, fails) in zip(preps, devs, passes, ins, outs):
        dev.eval_sums(p, sh, lm, sums, fails)
        torch.cuda.synchronize()
        alone.append((sums.clone(), fails.clone()))
        sums.zero_()
        fails.zero_()
    items = (N.qmc_batch_item * len(specs))()
    keep = []
    for i, (prep, dev, p, (sh, lm), (sums, fails)) in enumerate(zip(preps, devs, passes, ins, outs)):
        buf = ctypes.create_string_buffer(prep.packed)
        keep.append(buf)
        items[i].packed_host = ctypes.addressof(buf)
        items[i].packed_dev = dev.dpacked.data_ptr()
        items[i].pass_ = p
        items[i].shifts_dev = sh.data_ptr()
        items[i].lambda_dev = lm.data_ptr()
        items[i].sums_dev = sums.data_ptr()
        items[i].fails_dev = fails.data_ptr()
    need = N.lib().qmc_batch_scratch_bytes(items, len(specs))
    assert need > 0
    scratch = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    base = scratch.data_ptr() + ((-scratch.data_ptr()) % 256)
    rc = N.lib().qmc_eval_batch(items, len(specs), base, need, torch.cuda.current_stream().cuda_stream)
    assert rc == 0, N.strerror(rc)
    torch.cuda.synchronize()
    for (s_a, f_a), (sums, fails) in zip(alone, outs):
        assert torch.equal(s_a, sums) and torch.equal(f_a, fails)
    # the same batch with an FP64 and a mixed pass stopped before they start (qmc_batch_item.abort_flag, here in
    # device memory): every item of theirs is skipped, so their sums are zero; the other passes are unchanged
    stop = torch.ones(1, dtype=torch.int32, device="cuda")
    for i in (1, 3):
        items[i].abort_flag = stop.data_ptr()
    for sums, fails in outs:
        sums.fill_(7.0)
        fails.fill_(7)
    rc = N.lib().qmc_eval_batch(items, len(specs), base, need, torch.cuda.current_stream().cuda_stream)
    assert rc == 0, N.strerror(rc)
    torch.cuda.synchronize()
    for i, ((s_a, f_a), (sums, fails)) in enumerate(zip(alone, outs)):
        if i in (1, 3):
            assert int(torch.count_nonzero(sums)) == 0 and int(torch.count_nonzero(fails)) == 0
        else:
            assert torch.equal(s_a, sums) and torch.equal(f_a, fails)


def req_opts(prec, seed):
    return dict(rel_tol=1e-4, n_shifts=8, seed=seed, lam=0.5, precision=prec)


def same(r1, r2):
    v1, e1 = api.result_arrays(r1)
    v2, e2 = api.result_arrays(r2)
    return (r1.status == r2.status and r1.n_final == r2.n_final and r1.passes == r2.passes and np.array_equal(v1, v2)
            and np.array_equal(e1, e2))


@pytest.mark.parametrize("prec", [N.QMC_PREC_FP64, N.QMC_PREC_MIXED], ids=["fp64", "mixed"])
def test_serving_result_same_alone_and_in_the_mix(prec):
    ctx = api.Context(0, 2 << 30)
    ids = {c.name: ctx.load_sectors(table(c)) for c in (W.CONFIG0, W.CONFIG1, W.CONFIG2)}
    target = (W.CONFIG1, point(W.CONFIG1, s=6.5, t=-1.0), 0, 0)
    # alone
    rid = ctx.submit(ids[target[0].name], target[1], target[2], target[3], **req_opts(prec, 7))
    alone = ctx.wait(rid)
    assert alone.status == 0
    # the same request in a mix of uneven sector counts and dimensions, arriving while others run
    others = [(W.CONFIG2, point(W.CONFIG2, s=7.0), -2, 0, dict(rel_tol=2e-2, n_shifts=8, seed=1, lam=0.5)),
              (W.CONFIG0, point(W.CONFIG0, s=6.0, t=-1.2), -2, 0, req_opts(prec, 2)),
              (W.CONFIG1, point(W.CONFIG1), 0, 0, req_opts(prec, 3)),
              (W.CONFIG0, point(W.CONFIG0), -2, 0, req_opts(prec, 4))]
    mix_ids = [ctx.submit(ids[c.name], kin, a, b, **o) for c, kin, a, b, o in others[:2]]
    time.sleep(0.01)
    rid2 = ctx.submit(ids[target[0].name], target[1], target[2], target[3], **req_opts(prec, 7))
    mix_ids += [ctx.submit(ids[c.name], kin, a, b, **o) for c, kin, a, b, o in others[2:]]
    in_mix = ctx.wait(rid2)
    rest = [ctx.wait(i) for i in mix_ids]
    assert same(alone, in_mix), (api.result_arrays(alone), api.result_arrays(in_mix))
    assert all(r.status == 0 for r in rest), [r.status for r in rest]
    st = ctx.serving_stats()
    assert st.completed == 6 and st.peak_active >= 2 and st.batched_passes > st.rounds
    # and the same as qmc_integrate with these options
    ctx2 = api.Context(0, 1 << 30)
    i2 = ctx2.load_sectors(table(target[0]))
    ctx2.set_kinematics(i2, target[1], target[2], target[3])
    direct = ctx2.integrate(i2, **req_opts(prec, 7))
    assert same(alone, direct)
    ctx2.close()
    ctx.close()


def test_serving_cancel():
    ctx = api.Context(0, 1 << 30)
    iid = ctx.load_sectors(table(W.CONFIG3))
    long_id = ctx.submit(iid, point(W.CONFIG3), -2, 0, rel_tol=1e-7, n_shifts=8, seed=5, lam=0.5, max_n=1 << 20)
    ctx.cancel(long_id)
    r = ctx.wait(long_id, timeout=120)
    assert r.status == N.QMC_ERR_CANCELLED, (r.status, r.n_final)
    ctx.close()


def test_serving_deadline_passed_in_queue_finishes_without_work():
    """max_seconds counts from submission: a request whose limit has passed by the time the loop would admit
    it leaves with QMC_ERR_TIMEOUT and no evaluations; a request with room to run is unaffected."""
    ctx = api.Context(0, 1 << 30)
    iid = ctx.load_sectors(table(W.CONFIG1))
    late = ctx.submit(iid, point(W.CONFIG1), 0, 0, rel_tol=1e-3, n_shifts=8, seed=3, max_seconds=1e-9)
    ok = ctx.submit(iid, point(W.CONFIG1), 0, 0, rel_tol=1e-3, n_shifts=8, seed=3, max_seconds=60.0)
    r = ctx.wait(late, timeout=60)
    assert r.status == N.QMC_ERR_TIMEOUT and r.evals == 0, (r.status, r.evals)
    assert ctx.wait(ok, timeout=60).status == 0
    ctx.close()


def test_serving_admission_by_memory():
    """A budget that holds only a few requests at a time: the rest wait in the queue, all complete, and the
    context never holds more device memory than its budget."""
    budget = 24 << 20
    ctx = api.Context(0, budget)
    i1 = ctx.load_sectors(table(W.CONFIG1))
    i0 = ctx.load_sectors(table(W.CONFIG0))
    ids = []
    for k in range(8):
        if k % 2:
            ids.append(ctx.submit(i1, point(W.CONFIG1, s=5.0 + 0.5 * k), 0, 0, rel_tol=1e-5, n_shifts=8, seed=k))
        else:
            ids.append(ctx.submit(i0, point(W.CONFIG0, s=-2.0 - k), -2, 0, rel_tol=1e-6, n_shifts=8, seed=k))
    peak_bytes, saw_queue = 0, False
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < 120:
        st = ctx.serving_stats()
        peak_bytes = max(peak_bytes, st.device_bytes)
        saw_queue |= st.queued > 0 and st.active > 0
        if st.completed == len(ids):
            break
        time.sleep(0.001)
    for i in ids:
        assert ctx.wait(i, timeout=60).status == 0
    st = ctx.serving_stats()
    # the budget admits only a few requests at once (each reserves room for its first pass), so some waited
    assert peak_bytes <= budget and 1 <= st.peak_active < len(ids)
    ctx.close()


def test_overload_sheds_requests_that_cannot_meet_their_deadline():
    """A burst of two-loop requests far above the loop's capacity, each with a time limit of a few single-request
    times: once the loop has the cost (charged loop seconds) of completed requests for that integral, it turns
    away, before they run, the requests whose limit the work ahead of them would pass (status QMC_ERR_TIMEOUT with
    no evaluation, counted in qmc_serving_stats.shed), while the admitted ones still converge."""
    cfg = W.CONFIG2
    ctx = api.Context(0, 8 << 30)
    iid = ctx.load_sectors(table(cfg))
    kw = dict(rel_tol=1e-3, n_shifts=16, lam=0.5, precision=N.QMC_PREC_MIXED)
    first = ctx.wait(ctx.submit(iid, point(cfg), -2, 0, seed=1, **kw))  # compiles, and gives the work history
    assert first.status == 0
    again = ctx.wait(ctx.submit(iid, point(cfg), -2, 0, seed=2, **kw))
    assert again.status == 0
    limit = max(6.0 * again.seconds, 1.0)
    rids = [ctx.submit(iid, point(cfg, s=6.0 + 0.05 * k), -2, 0, seed=100 + k, max_seconds=limit, **kw)
            for k in range(40)]
    res = [ctx.wait(r, timeout=600.0) for r in rids]
    st = ctx.serving_stats()
    ctx.close()
    shed = [r for r in res if r.status == N.QMC_ERR_TIMEOUT and r.evals == 0]
    ok = [r for r in res if r.status == 0]
    print(f"limit {limit:.2f} s: {len(ok)} converged, {st.shed} shed, {len(shed)} left without running, "
          f"{len(res) - len(ok) - len(shed)} ran out of time; shed after "
          f"{max((r.seconds for r in shed), default=0):.2f} s at most")
    assert st.shed > 0 and len(shed) >= st.shed
    assert len(ok) > 0
    # turned away early, not when their limit passed
    assert min(r.seconds for r in shed) < limit


def test_cancel_and_time_limit_stop_a_running_round():
    """A request with long rounds (the massive box in FP64 from a lattice of 33554393 points, 16 shifts: ~0.8 s for
    its one round) stops within that round when it is cancelled or its time limit passes: the kernels read its
    abort flag (mapped pinned host memory) at every work item and skip the rest.  Without the flag it would end
    only at the round boundary, a whole round later."""
    cfg = W.CONFIG1
    ctx = api.Context(0, 8 << 30)
    iid = ctx.load_sectors(table(cfg))
    fp64 = dict(n_shifts=16, lam=0.5, precision=N.QMC_PREC_FP64)
    # compiles the family's generated FP64 evaluator, which an admitted request would otherwise wait for
    assert ctx.wait(ctx.submit(iid, point(cfg), 0, 0, seed=1, rel_tol=1e-3, **fp64)).status == 0
    big = dict(rel_tol=1e-12, ladder_start=15, max_n=33554393, **fp64)
    full = ctx.wait(ctx.submit(iid, point(cfg), 0, 0, seed=2, **big))
    assert full.status in (0, N.QMC_ERR_NOT_CONVERGED) and full.seconds > 0.4  # one long round, whatever its end
    rid = ctx.submit(iid, point(cfg), 0, 0, seed=3, **big)
    time.sleep(0.1)
    ctx.cancel(rid)
    cancelled = ctx.wait(rid)
    # the same table under a new id has no cost history, so the loop admits it (for this id it would be shed)
    fresh = ctx.load_sectors(table(cfg))
    limited = ctx.wait(ctx.submit(fresh, point(cfg), 0, 0, seed=4, max_seconds=0.15, **big))
    st = ctx.serving_stats()
    ctx.close()
    print(f"one round {full.seconds:.3f} s; cancelled after 0.1 s: done at {cancelled.seconds:.3f} s; "
          f"time limit 0.15 s: done at {limited.seconds:.3f} s; {st.rounds} rounds")
    assert cancelled.status == N.QMC_ERR_CANCELLED and cancelled.seconds < 0.5 * full.seconds
    assert limited.status == N.QMC_ERR_TIMEOUT and 0.14 < limited.seconds < 0.5 * full.seconds
    assert limited.evals > 0  # it ran (stopped by the watchdog within its round, not shed before it)


def test_time_limit_stops_a_running_pass_of_qmc_integrate():
    """The blocking qmc_integrate with a time limit inside one long pass (the massive box in FP64 on 33554393
    points, 16 shifts: ~0.8 s): a timer sets the context's abort flag at the limit, the kernels skip the rest of
    the pass, and the call returns QMC_ERR_TIMEOUT well before the pass would have ended."""
    cfg = W.CONFIG1
    ctx = api.Context()
    iid = ctx.load_sectors(table(cfg))
    ctx.set_kinematics(iid, point(cfg), 0, 0)
    fp64 = dict(n_shifts=16, lam=0.5, precision=N.QMC_PREC_FP64)
    assert ctx.integrate(iid, rel_tol=1e-3, **fp64).status == 0  # compiles the generated evaluator
    big = dict(rel_tol=1e-12, ladder_start=15, max_n=33554393, **fp64)
    full = ctx.integrate(iid, seed=2, **big)
    t0 = time.perf_counter()
    limited = ctx.integrate(iid, seed=3, max_seconds=0.15, **big)
    wall = time.perf_counter() - t0
    again = ctx.integrate(iid, seed=2, **big)  # the flag is cleared for the next call
    ctx.close()
    print(f"one pass {full.seconds:.3f} s; time limit 0.15 s: returned after {wall:.3f} s")
    assert full.seconds > 0.4 and full.status in (0, N.QMC_ERR_NOT_CONVERGED)
    assert limited.status == N.QMC_ERR_TIMEOUT and wall < 0.5 * full.seconds
    assert again.status == full.status and np.array_equal(api.result_arrays(again)[0], api.result_arrays(full)[0])
