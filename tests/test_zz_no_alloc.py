"""qmc_eval_sums_noalloc: the allocation-free variant of qmc_eval_sums, for callers that cannot allocate device
memory (an application whose pool allocator holds all device memory, or a loop that forbids allocation after
start-up).  Its output must match qmc_eval_sums (caller-provided scratch) on identical inputs within the parity
tolerance of the other GPU tests, on two calls in a row with different inputs (the shared fixed scratch keeps the
previous call's contents).  Both entry points run the same kernels on the same work partition and reduce in the
same fixed order, so their sums must agree bit for bit.  Passes larger than its fixed scratch must be rejected
without writing the outputs.

This file is collected last on purpose: it only adds an entry point, so a failure here leaves the other tests'
results intact."""
import ctypes

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1508_02512_gb300 import _native as N  # noqa: E402
from paper_1508_02512_gb300 import api  # noqa: E402
from paper_1508_02512_gb300 import tables as T  # noqa: E402



@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cfg = W.CONFIG0
    blob = T.compile_integral(cfg.topology, T.zero_invariants_of(cfg.topology, cfg.point))
    prep = api.prepare(blob, cfg.kin, cfg.order_min, cfg.order_max)
    return prep, api.DeviceIntegral(prep)


def run_both(prep, dev, p, shifts):
    L = N.lib()
    sh = torch.tensor(shifts, device="cuda")
    lam = torch.zeros(prep.info.n_sectors, dtype=torch.float64, device="cuda")
    ref_sums, ref_fails = dev.outputs(p)
    dev.eval_sums(p, sh, lam, ref_sums, ref_fails)
    sums, fails = dev.outputs(p)
    sums.fill_(np.nan)
    st = torch.cuda.current_stream().cuda_stream
    rc = L.qmc_eval_sums_noalloc(prep.packed, dev.dpacked.data_ptr(), ctypes.byref(p), sh.data_ptr(),
                                 lam.data_ptr(), sums.data_ptr(), fails.data_ptr(), st)
    assert rc == 0, N.strerror(rc)
    torch.cuda.synchronize()
    return ref_sums.cpu().numpy(), ref_fails.cpu().numpy(), sums.cpu().numpy(), fails.cpu().numpy()


def test_noalloc_matches_eval_sums_on_two_calls(setup):
    prep, dev = setup
    for n, m, seed in ((4093, 8, 21), (8191, 5, 22)):
        z = dict(api.builtin_lattices())[n]
        p = api.make_pass(n, z, m, 3)
        ref, rf, got, gf = run_both(prep, dev, p, W.shifts(seed, m))
        assert np.array_equal(got, ref)
        assert np.array_equal(gf, rf)


def test_noalloc_rejects_passes_beyond_its_scratch(setup):
    prep, dev = setup
    n = 33554393  # largest prime below 2^25: 12 sectors x 64 shifts x 32768 chunks of partials >> 32 MiB
    p = api.make_pass(n, [1, 3, 5, 7, 9, 11], 64, 3)
    assert api.scratch_bytes(prep, p) > (32 << 20)
    sh = torch.zeros((64, 6), dtype=torch.float64, device="cuda")
    lam = torch.zeros(prep.info.n_sectors, dtype=torch.float64, device="cuda")
    sums = torch.full((prep.info.n_sectors, 64, prep.info.n_slots, 2), 1234.5, dtype=torch.float64, device="cuda")
    fails = torch.full((prep.info.n_sectors, 64), -7, dtype=torch.int64, device="cuda")
    rc = N.lib().qmc_eval_sums_noalloc(prep.packed, dev.dpacked.data_ptr(), ctypes.byref(p), sh.data_ptr(),
                                       lam.data_ptr(), sums.data_ptr(), fails.data_ptr(), None)
    assert rc == N.QMC_ERR_MEMORY
    torch.cuda.synchronize()
    assert bool((sums == 1234.5).all()) and bool((fails == -7).all())  # the rejected call wrote nothing
