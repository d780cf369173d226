"""CUDA-graph capture of a pass: qmc_eval_sums only enqueues stream-ordered work (a memset and kernel launches),
so a pass captured into a CUDA graph replays with results identical to a direct call, and reads its inputs
(shifts, lambda) from device memory at replay time.  Generated evaluators must be compiled before capture."""
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


@pytest.mark.parametrize("precision", [N.QMC_PREC_FP64, N.QMC_PREC_MIXED], ids=["fp64", "mixed"])
def test_captured_pass_replays_identically(precision):
    cfg = W.CONFIG1
    blob = T.compile_integral(cfg.topology, T.zero_invariants_of(cfg.topology, cfg.point))
    prep = api.prepare(blob, cfg.kin, 0, 0)
    dev = api.DeviceIntegral(prep)
    api.gen_compile(prep)
    n = 65521
    p = api.make_pass(n, dict(api.builtin_lattices())[n], 8, 3, precision=precision, block=128,
                      points_per_thread=16)
    side = torch.cuda.Stream()
    sh = torch.tensor(W.shifts(9, 8), device="cuda")
    lam = torch.full((prep.info.n_sectors,), 0.5, dtype=torch.float64, device="cuda")
    ref, fref = dev.outputs(p)
    out, fout = dev.outputs(p)
    with torch.cuda.stream(side):
        dev.eval_sums(p, sh, lam, ref, fref)  # direct call; also sizes the scratch before capture
    side.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side, capture_error_mode="relaxed"):
        dev.eval_sums(p, sh, lam, out, fout)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref) and torch.equal(fout, fref)
    # new lambda in place: the replay reads it, and equals a direct pass with that lambda (the replay and the
    # direct pass share the scratch buffer, so they run one after the other)
    lam.fill_(0.25)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    got = out.clone()
    with torch.cuda.stream(side):
        dev.eval_sums(p, sh, lam, ref, fref)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    assert not np.allclose(got.cpu().numpy(), 0.0)
