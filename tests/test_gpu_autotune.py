"""Launch-shape autotuner: it times every candidate (block x points per thread), records the fastest per family,
precision, evaluator and lattice-size bucket, and default-shape passes then use it (scratch size and results)."""
import ctypes

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
    yield
    N.lib().qmc_autotune_clear()


@pytest.mark.parametrize("precision", [N.QMC_PREC_FP64, N.QMC_PREC_MIXED], ids=["fp64", "mixed"])
def test_autotune_records_the_fastest_shape_and_default_passes_use_it(precision):
    cfg = W.CONFIG1
    blob = T.compile_integral(cfg.topology, T.zero_invariants_of(cfg.topology, cfg.point))
    prep = api.prepare(blob, cfg.kin, 0, 0)
    dev = api.DeviceIntegral(prep)
    n, z = 262139, dict(api.builtin_lattices())[262139]
    sh = torch.tensor(W.shifts(3, 8), device="cuda")
    lam = torch.full((prep.info.n_sectors,), 0.5, dtype=torch.float64, device="cuda")
    N.lib().qmc_autotune_clear()
    default = api.make_pass(n, z, 8, 3, precision=precision)
    untuned_scratch = api.scratch_bytes(prep, default)
    r = dev.autotune(default, sh, lam)
    assert r.n_candidates == 12
    ms = [r.candidate_ms[k] for k in range(r.n_candidates)]
    shapes = [(r.candidate_block[k], r.candidate_points_per_thread[k]) for k in range(r.n_candidates)]
    print("autotune", "fp64" if precision == 0 else "mixed", dict(zip(shapes, np.round(ms, 3))), "->",
          (r.block, r.points_per_thread))
    assert all(m > 0 for m in ms) and r.ms == min(ms)
    assert (r.block, r.points_per_thread) == shapes[int(np.argmin(ms))]
    explicit = api.make_pass(n, z, 8, 3, precision=precision, block=r.block, points_per_thread=r.points_per_thread)
    assert api.scratch_bytes(prep, default) == api.scratch_bytes(prep, explicit)
    s1, f1 = dev.outputs(default)
    s2, f2 = dev.outputs(explicit)
    dev.eval_sums(default, sh, lam, s1, f1)
    dev.eval_sums(explicit, sh, lam, s2, f2)
    torch.cuda.synchronize()
    assert torch.equal(s1, s2)
    # another lattice-size bucket is not affected; clearing restores the built-in default
    other = api.make_pass(65521, dict(api.builtin_lattices())[65521], 8, 3, precision=precision)
    d_other = api.make_pass(65521, dict(api.builtin_lattices())[65521], 8, 3, precision=precision,
                            block=128, points_per_thread=16 if precision else 8)
    assert api.scratch_bytes(prep, other) == api.scratch_bytes(prep, d_other)
    N.lib().qmc_autotune_clear()
    assert api.scratch_bytes(prep, default) == untuned_scratch
