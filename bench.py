#!/usr/bin/env python
"""Benchmark of the QMC sector-integration hot path on GB300: integrand evaluations per second.

A step is one pass of the whole hot path over the massive one-loop box in the physical region (4 sectors,
contour deformation lambda = 0.5, s = 5, t = -1.5, m = 1, massless legs): every sector x 16 random shifts x
every point of the rank-1 lattice of size n = 16777213 (largest prime below 2^24), Korobov transform r = 3,
FP64 -- 1.07e9 integrand evaluations, reduced per (sector, shift) -- through qmc_eval_partials +
qmc_reduce_partials (the two launches of qmc_eval_sums).

Output: one JSON line (rank 0).  `value` = evaluations/s of the whole job with the table, shifts and lambda
already resident on the device; `e2e` = the same metric through qmc_eval_sums_host (host buffers, copies inside
the timed region); `roofline` = algorithmic FP64 throughput of the evaluation kernel against the FP64 peak
derived from the SM count, FP64 units and clock; `cpu_baseline` = the oracle (plain C, all host cores) on a
bounded sample of the same workload; `time_to_1e-3` = qmc_integrate to 1e-3 relative error over 32 seeds;
`paper_ia_scan` and `paper_table2` = the paper's own workloads (its one-loop s-scan of 1000 points through the
serving loop, and the three points of its Table 2) with its printed timings beside them.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --integral planar_dbox|nonplanar_dbox|massless_dbox_table2 [--log2n 18]   the same
        measurement on a two-loop double box (46/48/143 six-dimensional sectors, eps^-2 or eps^-4 ..eps^0,
        lambda adapted per sector beforehand)
    python bench.py --serving N   the serving workload: N Poisson arrivals of random integrals
    python bench.py --paper-ia-scan N | --paper-table2   only those workloads
Multi-GPU (torchrun, one rank per GPU): every rank integrates its own replica with its own shifts (weak
scaling, no data-path collective); the barrier and max-over-ranks timing use torch.distributed.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

LOG2_N = 24
N_PREC_FP64 = 0
N_PREC_MIXED = 1
N_SHIFTS = 16
LAMBDA = 0.5
METRIC = "integrand evals/s"
# FP64 peak of a GB300: 152 SMs x 2 FP64 FMA per clock per SM (4 flop) x 2070 MHz maximum SM clock
FP64_PEAK_TFLOPS = 152 * 4 * 2070e6 / 1e12
# FP32 peak: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2070 MHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2070e6 / 1e12
# DRAM bytes per launch of the FP64 evaluation kernel (qd_eval_c1) of the bench step, from one single-pass ncu
# capture of that launch (profiles/qmc_eval_kernel_massive_box.md); valid while the device code and the
# generator hash to KERNEL_HASH, null otherwise
TRAFFIC_BYTES = 771584 + 0  # dram__bytes_read.sum + dram__bytes_write.sum of one full-size launch
KERNEL_HASH = "c71d0d47b057653d"


INTEGRALS = {"massive_box": W.CONFIG1, "planar_dbox": W.CONFIG2, "nonplanar_dbox": W.CONFIG3,
             "massless_dbox_table2": W.PAPER_IB}


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in ("qmc_dev.cuh", "qmc_jit.cpp"):
        with open(os.path.join(ROOT, "paper_1508_02512_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-extras", action="store_true", help="skip time-to-accuracy and CPU baseline")
    ap.add_argument("--integral", choices=sorted(INTEGRALS), default="massive_box",
                    help="integral of the timed pass (default: the massive one-loop box)")
    ap.add_argument("--evaluator", choices=["auto", "table", "generated"], default="auto",
                    help="polynomial evaluator of the FP64 pass (the mixed pass always uses the generated one)")
    ap.add_argument("--log2n", type=int, default=0, help="lattice size: largest prime below 2^log2n (default "
                                                         "24 one-loop, 18 two-loop)")
    ap.add_argument("--profile-pass", action="store_true",
                    help="run two passes of the same integral at n = 1048573 and exit (small case for ncu)")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64", help="precision of --profile-pass")
    ap.add_argument("--serving", type=int, default=0,
                    help="run only the serving workload with this many requests and print its JSON line")
    ap.add_argument("--paper-ia-scan", type=int, default=0,
                    help="run only the paper's one-loop s-scan I_A with this many points through the serving loop "
                         "and print its JSON line")
    ap.add_argument("--paper-table2", action="store_true",
                    help="run only the paper's Table 2 points (massless double box, Euclidean) to 1e-4 and print "
                         "their JSON line")
    ap.add_argument("--serving-baseline", action="store_true",
                    help="with --serving: also run the requests one at a time through the plain FP64 path")
    return ap.parse_args()


def workload_config(cfg, n, ns, lam_desc):
    if cfg is W.CONFIG1:
        what = f"massive one-loop box, physical s=5 t=-1.5 m^2=1, lambda={lam_desc}, {ns} sectors"
    elif cfg is W.PAPER_IB:
        what = (f"massless planar double box (the paper's Table 2, legs p1^2 = p4^2 = -1), Euclidean s=t=u=-2/3, "
                f"eps^-4..eps^0, geometric decomposition, {ns} six-dimensional sectors")
    else:
        what = (f"{'planar' if cfg is W.CONFIG2 else 'non-planar'} two-loop double box, physical s=6 t=-2, "
                f"m^2=1 on four lines, eps^-2..eps^0, lambda={lam_desc}, {ns} six-dimensional sectors")
    return {"workload": f"{what} x {N_SHIFTS} shifts x n={n} rank-1 lattice, Korobov r=3",
            "integral": cfg.name, "sectors": ns, "shifts": N_SHIFTS, "lattice_n": n,
            "l2": "inputs (the sector table, shifts) live in shared memory; a 256 MiB buffer is written between "
                  "steps to flush L2"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return world, rank, local, dist


def max_over_ranks(value, dist, device="cpu"):
    """The largest of the ranks' values (timing of the slowest replica); the value itself on one rank."""
    if not dist:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def korobov_vector(n, a=76):
    """An admissible generating vector (1, a, a^2, ...) mod n for timing the oracle: the cost of an evaluation
    does not depend on which vector the lattice uses."""
    return [pow(a, j, n) for j in range(6)]


def cpu_baseline(cfg=None, n_log2=0):
    """The oracle as it stands (plain C, OpenMP over all host cores) on a bounded sample of the workload:
    n = largest prime below 2^18 for the one-loop box, 2^12 for a double box (about 10-20 s of CPU work)."""
    from oracle import integrate as OI
    from oracle import lattice as OL
    cfg = cfg or W.CONFIG1
    n_log2 = n_log2 or (18 if cfg.topology.loops == 1 else 12)
    prob = OI.make_problem(cfg.topology, {**cfg.point}, cfg.order_min, cfg.order_max, cfg.strategy)
    n = OL.prime_below(1 << n_log2)
    z = korobov_vector(n)
    shifts = W.shifts(12345, N_SHIFTS)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    OI.integrate(prob, n, z, shifts, LAMBDA, 3, nthreads=cores)
    dt = time.perf_counter() - t0
    evals = len(prob.sectors) * N_SHIFTS * n
    return {"value": evals / dt, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"{cfg.name}, n={n} (largest prime < 2^{n_log2}), {N_SHIFTS} shifts, {len(prob.sectors)} "
                      f"sectors = {evals} evals in {dt:.2f} s"}


def main_reference(args):
    world, rank, local, dist = dist_setup(args)
    if rank != 0:  # the oracle runs once, on rank 0; the other ranks leave without work
        if dist:
            dist.destroy_process_group()
        return
    from oracle import integrate as OI
    from oracle import lattice as OL
    cfg = W.CONFIG1
    prob = OI.make_problem(cfg.topology, {**cfg.point}, 0, 0)
    n = OL.prime_below(1 << 16)
    z = korobov_vector(n)
    shifts = W.shifts(12345, N_SHIFTS)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        OI.integrate(prob, n, z, shifts, LAMBDA, 3, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        OI.integrate(prob, n, z, shifts, LAMBDA, 3, nthreads=cores)
    dt = time.perf_counter() - t0
    evals = len(prob.sectors) * N_SHIFTS * n
    v = evals * args.steps / dt
    sample = f"each step: massive box, n={n} (largest prime < 2^16), {N_SHIFTS} shifts, 4 sectors = {evals} evals"
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "evals/s", "n_gpus": args.gpus,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": workload_config(W.CONFIG1, n, len(prob.sectors), f"{LAMBDA}"),
                      "cpu_baseline": {"value": v, "unit": "evals/s", "cores": cores, "kind": "oracle",
                                       "sample": sample},
                      "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
    if dist:
        dist.destroy_process_group()


def main_ours(args):
    import torch

    from paper_1508_02512_gb300 import _native as N
    from paper_1508_02512_gb300 import api
    from paper_1508_02512_gb300 import tables as T

    world, rank, local, dist = dist_setup(args)
    torch.cuda.set_device(local)
    dev_name = f"cuda:{local}"
    cfg = INTEGRALS[args.integral]
    blob = T.compile_integral(cfg.topology, T.zero_invariants_of(cfg.topology, cfg.point), strategy=cfg.strategy)
    prep = api.prepare(blob, cfg.kin, cfg.order_min, cfg.order_max)
    di = api.DeviceIntegral(prep, dev_name)
    lat = dict(api.builtin_lattices())
    log2n = args.log2n or (LOG2_N if cfg.topology.loops == 1 else 18)
    n = max(k for k in lat if k < (1 << log2n))
    z = lat[n]
    shifts = W.shifts(cfg.seed + rank, N_SHIFTS)
    evaluator = {"auto": N.QMC_EVAL_AUTO, "table": N.QMC_EVAL_TABLE, "generated": N.QMC_EVAL_GENERATED}[args.evaluator]
    if evaluator != N.QMC_EVAL_TABLE:
        api.gen_compile(prep, precision=N.QMC_PREC_FP64)  # generated FP64 evaluator compiled before any timing
    p = api.make_pass(n, z, N_SHIFTS, 3, evaluator=evaluator)
    ns = prep.info.n_sectors
    stream = torch.cuda.Stream(device=dev_name)
    sh = torch.tensor(shifts, device=dev_name)
    lam = torch.full((ns,), LAMBDA, dtype=torch.float64, device=dev_name)
    sums, fails = di.outputs(p)
    scr, scr_bytes = di.scratch(p)
    # lambda per sector: halved where the sign check of Eq. 14 fails on this workload (as qmc_integrate does)
    halvings = 0
    for _ in range(6):
        di.eval_sums(p, sh, lam, sums, fails)
        bad = fails.sum(dim=1) > 0
        if not bool(bad.any()):
            break
        lam[bad] *= 0.5
        halvings += int(bad.sum().item())
    lam_desc = f"{LAMBDA}" if halvings == 0 else f"{LAMBDA} halved per failing sector ({halvings} halvings)"
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev_name)
    L = N.lib()
    evals_per_step = ns * N_SHIFTS * n

    def step(evs):
        with torch.cuda.stream(stream):
            flush.fill_(1)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            N.check(L.qmc_eval_partials(prep.packed, di.dpacked.data_ptr(), p, sh.data_ptr(), lam.data_ptr(), scr,
                                        scr_bytes, stream.cuda_stream), "qmc_eval_partials")
            e1.record(stream)
            N.check(L.qmc_reduce_partials(prep.packed, di.dpacked.data_ptr(), p, scr, scr_bytes, sums.data_ptr(),
                                          fails.data_ptr(), stream.cuda_stream), "qmc_reduce_partials")
            e2.record(stream)
            evs.append((e0, e1, e2))

    warm = []
    for _ in range(args.warmup):
        step(warm)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    evs = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(evs)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    elapsed = t1 - t0
    if dist:
        elapsed = max_over_ranks(elapsed, dist, dev_name)
    eval_ms = [a.elapsed_time(b) for a, b, c in evs]
    pass_ms = [a.elapsed_time(c) for a, b, c in evs]
    sign_failures = int(fails.sum().item())
    value = world * evals_per_step * args.steps / elapsed
    flops_launch = prep.info.flops_per_eval * evals_per_step
    achieved = flops_launch / (statistics.mean(eval_ms) * 1e-3) / 1e12
    kh = kernel_hash()
    traffic = TRAFFIC_BYTES if (TRAFFIC_BYTES is not None and kh == KERNEL_HASH) else None

    # the same pass in mixed precision (FP32 evaluation, FP64 lattice arithmetic and accumulation), with the
    # evaluator generated for this family (compiled here, before any timing) and with the table evaluator
    gen_info = api.gen_compile(prep)
    pm = api.make_pass(n, z, N_SHIFTS, 3, precision=N.QMC_PREC_MIXED, evaluator=N.QMC_EVAL_GENERATED)
    scr_m, scr_m_bytes = di.scratch(pm)
    sums_m, fails_m = di.outputs(pm)

    def step_mixed(evs_m):
        with torch.cuda.stream(stream):
            flush.fill_(1)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            N.check(L.qmc_eval_partials(prep.packed, di.dpacked.data_ptr(), pm, sh.data_ptr(), lam.data_ptr(), scr_m,
                                        scr_m_bytes, stream.cuda_stream), "qmc_eval_partials")
            e1.record(stream)
            N.check(L.qmc_reduce_partials(prep.packed, di.dpacked.data_ptr(), pm, scr_m, scr_m_bytes,
                                          sums_m.data_ptr(), fails_m.data_ptr(), stream.cuda_stream),
                    "qmc_reduce_partials")
            e2.record(stream)
            evs_m.append((e0, e1, e2))

    for _ in range(args.warmup):
        step_mixed([])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    evs_m = []
    tm0 = time.perf_counter()
    for _ in range(args.steps):
        step_mixed(evs_m)
    torch.cuda.synchronize()
    tmix = time.perf_counter() - tm0
    if dist:
        tmix = max_over_ranks(tmix, dist, dev_name)
    mix_eval_ms = statistics.mean(a.elapsed_time(b) for a, b, c in evs_m)
    s64 = sums.cpu().numpy()
    s32 = sums_m.cpu().numpy()
    mixed_dev = float(np.max(np.abs(s32 - s64)) / np.max(np.abs(s64)))
    # table evaluator on the same pass (for comparison; fewer steps)
    pt = api.make_pass(n, z, N_SHIFTS, 3, precision=N.QMC_PREC_MIXED, evaluator=N.QMC_EVAL_TABLE)
    evs_t = []
    for i in range(2 + max(1, args.steps // 2)):
        with torch.cuda.stream(stream):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            N.check(L.qmc_eval_partials(prep.packed, di.dpacked.data_ptr(), pt, sh.data_ptr(), lam.data_ptr(), scr_m,
                                        scr_m_bytes, stream.cuda_stream), "qmc_eval_partials")
            e1.record(stream)
            if i >= 2:
                evs_t.append((e0, e1))
    torch.cuda.synchronize()
    tab_eval_ms = statistics.mean(a.elapsed_time(b) for a, b in evs_t)
    mixed = {"value": world * evals_per_step * args.steps / tmix, "unit": "evals/s", "dtype": "f32+f64",
             "evaluator": "generated", "codegen_compile_ms": gen_info.compile_ms,
             "table_evaluator": {"eval_kernel_ms": tab_eval_ms, "evals_per_s_kernel": evals_per_step / (tab_eval_ms * 1e-3),
                                 "frac": flops_launch / (tab_eval_ms * 1e-3) / 1e12 / FP32_PEAK_TFLOPS},
             "ms_per_step": 1e3 * tmix / args.steps, "eval_kernel_ms": mix_eval_ms,
             "roofline": {"bound": "alu", "achieved": flops_launch / (mix_eval_ms * 1e-3) / 1e12,
                          "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                          "frac": flops_launch / (mix_eval_ms * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
                          "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x 2070 MHz"},
             "max_rel_dev_from_fp64_sums": mixed_dev, "sign_failures": int(fails_m.sum().item())}

    # e2e: the same pass through the host-buffer entry point, copies inside the timed region
    ctx = api.Context(local, 1 << 30, stream)
    import ctypes
    packed_pinned = torch.frombuffer(bytearray(prep.packed), dtype=torch.uint8).pin_memory()
    sh_pinned = torch.tensor(shifts).pin_memory()
    lam_pinned = torch.full((ns,), LAMBDA, dtype=torch.float64).pin_memory()
    sums_h = torch.zeros((ns, N_SHIFTS, prep.info.n_slots, 2), dtype=torch.float64).pin_memory()
    fails_h = torch.zeros((ns, N_SHIFTS), dtype=torch.int64).pin_memory()

    def e2e_step():
        N.check(L.qmc_eval_sums_host(ctx._c, ctypes.c_void_p(packed_pinned.data_ptr()), p, sh_pinned.data_ptr(),
                                     lam_pinned.data_ptr(), sums_h.data_ptr(), fails_h.data_ptr()),
                "qmc_eval_sums_host")

    for _ in range(max(1, args.warmup)):
        e2e_step()
    if dist:
        dist.barrier()
    te0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    te = time.perf_counter() - te0
    if dist:
        te = max_over_ranks(te, dist, dev_name)
    h2d = len(prep.packed) + sh_pinned.numel() * 8 + lam_pinned.numel() * 8
    d2h = sums_h.numel() * 8 + fails_h.numel() * 8
    ctx.close()

    extras = {"mixed": mixed}
    if not args.no_extras and rank == 0:
        seeds = 32 if cfg.topology.loops == 1 else 6
        extras["time_to_1e-3"] = time_to_accuracy(api, blob, cfg, local, stream, seeds, lock_step=1)
        extras["time_to_1e-3_fp64_per_sector"] = time_to_accuracy(api, blob, cfg, local, stream, seeds)
        extras["time_to_1e-3_mixed"] = time_to_accuracy(api, blob, cfg, local, stream, seeds,
                                                         precision=N.QMC_PREC_MIXED)
        if cfg is W.CONFIG1:
            # the paper's own workloads beside the headline: its one-loop scan through the serving loop and its
            # Table 2 points (each guarded, so that a failure there cannot cost the line)
            for key, fn in (("paper_ia_scan", lambda: paper_ia_scan(1000, device=local)),
                            ("paper_table2", lambda: paper_table2(seeds=4, device=local))):
                try:
                    extras[key] = fn()
                except Exception as exc:  # noqa: BLE001
                    extras[key] = {"error": f"{type(exc).__name__}: {exc}"}
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(cfg, n, ns, lam_desc),
            "e2e": {"value": world * evals_per_step * args.steps / te, "unit": "evals/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": 2 * args.steps,  # per step: qmc_eval_kernel + qmc_finalize_kernel
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                         "kernel": ("qd_eval_c1 (generated FP64 evaluator)" if evaluator != N.QMC_EVAL_TABLE
                                    else f"qmc_eval_kernel<{prep.info.dim},deform,{maxm_of(prep)}>"),
                         "flops_per_eval": prep.info.flops_per_eval, "sign_failures": sign_failures,
                         "eval_kernel_ms": statistics.mean(eval_ms), "pass_ms": statistics.mean(pass_ms),
                         "peak_source": "derived: 152 SM x 2 FP64 FMA/clk x 2070 MHz (recipe FP64 1.25 TFLOP/s)",
                         "kernel_hash": kh},
            "clocks": clocks,
        }
        if not args.no_extras:
            out["cpu_baseline"] = cpu_baseline(cfg)
        out.update(extras)
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def maxm_of(prep):
    k = prep.info.n_slots - 1
    return 0 if k == 0 else (2 if k <= 2 else 4)


def pct(v, q):
    v = sorted(v)
    return v[min(len(v) - 1, max(0, int(math.ceil(q * len(v))) - 1))]


def serving_run(n_requests=24, rate=50.0, seed=0, precision=1, device=0, baseline=False, max_seconds=300.0):
    """Config 4: Poisson arrivals of requests for random integrals (massless box, massive box, planar and
    non-planar double box) at random s ~ U[4.5,12], t ~ U[-4,-0.5], each integrated to 1e-3 relative error with 16
    shifts by the serving loop (continuous batching, per-sector lattices).  Latency = submission to completion.
    baseline: the same requests afterwards one at a time through the plain FP64 per-integral path (qmc_integrate,
    FP64, all sectors on one lattice ladder); its latency is the request's own integration time, i.e. as if each
    arrived at an idle GPU, which favours the baseline."""
    from paper_1508_02512_gb300 import api
    from paper_1508_02512_gb300 import tables as T
    arrivals = W.serving_arrivals(n_requests, rate, seed)
    ctx = api.Context(device, 8 << 30)
    blobs = [T.compile_integral(c.topology, T.zero_invariants_of(c.topology, c.point)) for c in W.CONFIGS]
    ids = [ctx.load_sectors(b) for b in blobs]
    # generated evaluators (FP32 and FP64) of the four families, compiled before the arrivals start
    compile_ms = {}
    for c, b in zip(W.CONFIGS, blobs):
        prep = api.prepare(b, c.kin, c.order_min, c.order_max)
        compile_ms[c.name] = sum(api.gen_compile(prep, precision=pr).compile_ms
                                 for pr in (N_PREC_MIXED, N_PREC_FP64))
    # warm the kernels once
    w = ctx.submit(ids[1], W.CONFIG1.kin, 0, 0, rel_tol=1e-3, n_shifts=N_SHIFTS, seed=1, precision=precision)
    ctx.wait(w)
    base = ctx.serving_stats()
    reqs = []
    t0 = time.perf_counter()
    k = 0
    pending = {}
    done = {}
    while len(done) < n_requests:
        now = time.perf_counter() - t0
        while k < n_requests and arrivals[k][0] <= now:
            at, ci, sv, tv = arrivals[k]
            cfg = W.CONFIGS[ci]
            kin = W.kinematics(cfg.topology, **{**cfg.point, "s": sv, "t": tv})
            rid = ctx.submit(ids[ci], kin, cfg.order_min, cfg.order_max, rel_tol=1e-3, n_shifts=N_SHIFTS,
                             seed=100 + k, lam=LAMBDA, precision=precision, max_seconds=300.0)
            pending[rid] = (k, ci, time.perf_counter() - t0)
            k += 1
        for rid in list(pending):
            st, r = ctx.poll(rid)
            if st != 1:
                done[rid] = (pending.pop(rid), r)
        time.sleep(0.0005)
    wall = time.perf_counter() - t0
    stats = ctx.serving_stats()
    lat = sorted(r.seconds for (_, r) in done.values())
    ok = sum(1 for (_, r) in done.values() if r.status == 0)
    per_cfg = {}
    for (k_, ci, _), r in done.values():
        per_cfg.setdefault(W.CONFIGS[ci].name, []).append(r.seconds)
    ctx.close()
    out = {"requests": n_requests, "converged": ok, "offered_rate_per_s": rate, "wall_s": wall,
           "throughput_req_per_s": n_requests / wall, "p50_s": statistics.median(lat), "p99_s": pct(lat, 0.99),
           "per_integral_p50_s": {k2: statistics.median(v) for k2, v in per_cfg.items()},
           "rounds": stats.rounds - base.rounds, "batched_passes": stats.batched_passes - base.batched_passes,
           "peak_active": stats.peak_active, "precision": "f32+f64" if precision == 1 else "f64",
           "codegen_compile_ms": compile_ms, "rel_tol": 1e-3, "shifts": N_SHIFTS}
    if baseline:
        ctx = api.Context(device, 8 << 30)
        ids = [ctx.load_sectors(b) for b in blobs]
        secs, ok_b, evals = [], 0, 0
        for k, (at, ci, sv, tv) in enumerate(arrivals):
            cfg = W.CONFIGS[ci]
            ctx.set_kinematics(ids[ci], W.kinematics(cfg.topology, **{**cfg.point, "s": sv, "t": tv}),
                               cfg.order_min, cfg.order_max)
            r = ctx.integrate(ids[ci], rel_tol=1e-3, n_shifts=N_SHIFTS, seed=100 + k, lam=LAMBDA,
                              precision=N_PREC_FP64, lock_step=1, max_seconds=max_seconds)
            secs.append(r.seconds)
            ok_b += r.status == 0
            evals += r.evals
        ctx.close()
        out["fp64_per_integral_baseline"] = {
            "path": "qmc_integrate, FP64, one integral at a time, all sectors on one lattice ladder",
            "converged": ok_b, "max_seconds": max_seconds, "total_s": sum(secs),
            "p50_s": statistics.median(secs), "p99_s": pct(secs, 0.99), "evals": evals}
    return out


def paper_ia_scan(n_points=1000, rel_tol=1e-4, precision=1, device=0, max_seconds=60.0):
    """The paper's one-loop scan I_A (Sec. IV): the gg -> HH box with four top-quark lines at n_points values of
    s from 70000 to 500000 GeV^2 (t = -6000 GeV^2), submitted together to the serving loop, each integrated to
    rel_tol with 16 shifts.  Reports the scan's wall time per point beside the paper's 83 ms per point (K20),
    request latencies, the achieved relative errors, the imaginary part below threshold (s < 4 M_t^2, where the
    integral is real), and a few values converted to the paper's I_A = i/(16 pi^2) I / M_t^4 (GeV^-4)."""
    from paper_1508_02512_gb300 import api
    from paper_1508_02512_gb300 import tables as T
    topo = W.box(True)
    s_vals = np.linspace(*W.PAPER_IA_S_RANGE_GEV2, n_points)
    pts = [W.paper_ia_point(s) for s in s_vals]
    blob = T.compile_integral(topo, T.zero_invariants_of(topo, pts[0]))
    ctx = api.Context(device, 8 << 30)
    iid = ctx.load_sectors(blob)
    prep = api.prepare(blob, W.kinematics(topo, **pts[0]), 0, 0)
    compile_ms = sum(api.gen_compile(prep, precision=pr).compile_ms for pr in (N_PREC_MIXED, N_PREC_FP64))
    ctx.wait(ctx.submit(iid, W.kinematics(topo, **pts[-1]), 0, 0, rel_tol=rel_tol, n_shifts=N_SHIFTS, seed=1,
                        precision=precision))  # warm-up
    t0 = time.perf_counter()
    rids = [ctx.submit(iid, W.kinematics(topo, **pt), 0, 0, rel_tol=rel_tol, n_shifts=N_SHIFTS, seed=100 + i,
                       lam=LAMBDA, precision=precision, max_seconds=max_seconds) for i, pt in enumerate(pts)]
    res = [ctx.wait(r, timeout=max_seconds + 600.0) for r in rids]
    wall = time.perf_counter() - t0
    stats = ctx.serving_stats()
    ctx.close()
    mt4 = W.M_T_GEV ** 4
    vals = [complex(r.value[0][0], r.value[0][1]) for r in res]
    errs = [math.hypot(r.error[0][0], r.error[0][1]) for r in res]
    rel = [e / abs(v) if v != 0 else float("inf") for v, e in zip(vals, errs)]
    thr = 4.0 * W.M_T_GEV ** 2
    below = [abs(v.imag) / max(e, 1e-300) for s, v, e in zip(s_vals, vals, errs) if s < thr]
    samples = []
    for s_want in (70000.0, 100000.0, 118000.0, 120000.0, 150000.0, 200000.0, 300000.0, 500000.0):
        i = int(np.argmin(np.abs(s_vals - s_want)))
        ia = 1j / (16.0 * math.pi ** 2) * vals[i] / mt4
        samples.append({"s_gev2": float(s_vals[i]), "I_A_re": ia.real, "I_A_im": ia.imag, "rel_err": rel[i],
                        "latency_s": res[i].seconds, "status": res[i].status})
    lat = sorted(r.seconds for r in res)
    return {"metric": "paper I_A scan: wall time per point", "points": n_points, "rel_tol": rel_tol,
            "shifts": N_SHIFTS, "precision": "f32+f64" if precision == 1 else "f64",
            "converged": sum(r.status == 0 for r in res), "wall_s": wall, "ms_per_point": 1e3 * wall / n_points,
            "latency_p50_s": statistics.median(lat), "latency_p99_s": pct(lat, 0.99),
            "median_rel_err": statistics.median(rel), "max_rel_err": max(rel),
            "below_threshold_max_abs_im_over_err": max(below) if below else None,
            "evals": sum(r.evals for r in res), "rounds": stats.rounds, "peak_active": stats.peak_active,
            "codegen_compile_ms": compile_ms, "samples": samples,
            "paper": {"ms_per_point": 83, "hardware": "NVIDIA K20", "accuracy": "within 1e-3, mostly below 1e-4"}}


def time_to_accuracy(api, blob, cfg, device, stream, seeds=32, precision=0, lock_step=0):
    """qmc_integrate of the integral to 1e-3 relative error (lattice ladder from 2^10), over `seeds` seeds.
    precision FP64 with lock_step = 1 is the plain FP64 per-integral path (all sectors on one ladder)."""
    ctx = api.Context(device, 4 << 30, stream)
    iid = ctx.load_sectors(blob)
    ctx.set_kinematics(iid, cfg.kin, cfg.order_min, cfg.order_max)
    kw = dict(rel_tol=1e-3, n_shifts=N_SHIFTS, lam=LAMBDA, precision=precision, lock_step=lock_step, max_seconds=120)
    ctx.integrate(iid, seed=999, **kw)  # warm-up (kernels, generated evaluator)
    ts, ns, ev, ok = [], [], [], 0
    for s in range(seeds):
        t0 = time.perf_counter()
        r = ctx.integrate(iid, seed=1000 + s, **kw)
        ts.append(1e3 * (time.perf_counter() - t0))
        ns.append(r.n_final)
        ev.append(r.evals)
        ok += r.status == 0
    ctx.close()
    return {"p50_ms": statistics.median(ts), "p99_ms": pct(ts, 0.99), "seeds": seeds, "converged": ok,
            "median_final_n": int(statistics.median(ns)), "median_evals": int(statistics.median(ev)),
            "precision": "f64" if precision == 0 else "f32+f64",
            "lattices": "one ladder for all sectors" if lock_step else "per sector"}


def paper_table2(seeds=8, rel_tol=1e-4, device=0):
    """The paper's Table 2 (massless planar double box with two off-shell legs, Euclidean, geometric
    decomposition): qmc_integrate of each of its three points to `rel_tol` per order, FP64 and mixed precision,
    p50 over `seeds` shift seeds after a warm-up integration (which compiles the generated evaluators); the
    converted P_i of the first seed beside the paper's printed QMC values."""
    import torch
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from paper_tables import golden_table2, to_paper_euclid
    from paper_1508_02512_gb300 import _native as N
    from paper_1508_02512_gb300 import api
    from paper_1508_02512_gb300 import tables as T
    torch.cuda.set_device(device)
    topo = W.double_box_planar(False)
    table = golden_table2()
    out = {}
    for tag, pt in W.PAPER_IB_POINTS.items():
        blob = T.compile_integral(topo, T.zero_invariants_of(topo, pt), strategy="geometric")
        row = {}
        for prec, name in ((N.QMC_PREC_FP64, "fp64"), (N.QMC_PREC_MIXED, "mixed")):
            ctx = api.Context(device, 4 << 30)
            iid = ctx.load_sectors(blob)
            ctx.set_kinematics(iid, W.kinematics(topo, **pt), -4, 0)
            kw = dict(rel_tol=rel_tol, n_shifts=N_SHIFTS, lam=0.0, precision=prec, max_seconds=120)
            t0 = time.perf_counter()
            ctx.integrate(iid, seed=999, **kw)
            first = time.perf_counter() - t0
            ts, res = [], []
            for s in range(seeds):
                t0 = time.perf_counter()
                r = ctx.integrate(iid, seed=1000 + s, **kw)
                ts.append(time.perf_counter() - t0)
                res.append(r)
            ctx.close()
            val, err = api.result_arrays(res[0])
            P = to_paper_euclid(val.real, np.hypot(err[:, 0], err[:, 1]), pt["s"])
            row[name] = {"p50_s": statistics.median(ts), "max_s": max(ts), "first_call_s": first,
                         "converged": sum(r.status == 0 for r in res), "median_evals": int(statistics.median(
                             r.evals for r in res)), "P": {f"P{i}": [P[i][0], P[i][1]] for i in (4, 3, 2, 1, 0)}}
        row["sectors"] = api.prepare(blob, W.kinematics(topo, **pt), -4, 0).info.n_sectors
        row["paper_qmc_gpu"] = {f"P{i}": list(table[(tag, "qmc")][i]) for i in (4, 3, 2, 1, 0)}
        out[f"legs {tag}"] = row
    return {"metric": f"time to {rel_tol:g} relative error per order, Table 2 points", "rel_tol": rel_tol,
            "shifts": N_SHIFTS, "seeds": seeds, "points": out,
            "paper_times_s": {"legs -1,0,0,-1": 2.2, "legs 0,-1,0,-1": 0.84, "legs 0,0,-1,-1": 2.2}}


def profile_pass(precision="fp64", integral="massive_box"):
    """Two passes of the benchmark integral at n = 1048573 (largest prime below 2^20; 65521 for a two-loop
    integral), 16 shifts: the small case for ncu captures."""
    import torch
    from paper_1508_02512_gb300 import _native as N
    from paper_1508_02512_gb300 import api
    from paper_1508_02512_gb300 import tables as T
    cfg = INTEGRALS[integral]
    blob = T.compile_integral(cfg.topology, T.zero_invariants_of(cfg.topology, cfg.point), strategy=cfg.strategy)
    prep = api.prepare(blob, cfg.kin, cfg.order_min, cfg.order_max)
    dev = api.DeviceIntegral(prep)
    n = 1048573 if cfg.topology.loops == 1 else 65521
    p = api.make_pass(n, dict(api.builtin_lattices())[n], N_SHIFTS, 3,
                      precision=N.QMC_PREC_MIXED if precision == "mixed" else N.QMC_PREC_FP64)
    sh = torch.tensor(W.shifts(cfg.seed, N_SHIFTS), device="cuda")
    lam = torch.full((prep.info.n_sectors,), LAMBDA, dtype=torch.float64, device="cuda")
    sums, fails = dev.outputs(p)
    for _ in range(2):
        dev.eval_sums(p, sh, lam, sums, fails)
    torch.cuda.synchronize()
    print("profile pass ok", int(fails.sum().item()))


if __name__ == "__main__":
    a = parse()
    if a.serving:
        print(json.dumps({"metric": "serving time-to-1e-3", **serving_run(a.serving, baseline=a.serving_baseline)}))
    elif a.paper_ia_scan:
        print(json.dumps(paper_ia_scan(a.paper_ia_scan)))
    elif a.paper_table2:
        print(json.dumps(paper_table2()))
    elif a.profile_pass:
        profile_pass(a.precision, a.integral)
    elif a.impl == "reference":
        main_reference(a)
    else:
        main_ours(a)
