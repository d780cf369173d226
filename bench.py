#!/usr/bin/env python
"""Benchmark of the QMC sector-integration hot path on GB300: integrand evaluations per second and
time-to-1e-3 relative error, mixed precision beside FP64.

Default workload: the two-loop non-planar double box in the physical region (7 propagators, m^2 = 1 on four
lines, massless legs, s = 6, t = -2, u = -4; eps^-2..eps^0; 48 six-dimensional sectors of the iterated
decomposition, every one contour-deformed with lambda = 0.5, halved per sector where the sign check of Eq. 14
fails).  A step is one pass of the whole hot path over it: every sector x 16 random shifts x every point of the
rank-1 lattice of size n = 1048573 (largest prime below 2^20), Korobov transform r = 3 -- 8.05e8 integrand
evaluations, reduced per (sector, shift) -- in mixed precision as the library runs it: the FP32/FP64 probe
with island bins (qmc_probe_islands, 4096 points per sector) and qmc_choose_precision keep a sector in FP32 (with
FP64 islands near its singular faces where that is cheaper) unless its FP32 error exceeds 1e-4 of its magnitude,
and the sectors it flags run in FP64 in the same step.

Output: one JSON line (rank 0).
  value      evaluations/s of the mixed step, with the table, shifts and lambda already resident on the device
  e2e        the same metric through qmc_eval_sums_host (host buffers; copies inside the timed region)
  roofline   algorithmic FP32 throughput of the FP32 evaluation kernel (flop counted per sector from the tables by
             the library, times the evaluations of one launch, over its CUDA-event time) against the FP32 peak
             derived from the SM count, FP32 lanes and clock
  fp64       the same pass in FP64 alone (n = 262139), with its roofline against the derived FP64 peak
  mixed_error_vs_fp64   per order, the mixed pass's deviation from the FP64 pass on identical points
  time_to_1e-3          qmc_integrate to 1e-3 relative error over 32 seeds: mixed with per-sector lattices (the
                        library's default), FP64 with per-sector lattices, and the plain FP64 per-integral path
                        (all sectors on one lattice ladder)
  serving    a bounded sample of the serving workload (Poisson arrivals at 50/s of random integrals)
  paper_table2, paper_ia_scan   the paper's own workloads with its printed timings beside them
  cpu_baseline   the oracle (plain C, all host cores) on a bounded sample of the same workload

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --integral massive_box|planar_dbox|nonplanar_dbox|massless_dbox_table2 [--log2n 20]
    python bench.py --serving N [--serving-baseline]   the serving workload: N Poisson arrivals
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

N_PREC_FP64 = 0
N_PREC_MIXED = 1
N_SHIFTS = 16
LAMBDA = 0.5
REL_TOL = 1e-3
FP32_BUDGET = 0.1  # the library's default: a sector stays in FP32 while its probe error <= 0.1 * rel_tol
METRIC = "integrand evals/s"
# FP64 peak of a GB300: 152 SMs x 2 FP64 FMA per clock per SM (4 flop) x 2070 MHz maximum SM clock
FP64_PEAK_TFLOPS = 152 * 4 * 2070e6 / 1e12
# FP32 peak: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2070 MHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2070e6 / 1e12
# DRAM bytes per launch of the FP32 evaluation kernel of the default step (the generated qg_eval_c1 of the
# non-planar family at n = 1048573, 16 shifts), dram__bytes_read.sum + dram__bytes_write.sum from one
# single-pass ncu capture of a full-size launch; valid while the device code and the generator hash to
# KERNEL_HASH, null otherwise
TRAFFIC_BYTES = 2267136 + 41216  # read + write
KERNEL_HASH = "01ea503186b1629e"


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
    ap.add_argument("--integral", choices=sorted(INTEGRALS), default="nonplanar_dbox",
                    help="integral of the timed pass (default: the non-planar two-loop double box)")
    ap.add_argument("--evaluator", choices=["auto", "table", "generated"], default="auto",
                    help="polynomial evaluator of the FP64 pass (the mixed pass always uses the generated one)")
    ap.add_argument("--log2n", type=int, default=0, help="lattice size of the timed step: largest prime below "
                                                         "2^log2n (default 24 one-loop, 20 two-loop)")
    ap.add_argument("--tta-seeds", type=int, default=32, help="seeds per path of the time-to-1e-3 figures")
    ap.add_argument("--serving-sample", type=int, default=48,
                    help="requests of the bounded serving sample in the default run (0 = none)")
    ap.add_argument("--profile-pass", action="store_true",
                    help="run two passes of the same integral at n = 1048573 and exit (small case for ncu)")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64", help="precision of --profile-pass")
    ap.add_argument("--profile-log2n", type=int, default=0,
                    help="lattice size of --profile-pass (default 2^20 one-loop, 2^16 two-loop)")
    ap.add_argument("--profile-islands", type=int, default=-1,
                    help="run one mixed pass of the paper's Table 2 point (legs -1,0,0,-1) at n = 32749 with every "
                         "sector at this FP64-island level and exit (the case for ncu captures of the island mode)")
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


def workload_config(cfg, n, ns, lam_desc, precision="mixed"):
    if cfg is W.CONFIG1:
        what = f"massive one-loop box, physical s=5 t=-1.5 m^2=1, lambda={lam_desc}, {ns} sectors"
    elif cfg is W.PAPER_IB:
        what = (f"massless planar double box (the paper's Table 2, legs p1^2 = p4^2 = -1), Euclidean s=t=u=-2/3, "
                f"eps^-4..eps^0, geometric decomposition, {ns} six-dimensional sectors")
    elif cfg is W.CONFIG2:
        what = (f"planar two-loop double box, physical s=6 t=-2, m^2=1 on four lines, massless legs, "
                f"eps^-2..eps^0, lambda={lam_desc}, {ns} six-dimensional sectors")
    else:
        what = (f"non-planar two-loop double box, physical s=6 t=-2 u=-4, m^2=1 on four lines, massless legs, "
                f"eps^-2..eps^0, lambda={lam_desc}, {ns} six-dimensional sectors")
    prec = ("mixed precision (FP32 evaluation of the sectors the FP32/FP64 probe keeps, FP64 for the others; FP64 "
            "lattice arithmetic and accumulation)" if precision == "mixed" else "FP64")
    return {"workload": f"{what} x {N_SHIFTS} shifts x n={n} rank-1 lattice, Korobov r=3, {prec}",
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


def phase(name, t0):
    """Duration of a bench phase, on stderr (stdout carries the one JSON line)."""
    print(f"bench: {name} took {time.perf_counter() - t0:.1f} s", file=sys.stderr, flush=True)


def korobov_vector(n, a=76):
    """An admissible generating vector (1, a, a^2, ...) mod n for timing the oracle: the cost of an evaluation
    does not depend on which vector the lattice uses."""
    return [pow(a, j, n) for j in range(6)]


def cpu_baseline(cfg=None, n_log2=0):
    """The oracle as it stands (plain C, OpenMP over all host cores) on a bounded sample of the workload:
    n = largest prime below 2^18 for the one-loop box, 2^14 for a double box (about 10-20 s of CPU work)."""
    from oracle import integrate as OI
    from oracle import lattice as OL
    cfg = cfg or W.CONFIG3
    n_log2 = n_log2 or (18 if cfg.topology.loops == 1 else 14)
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
    """The oracle on the same integral as our arm (default: the non-planar double box), each step a bounded
    sample: n = largest prime below 2^16 (one-loop) or 2^12 (two-loop), 16 shifts, all sectors."""
    world, rank, local, dist = dist_setup(args)
    if rank != 0:  # the oracle runs once, on rank 0; the other ranks leave without work
        if dist:
            dist.destroy_process_group()
        return
    from oracle import integrate as OI
    from oracle import lattice as OL
    cfg = INTEGRALS[args.integral]
    prob = OI.make_problem(cfg.topology, {**cfg.point}, cfg.order_min, cfg.order_max, cfg.strategy)
    lg = 16 if cfg.topology.loops == 1 else 12
    n = OL.prime_below(1 << lg)
    z = korobov_vector(n)
    shifts = W.shifts(12345, N_SHIFTS)
    cores = os.cpu_count() or 1
    lam = LAMBDA if cfg.lam > 0 else 0.0
    for _ in range(args.warmup):
        OI.integrate(prob, n, z, shifts, lam, 3, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        OI.integrate(prob, n, z, shifts, lam, 3, nthreads=cores)
    dt = time.perf_counter() - t0
    ns = len(prob.sectors)
    evals = ns * N_SHIFTS * n
    v = evals * args.steps / dt
    sample = (f"each step: {cfg.name}, n={n} (largest prime < 2^{lg}), {N_SHIFTS} shifts, {ns} sectors = {evals} "
              f"evals, FP64")
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "evals/s", "n_gpus": args.gpus,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": workload_config(cfg, n, ns, f"{lam}", "fp64"),
                      "cpu_baseline": {"value": v, "unit": "evals/s", "cores": cores, "kind": "oracle",
                                       "sample": sample},
                      "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
    if dist:
        dist.destroy_process_group()


def probe_codes(L, N, prep, di, p_mixed, sh, lam, rel_tol, fp32_budget):
    """Per-sector precision codes of the timed mixed pass, as the library chooses them before it has an estimate
    of the integral: the FP32/FP64 probe with island bins (qmc_probe_islands, 4096 strided points of the first
    shift) and qmc_choose_precision without sums (each sector held to fp32_budget * rel_tol of its own
    magnitude).  Returns (codes: 1 FP32, 2 + L FP32 with FP64 islands, 0 FP64; the probe's largest ratio
    sum|v32 - v64| / sum|v64| per sector), table order."""
    import ctypes
    import torch
    ns, slots = prep.info.n_sectors, prep.info.n_slots
    out = torch.zeros((ns, slots, 4), dtype=torch.float64, device=sh.device)
    bins = torch.zeros((ns, N.QMC_ISLAND_BINS, N.island_bin_words(slots)), dtype=torch.float64, device=sh.device)
    N.check(L.qmc_probe_islands(prep.packed, di.dpacked.data_ptr(), ctypes.byref(p_mixed), sh.data_ptr(),
                                lam.data_ptr(), 4096, out.data_ptr(), bins.data_ptr(), None), "qmc_probe_islands")
    torch.cuda.synchronize()
    pr = np.ascontiguousarray(out.cpu().numpy())
    bn = np.ascontiguousarray(bins.cpu().numpy())
    codes = np.zeros(ns, dtype=np.int32)
    N.check(L.qmc_choose_precision(prep.packed, 0, None, None, pr.ctypes.data, bn.ctypes.data, 4096, rel_tol,
                                   fp32_budget, codes.ctypes.data, None), "qmc_choose_precision")
    ratio = pr[:, :, 1] / np.maximum(pr[:, :, 0], 1e-300)
    return codes, ratio.max(axis=1)


def start_compiles(preps):
    """Start background compilations (qmc_gen_compile with load = 2) of the generated FP32 and FP64 evaluators of
    every family the run uses: NVRTC runs them in parallel threads while the measurement proceeds, and each later
    compilation request of a family waits for its own."""
    import ctypes
    from paper_1508_02512_gb300 import _native as N
    for prep in preps:
        for prec in (N.QMC_PREC_MIXED, N.QMC_PREC_FP64):
            info = N.qmc_gen_info()
            rc = N.lib().qmc_gen_compile(prep.packed, prec, 2, ctypes.byref(info))
            if rc < 0:
                raise N.QMCError(rc, "qmc_gen_compile")


def extra_families():
    """Prepared images of the families the extras use (serving mix, the paper's Table 2 points and its I_A scan)."""
    from paper_1508_02512_gb300 import api
    from paper_1508_02512_gb300 import tables as T
    out = []
    for c in W.CONFIGS:
        blob = T.compile_integral(c.topology, T.zero_invariants_of(c.topology, c.point))
        out.append(api.prepare(blob, c.kin, c.order_min, c.order_max))
    topo = W.double_box_planar(False)
    for pt in W.PAPER_IB_POINTS.values():
        blob = T.compile_integral(topo, T.zero_invariants_of(topo, pt), strategy="geometric")
        out.append(api.prepare(blob, W.kinematics(topo, **pt), -4, 0))
    box = W.box(True)
    pt = W.paper_ia_point(W.PAPER_IA_S_RANGE_GEV2[0])
    blob = T.compile_integral(box, T.zero_invariants_of(box, pt))
    out.append(api.prepare(blob, W.kinematics(box, **pt), 0, 0))
    return out


def main_ours(args):
    import ctypes

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
    L = N.lib()
    ns = prep.info.n_sectors
    lat = dict(api.builtin_lattices())
    two_loop = cfg.topology.loops == 2
    log2n = args.log2n or (20 if two_loop else 24)
    n = max(k for k in lat if k < (1 << log2n))
    n64 = max(k for k in lat if k < (1 << (18 if two_loop else 24)))  # lattice of the FP64-alone pass
    evaluator = {"auto": N.QMC_EVAL_AUTO, "table": N.QMC_EVAL_TABLE, "generated": N.QMC_EVAL_GENERATED}[args.evaluator]
    # generated evaluators (FP32 and FP64) compiled before any timing; those of the extras start in parallel
    t_ph = time.perf_counter()
    start_compiles([prep] + (extra_families() if not args.no_extras and rank == 0 else []))
    compile_ms = {"fp32": api.gen_compile(prep, precision=N.QMC_PREC_MIXED).compile_ms}
    if evaluator != N.QMC_EVAL_TABLE:
        compile_ms["fp64"] = api.gen_compile(prep, precision=N.QMC_PREC_FP64).compile_ms
    phase("code generation", t_ph)
    shifts = W.shifts(cfg.seed + rank, N_SHIFTS)
    stream = torch.cuda.Stream(device=dev_name)
    sh = torch.tensor(shifts, device=dev_name)
    lam0 = LAMBDA if cfg.lam > 0 else 0.0
    lam = torch.full((ns,), lam0, dtype=torch.float64, device=dev_name)
    flops = np.array([prep.sector(s).flops for s in range(ns)])

    def mkpass(nn, prec, active=None):
        p = api.make_pass(nn, lat[nn], N_SHIFTS, 3, precision=prec,
                          evaluator=evaluator if prec == N.QMC_PREC_FP64 else N.QMC_EVAL_GENERATED)
        keep = None
        if active is not None:
            keep = (ctypes.c_int32 * ns)(*[int(v) for v in active])
            p.sector_active = ctypes.cast(keep, ctypes.c_void_p)
        return p, keep

    # lambda per sector: halved where the sign check of Eq. 14 fails (as qmc_integrate does), checked by the FP64
    # pass and by the mixed pass of the timed step
    halvings = 0
    sums, fails = di.outputs(api.make_pass(n, lat[n], N_SHIFTS, 3))
    for _ in range(6):
        bad = torch.zeros(ns, dtype=torch.bool, device=dev_name)
        for nn, prec in ((n64, N.QMC_PREC_FP64), (n, N.QMC_PREC_MIXED)):
            p, _k = mkpass(nn, prec)
            di.eval_sums(p, sh, lam, sums, fails)
            bad |= fails.sum(dim=1) > 0
        if not bool(bad.any()):
            break
        lam[bad] *= 0.5
        halvings += int(bad.sum().item())
    lam_desc = f"{lam0}" if halvings == 0 else f"{lam0} halved per failing sector ({halvings} halvings)"

    # precision of each sector in the mixed step: the probe's decision at this lattice size
    p_probe, _k = mkpass(n, N.QMC_PREC_MIXED)
    codes, probe_ratio = probe_codes(L, N, prep, di, p_probe, sh, lam, REL_TOL, FP32_BUDGET)
    keep32 = (codes != 0).astype(np.int32)
    keep64 = 1 - keep32
    n32, n64s = int(keep32.sum()), int(keep64.sum())
    n_isl = int((codes >= 2).sum())
    p32, k32 = mkpass(n, N.QMC_PREC_MIXED, keep32) if n32 else (None, None)
    codes_dev = None
    if p32 is not None and n_isl:  # sectors with FP64 islands: the pass's FP64 kernel takes their island points
        codes_dev = torch.tensor(codes, device=dev_name)
        p32.sector_precision = codes_dev.data_ptr()
    p64m, k64 = mkpass(n, N.QMC_PREC_FP64, keep64) if n64s else (None, None)
    scr = {}

    def scratch(p, tag):
        need = api.scratch_bytes(prep, p)
        if tag not in scr or scr[tag].numel() < need + 256:
            scr[tag] = torch.empty(need + 256, dtype=torch.uint8, device=dev_name)
        base = scr[tag].data_ptr()
        return base + (-base) % 256, need

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev_name)
    sums_m, fails_m = di.outputs(api.make_pass(n, lat[n], N_SHIFTS, 3))

    def launch_eval(p, tag):
        b, nb = scratch(p, tag)
        N.check(L.qmc_eval_partials(prep.packed, di.dpacked.data_ptr(), ctypes.byref(p), sh.data_ptr(),
                                    lam.data_ptr(), b, nb, stream.cuda_stream), "qmc_eval_partials")

    def launch_reduce(p, tag, out_s, out_f):
        b, nb = scratch(p, tag)
        N.check(L.qmc_reduce_partials(prep.packed, di.dpacked.data_ptr(), ctypes.byref(p), b, nb, out_s.data_ptr(),
                                      out_f.data_ptr(), stream.cuda_stream), "qmc_reduce_partials")

    def step_mixed(evs):
        with torch.cuda.stream(stream):
            flush.fill_(1)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            e[0].record(stream)
            if p32 is not None:
                launch_eval(p32, "32")
            e[1].record(stream)
            if p64m is not None:
                launch_eval(p64m, "64m")
            e[2].record(stream)
            if p32 is not None:
                launch_reduce(p32, "32", sums_m, fails_m)
            if p64m is not None:
                launch_reduce(p64m, "64m", sums_m, fails_m)
            e[3].record(stream)
            evs.append(e)

    def timed(step, steps, warmup):
        for _ in range(warmup):
            step([])
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        evs = []
        t0 = time.perf_counter()
        for _ in range(steps):
            step(evs)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        if dist:
            dist.barrier()
            el = max_over_ranks(el, dist, dev_name)
        return el, evs

    t_ph = time.perf_counter()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    for _ in range(args.warmup):
        step_mixed([])
    elapsed, evs = timed(step_mixed, args.steps, 0)
    clocks = sampler.stop()
    evals_step = ns * N_SHIFTS * n
    value = world * evals_step * args.steps / elapsed
    ms32 = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    ms64m = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    step_ms = statistics.mean(e[0].elapsed_time(e[3]) for e in evs)
    fl32 = float((flops * keep32).sum()) * N_SHIFTS * n
    fl64m = float((flops * keep64).sum()) * N_SHIFTS * n
    ach32 = fl32 / (ms32 * 1e-3) / 1e12 if n32 else 0.0
    kh = kernel_hash()
    # kernels of our library launched per step: one evaluation launch per (precision, sector class) and one
    # reduction launch per pass
    cls = np.array([1 if prep.sector(s).kind == 2 else 0 for s in range(ns)])
    launches_mixed = sum(len(set(cls[np.asarray(mask) > 0])) + 1 for mask in (keep32, keep64) if np.any(mask))
    launches_mixed += len(set(cls[codes >= 2]))  # the FP64 kernel of the FP32 pass, for island points

    # the FP64 pass alone (all sectors) on the smaller lattice, and the mixed pass on the same points
    p64, _ = mkpass(n64, N.QMC_PREC_FP64)
    sums64, fails64 = di.outputs(p64)

    def step64(evs_):
        with torch.cuda.stream(stream):
            flush.fill_(1)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            launch_eval(p64, "64")
            e[1].record(stream)
            launch_reduce(p64, "64", sums64, fails64)
            e[2].record(stream)
            evs_.append(e)

    steps64 = max(2, args.steps // 4)
    el64, evs64 = timed(step64, steps64, 1)
    ms64 = statistics.mean(e[0].elapsed_time(e[1]) for e in evs64)
    ev64 = ns * N_SHIFTS * n64
    fl64 = float(flops.sum()) * N_SHIFTS * n64
    fp64 = {"value": world * ev64 * steps64 / el64, "unit": "evals/s", "dtype": "f64", "lattice_n": n64,
            "steps": steps64, "ms_per_step": 1e3 * el64 / steps64,
            "roofline": {"bound": "alu", "achieved": fl64 / (ms64 * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": fl64 / (ms64 * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                         "kernel": ("qd_eval_c1 (generated FP64 evaluator)" if evaluator != N.QMC_EVAL_TABLE
                                    else "qmc_eval_kernel (FP64 table evaluator)"),
                         "eval_kernel_ms": ms64, "flops_per_eval": prep.info.flops_per_eval,
                         "peak_source": "derived: 152 SM x 2 FP64 FMA/clk x 2070 MHz (recipe FP64 1.25 TFLOP/s)"},
            "sign_failures": int(fails64.sum().item())}
    # mixed on the FP64 pass's points: per-order deviation from FP64 (the FP64 sums equal the oracle's to 1e-12)
    pm32, km32 = mkpass(n64, N.QMC_PREC_MIXED, keep32) if n32 else (None, None)
    sums_c, fails_c = di.outputs(p64)
    sums_c.copy_(sums64)
    if pm32 is not None:
        di.eval_sums(pm32, sh, lam, sums_c, fails_c)
    torch.cuda.synchronize()
    a64 = sums64.cpu().numpy()
    am = sums_c.cpu().numpy()
    c64 = a64[..., 0] + 1j * a64[..., 1]
    cm = am[..., 0] + 1j * am[..., 1]
    dev_slot = []
    for k in range(prep.info.n_slots):
        tot = np.abs(c64[:, :, k]).sum(axis=0).max()
        dev_slot.append(float(np.abs(cm[:, :, k] - c64[:, :, k]).sum(axis=0).max() / max(tot, 1e-300)))
    Q64, mean64, err64 = api.combine(prep, p64, a64)
    Qm, meanm, errm = api.combine(prep, p64, am)
    order_dev = [float(abs(meanm[o] - mean64[o]) / max(abs(mean64[o]), 1e-300)) for o in range(len(mean64))]

    # e2e: the mixed step through the host-buffer entry point, copies inside the timed region
    ctx = api.Context(local, 1 << 30, stream)
    sh_pinned = torch.tensor(shifts).pin_memory()
    lam_pinned = lam.cpu().pin_memory()
    sums_h = torch.zeros((ns, N_SHIFTS, prep.info.n_slots, 2), dtype=torch.float64).pin_memory()
    fails_h = torch.zeros((ns, N_SHIFTS), dtype=torch.int64).pin_memory()
    packed_pinned = torch.frombuffer(bytearray(prep.packed), dtype=torch.uint8).pin_memory()
    host_passes = [p for p in (p32, p64m) if p is not None]

    def e2e_step():
        for p in host_passes:
            N.check(L.qmc_eval_sums_host(ctx._c, ctypes.c_void_p(packed_pinned.data_ptr()), ctypes.byref(p),
                                         sh_pinned.data_ptr(), lam_pinned.data_ptr(), sums_h.data_ptr(),
                                         fails_h.data_ptr()), "qmc_eval_sums_host")

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
    h2d = len(host_passes) * (len(prep.packed) + sh_pinned.numel() * 8 + lam_pinned.numel() * 8)
    d2h = len(host_passes) * (sums_h.numel() * 8 + fails_h.numel() * 8)
    ctx.close()

    phase("timed steps, FP64 pass, e2e", t_ph)
    extras = {}
    if not args.no_extras and rank == 0:
        seeds = args.tta_seeds
        tta = {}
        for key, kw in (("mixed_per_sector", dict(precision=N.QMC_PREC_MIXED)),
                        ("fp64_per_sector", dict(precision=N.QMC_PREC_FP64)),
                        ("fp64_per_integral", dict(precision=N.QMC_PREC_FP64, lock_step=1))):
            t_ph = time.perf_counter()
            try:
                tta[key] = time_to_accuracy(api, blob, cfg, local, stream, seeds, **kw)
            except Exception as exc:  # noqa: BLE001 -- a failure there must not cost the line
                tta[key] = {"error": f"{type(exc).__name__}: {exc}"}
            phase(f"time_to_1e-3 {key}", t_ph)
        if all("p50_ms" in tta[k] for k in ("fp64_per_integral", "mixed_per_sector")):
            tta["mixed_speedup_p50_vs_fp64_per_integral"] = (tta["fp64_per_integral"]["p50_ms"] /
                                                             tta["mixed_per_sector"]["p50_ms"])
        extras["time_to_1e-3"] = tta
        guarded = []
        if args.serving_sample > 0:
            guarded.append(("serving", lambda: serving_run(args.serving_sample, device=local, baseline=True,
                                                           baseline_count=min(8, args.serving_sample))))
        guarded += [("paper_table2", lambda: paper_table2(seeds=4, device=local)),
                    ("paper_ia_scan", lambda: paper_ia_scan(1000, device=local))]
        for key, fn in guarded:
            try:
                t_ph = time.perf_counter()
                extras[key] = fn()
                phase(key, t_ph)
            except Exception as exc:  # noqa: BLE001 -- a failure there must not cost the line
                extras[key] = {"error": f"{type(exc).__name__}: {exc}"}
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {**workload_config(cfg, n, ns, lam_desc), "fp32_sectors": n32, "fp64_sectors": n64s,
                       "fp64_island_sectors": n_isl,
                       "fp32_budget": f"{FP32_BUDGET} x rel_tol {REL_TOL}"},
            "e2e": {"value": world * evals_step * args.steps / te, "unit": "evals/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches_mixed * args.steps,
            "roofline": {"bound": "alu", "achieved": ach32, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": ach32 / FP32_PEAK_TFLOPS,
                         "traffic": TRAFFIC_BYTES if (TRAFFIC_BYTES is not None and kh == KERNEL_HASH) else None,
                         "kernel": "qg_eval_c1 (generated FP32 evaluator)", "eval_kernel_ms": ms32,
                         "evals_per_launch": n32 * N_SHIFTS * n,
                         "flops_per_eval": float((flops * keep32).sum() / max(n32, 1)),
                         "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 flop x 2070 MHz", "kernel_hash": kh},
            "fp64_sectors_kernel_ms": ms64m, "fp64_sectors_flop": fl64m, "step_device_ms": step_ms,
            "probe_max_ratio": {"max": float(probe_ratio.max()), "median": float(np.median(probe_ratio))},
            "sign_failures": int(fails_m.sum().item()),
            "codegen_compile_ms": compile_ms,
            "fp64": fp64,
            "mixed_error_vs_fp64": {"lattice_n": n64, "per_slot_l1": dev_slot, "per_order_rel": order_dev,
                                    "fp64_rel_err_per_order": [float(math.hypot(*err64[o]) / max(abs(mean64[o]), 1e-300))
                                                               for o in range(len(mean64))]},
            "clocks": clocks,
        }
        if not args.no_extras:
            t_ph = time.perf_counter()
            out["cpu_baseline"] = cpu_baseline(cfg)
            phase("cpu_baseline", t_ph)
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


def serving_run(n_requests=24, rate=50.0, seed=0, precision=1, device=0, baseline=False, max_seconds=300.0,
                baseline_count=0):
    """Config 4: Poisson arrivals of requests for random integrals (massless box, massive box, planar and
    non-planar double box) at random s ~ U[4.5,12], t ~ U[-4,-0.5], each integrated to 1e-3 relative error with 16
    shifts by the serving loop (continuous batching, per-sector lattices).  Latency = submission to completion.
    baseline: the same requests (the first baseline_count of them, all when 0) afterwards one at a time through
    the plain FP64 per-integral path (qmc_integrate, FP64, all sectors on one lattice ladder); its latency is the
    request's own integration time, i.e. as if each arrived at an idle GPU, which favours the baseline."""
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
        nb = baseline_count if baseline_count > 0 else n_requests
        for k, (at, ci, sv, tv) in enumerate(arrivals[:nb]):
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
            "requests": nb, "converged": ok_b, "max_seconds": max_seconds, "total_s": sum(secs),
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
    ts, ns, ev, ok, kms, rr, isl, worst = [], [], [], 0, [], [], [], 0.0
    for s in range(seeds):
        t0 = time.perf_counter()
        r = ctx.integrate(iid, seed=1000 + s, **kw)
        ts.append(1e3 * (time.perf_counter() - t0))
        ns.append(r.n_final)
        ev.append(r.evals)
        kms.append(r.kernel_ms)
        rr.append(r.fp64_reruns)
        isl.append(r.island_sectors)
        ok += r.status == 0
        val, err = api.result_arrays(r)
        vmax = float(np.max(np.abs(val)))
        for o in range(len(val)):
            worst = max(worst, math.hypot(*err[o]) / max(abs(val[o]), 1e-6 * vmax))
    ctx.close()
    return {"p50_ms": statistics.median(ts), "p99_ms": pct(ts, 0.99), "seeds": seeds, "converged": ok,
            "median_final_n": int(statistics.median(ns)), "median_evals": int(statistics.median(ev)),
            "median_kernel_ms": statistics.median(kms), "median_fp64_sectors": statistics.median(rr),
            "median_island_sectors": statistics.median(isl),
            "worst_rel_err": worst, "precision": "f64" if precision == 0 else "f32+f64",
            "lattices": "one ladder for all sectors" if lock_step else "per sector"}


def paper_table2(seeds=8, rel_tol=1e-4, device=0):
    """The paper's Table 2 (massless planar double box with two off-shell legs, Euclidean, geometric
    decomposition): qmc_integrate of each of its three points to `rel_tol` per order, FP64 and mixed precision,
    p50 over `seeds` shift seeds after a warm-up integration (which compiles the generated evaluators); the
    converted P_i of the first seed beside the paper's printed QMC values."""
    import torch
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


def golden_table2():
    """The paper's printed Table 2 (tests/golden/paper_table_2.txt, a data file): {(column tag, method): {i: (P_i,
    error)}}."""
    out = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "paper_table_2.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        tag, i, method, val, err = line.split()
        out.setdefault((tag, method), {})[int(i)] = (float(val), float(err))
    return out


def to_paper_euclid(c, e, s):
    """Table 2's normalisation: real coefficients c[k] of eps^(k-4) (k = 0..4) with errors e[k], at s < 0, to
    P(eps) = exp(2 eps gamma_E) (-s)^(3 + 2 eps) I(eps); returns {4 - k: (P_{4-k}, error)}, errors added
    linearly."""
    gamma_e = 0.5772156649015329
    a = 2.0 * (gamma_e + math.log(-s))
    out = {}
    for k in range(5):
        w = [a ** (k - q) / math.factorial(k - q) for q in range(k + 1)]
        out[4 - k] = ((-s) ** 3 * sum(w[q] * c[q] for q in range(k + 1)),
                      (-s) ** 3 * sum(abs(w[q]) * e[q] for q in range(k + 1)))
    return out


def profile_pass(precision="fp64", integral="massive_box", log2n=0):
    """Two passes of the benchmark integral at n = 1048573 (largest prime below 2^20; 65521 for a two-loop
    integral, or the largest prime below 2^log2n), 16 shifts: the case for ncu captures."""
    import torch
    from paper_1508_02512_gb300 import _native as N
    from paper_1508_02512_gb300 import api
    from paper_1508_02512_gb300 import tables as T
    cfg = INTEGRALS[integral]
    blob = T.compile_integral(cfg.topology, T.zero_invariants_of(cfg.topology, cfg.point), strategy=cfg.strategy)
    prep = api.prepare(blob, cfg.kin, cfg.order_min, cfg.order_max)
    dev = api.DeviceIntegral(prep)
    lat = dict(api.builtin_lattices())
    n = max(k for k in lat if k < (1 << log2n)) if log2n else (1048573 if cfg.topology.loops == 1 else 65521)
    p = api.make_pass(n, lat[n], N_SHIFTS, 3,
                      precision=N.QMC_PREC_MIXED if precision == "mixed" else N.QMC_PREC_FP64)
    sh = torch.tensor(W.shifts(cfg.seed, N_SHIFTS), device="cuda")
    lam = torch.full((prep.info.n_sectors,), LAMBDA if cfg.lam > 0 else 0.0, dtype=torch.float64, device="cuda")
    sums, fails = dev.outputs(p)
    for _ in range(2):
        dev.eval_sums(p, sh, lam, sums, fails)
    torch.cuda.synchronize()
    print("profile pass ok", int(fails.sum().item()))


def profile_islands(level):
    """One mixed pass of the paper's Table 2 integral (massless planar double box, legs -1,0,0,-1, geometric
    decomposition, 143 sectors) at n = 32749 with 16 shifts, every sector at precision code 2 + level (FP32 with
    FP64 islands): the FP64 kernel evaluates the island points, the FP32 kernel the rest."""
    import torch
    from paper_1508_02512_gb300 import _native as N
    from paper_1508_02512_gb300 import api
    from paper_1508_02512_gb300 import tables as T
    topo = W.double_box_planar(False)
    pt = W.PAPER_IB_POINTS["-1,0,0,-1"]
    blob = T.compile_integral(topo, T.zero_invariants_of(topo, pt), strategy="geometric")
    prep = api.prepare(blob, W.kinematics(topo, **pt), -4, 0)
    dev = api.DeviceIntegral(prep)
    ns = prep.info.n_sectors
    n = 32749
    p = api.make_pass(n, dict(api.builtin_lattices())[n], N_SHIFTS, 3, precision=N.QMC_PREC_MIXED)
    codes = torch.full((ns,), 2 + level, dtype=torch.int32, device="cuda")
    p.sector_precision = codes.data_ptr()
    sh = torch.tensor(W.shifts(7, N_SHIFTS), dtype=torch.float64, device="cuda")
    lam = torch.zeros(ns, dtype=torch.float64, device="cuda")
    sums, fails = dev.outputs(p)
    dev.eval_sums(p, sh, lam, sums, fails)
    torch.cuda.synchronize()
    print("island pass ok", float(sums.abs().sum()))


if __name__ == "__main__":
    a = parse()
    if a.serving:
        print(json.dumps({"metric": "serving time-to-1e-3", **serving_run(a.serving, baseline=a.serving_baseline)}))
    elif a.paper_ia_scan:
        print(json.dumps(paper_ia_scan(a.paper_ia_scan)))
    elif a.paper_table2:
        print(json.dumps(paper_table2()))
    elif a.profile_pass:
        profile_pass(a.precision, a.integral, a.profile_log2n)
    elif a.profile_islands >= 0:
        profile_islands(a.profile_islands)
    elif a.impl == "reference":
        main_reference(a)
    else:
        main_ours(a)
