"""Python-facing wrappers of the qmcfi C ABI (marshalling only; every step runs in the native library).

Device buffers are torch CUDA tensors (PyTorch is used for device memory and streams only); the evaluation
itself is one call into the library, which launches the sm_103a kernels on the given stream.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

from . import _native as N


def _dptr(arr) -> ctypes.c_double:
    return arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_lattice(n: int, z: Sequence[int]) -> N.qmc_lattice:
    L = N.qmc_lattice()
    L.n = int(n)
    for j in range(N.QMC_MAX_DIM):
        L.z[j] = int(z[j]) if j < len(z) else 0
    return L


def builtin_lattices():
    """[(n, z)] of the library's built-in ladder (largest prime below 2^k, fast-CBC vectors)."""
    cnt = N.lib().qmc_builtin_lattices(None, 0)
    arr = (N.qmc_lattice * cnt)()
    N.lib().qmc_builtin_lattices(arr, cnt)
    return [(int(a.n), [int(v) for v in a.z]) for a in arr]


def make_pass(n: int, z, n_shifts: int, transform_r: int = 3, precision: int = N.QMC_PREC_FP64, block: int = 0,
              points_per_thread: int = 0, grid: int = 0, evaluator: int = N.QMC_EVAL_AUTO) -> N.qmc_pass:
    p = N.qmc_pass()
    p.lattice = make_lattice(n, z)
    p.n_shifts = n_shifts
    p.transform_r = transform_r
    p.precision = precision
    p.block = block
    p.points_per_thread = points_per_thread
    p.grid = grid
    p.evaluator = evaluator
    return p


def combine_sectors(prep: Prepared, n_shifts: int, n_sector, sums: np.ndarray):
    """qmc_combine_sectors: like combine(), with the lattice size of each sector's sums (table order)."""
    sums = np.ascontiguousarray(sums, dtype=np.float64)
    nv = np.ascontiguousarray(np.asarray(n_sector, dtype=np.int64))
    nord = prep.info.order_max - prep.info.order_min + 1
    Q = np.zeros((n_shifts, nord, 2))
    mean = np.zeros((nord, 2))
    err = np.zeros((nord, 2))
    N.check(N.lib().qmc_combine_sectors(prep.packed, n_shifts, nv.ctypes.data, sums.ctypes.data, Q.ctypes.data,
                                        mean.ctypes.data, err.ctypes.data), "qmc_combine_sectors")
    return Q[..., 0] + 1j * Q[..., 1], mean[:, 0] + 1j * mean[:, 1], err


def gen_source(prep, precision: int = N.QMC_PREC_MIXED) -> str:
    """qmc_gen_source: the CUDA source generated for the family of a prepared integral (FP32 or FP64)."""
    n = ctypes.c_size_t()
    N.check(N.lib().qmc_gen_source(prep.packed, precision, None, 0, ctypes.byref(n)), "qmc_gen_source")
    buf = ctypes.create_string_buffer(n.value)
    N.check(N.lib().qmc_gen_source(prep.packed, precision, buf, n.value, ctypes.byref(n)), "qmc_gen_source")
    return buf.value.decode()


def gen_compile(prep, load: bool = True, precision: int = N.QMC_PREC_MIXED) -> N.qmc_gen_info:
    """qmc_gen_compile: compile (load=False: compile only, no device) or compile-and-cache the family's module."""
    info = N.qmc_gen_info()
    N.check(N.lib().qmc_gen_compile(prep.packed, precision, 1 if load else 0, ctypes.byref(info)), "qmc_gen_compile")
    return info


@dataclass
class Prepared:
    """Host image of a prepared integral (qmc_prepare) and its summary."""
    packed: bytes
    info: N.qmc_info

    @property
    def host_ptr(self):
        return ctypes.c_char_p(self.packed)

    def sector(self, s: int) -> N.qmc_sector_desc:
        d = N.qmc_sector_desc()
        N.check(N.lib().qmc_sector_desc_get(self.packed, s, ctypes.byref(d)), "qmc_sector_desc_get")
        return d


def prepare(table: bytes, invariants, order_min: int, order_max: int) -> Prepared:
    inv = np.ascontiguousarray(np.asarray(invariants, dtype=np.float64))
    info = N.qmc_info()
    L = N.lib()
    N.check(L.qmc_prepare(table, len(table), _dptr(inv), len(inv), order_min, order_max, None, 0,
                          ctypes.byref(info)), "qmc_prepare")
    buf = ctypes.create_string_buffer(int(info.packed_bytes))
    N.check(L.qmc_prepare(table, len(table), _dptr(inv), len(inv), order_min, order_max, buf, len(buf),
                          ctypes.byref(info)), "qmc_prepare")
    return Prepared(buf.raw, info)


def scratch_bytes(prep: Prepared, p: N.qmc_pass) -> int:
    return int(N.lib().qmc_scratch_bytes(prep.packed, ctypes.byref(p)))


def combine(prep: Prepared, p: N.qmc_pass, sums: np.ndarray):
    """Per-shift estimates Q[m, orders], mean[orders] and standard errors (re, im) from host sums."""
    sums = np.ascontiguousarray(sums, dtype=np.float64)
    nord = prep.info.order_max - prep.info.order_min + 1
    m = p.n_shifts
    Q = np.zeros((m, nord, 2))
    mean = np.zeros((nord, 2))
    err = np.zeros((nord, 2))
    N.check(N.lib().qmc_combine(prep.packed, ctypes.byref(p), sums.ctypes.data, Q.ctypes.data, mean.ctypes.data,
                                err.ctypes.data), "qmc_combine")
    return Q[..., 0] + 1j * Q[..., 1], mean[:, 0] + 1j * mean[:, 1], err


class DeviceIntegral:
    """A prepared integral resident on the GPU, with the buffers of one pass (torch-allocated)."""

    def __init__(self, prep: Prepared, device="cuda"):
        import torch
        self.torch = torch
        self.prep = prep
        self.device = torch.device(device)
        self.dpacked = torch.frombuffer(bytearray(prep.packed), dtype=torch.uint8).to(self.device)
        self._scratch = None

    def scratch(self, p: N.qmc_pass):
        need = scratch_bytes(self.prep, p)
        if need == 0:
            raise N.QMCError(N.QMC_ERR_ARG, "qmc_scratch_bytes")
        if self._scratch is None or self._scratch.numel() < need:
            self._scratch = self.torch.empty(need + 256, dtype=self.torch.uint8, device=self.device)
        base = self._scratch.data_ptr()
        off = (-base) % 256
        return base + off, need

    def outputs(self, p: N.qmc_pass):
        t = self.torch
        ns, slots = self.prep.info.n_sectors, self.prep.info.n_slots
        sums = t.zeros((ns, p.n_shifts, slots, 2), dtype=t.float64, device=self.device)
        fails = t.zeros((ns, p.n_shifts), dtype=t.int64, device=self.device)
        return sums, fails

    def eval_sums(self, p: N.qmc_pass, shifts, lam, sums, fails, stream=None):
        """Enqueue one pass (qmc_eval_sums) on `stream` (a torch.cuda.Stream or None for the current one)."""
        t = self.torch
        st = stream if stream is not None else t.cuda.current_stream(self.device)
        scr, nbytes = self.scratch(p)
        N.check(N.lib().qmc_eval_sums(self.prep.packed, self.dpacked.data_ptr(), ctypes.byref(p), shifts.data_ptr(),
                                      lam.data_ptr(), scr, nbytes, sums.data_ptr(), fails.data_ptr(),
                                      st.cuda_stream), "qmc_eval_sums")

    def autotune(self, p: N.qmc_pass, shifts, lam, stream=None) -> N.qmc_tune_result:
        """qmc_autotune: time the candidate launch shapes of pass p and record the fastest (synchronous)."""
        t = self.torch
        st = stream if stream is not None else t.cuda.current_stream(self.device)
        need = int(N.lib().qmc_autotune_scratch_bytes(self.prep.packed, ctypes.byref(p)))
        if need == 0:
            raise N.QMCError(N.QMC_ERR_ARG, "qmc_autotune_scratch_bytes")
        buf = t.empty(need + 256, dtype=t.uint8, device=self.device)
        base = buf.data_ptr() + (-buf.data_ptr()) % 256
        r = N.qmc_tune_result()
        N.check(N.lib().qmc_autotune(self.prep.packed, self.dpacked.data_ptr(), ctypes.byref(p), shifts.data_ptr(),
                                     lam.data_ptr(), base, need, ctypes.byref(r), st.cuda_stream), "qmc_autotune")
        return r

    def eval_points(self, sector: int, p: N.qmc_pass, shift, lam: float, idx, out, fails, stream=None):
        t = self.torch
        st = stream if stream is not None else t.cuda.current_stream(self.device)
        N.check(N.lib().qmc_eval_points(self.prep.packed, self.dpacked.data_ptr(), sector, ctypes.byref(p),
                                        shift.data_ptr(), float(lam), idx.data_ptr(), idx.numel(), out.data_ptr(),
                                        fails.data_ptr(), st.cuda_stream), "qmc_eval_points")



class Context:
    """qmc_create / qmc_load_sectors / qmc_set_kinematics / qmc_integrate."""

    def __init__(self, device: int = 0, mem_budget: int = 0, stream=None):
        self._c = ctypes.c_void_p()
        sp = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        N.check(N.lib().qmc_create(ctypes.byref(self._c), device, mem_budget, sp), "qmc_create")

    def close(self):
        if self._c:
            N.lib().qmc_destroy(self._c)
            self._c = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_sectors(self, table: bytes) -> int:
        i = ctypes.c_int32()
        N.check(N.lib().qmc_load_sectors(self._c, table, len(table), ctypes.byref(i)), "qmc_load_sectors")
        return i.value

    def set_kinematics(self, integral_id: int, invariants, order_min: int, order_max: int):
        inv = np.ascontiguousarray(np.asarray(invariants, dtype=np.float64))
        N.check(N.lib().qmc_set_kinematics(self._c, integral_id, _dptr(inv), len(inv), order_min, order_max),
                "qmc_set_kinematics")

    @staticmethod
    def options(rel_tol=1e-3, abs_tol=0.0, precision=N.QMC_PREC_FP64, n_shifts=16, seed=0, lam=0.5, transform_r=3,
                ladder_start=0, lattices=None, shifts=None, max_n=0, max_seconds=0.0, max_halvings=6, block=0,
                points_per_thread=0, evaluator=N.QMC_EVAL_AUTO, probe_samples=0, fp32_budget=0.0, lock_step=0):
        """qmc_options and the Python objects that must outlive the call that uses them."""
        o = N.qmc_options()
        o.rel_tol, o.abs_tol, o.precision, o.n_shifts, o.seed = rel_tol, abs_tol, precision, n_shifts, seed
        o.lambda_, o.max_halvings, o.transform_r, o.ladder_start = lam, max_halvings, transform_r, ladder_start
        o.max_n, o.max_seconds, o.block, o.points_per_thread = max_n, max_seconds, block, points_per_thread
        o.evaluator, o.probe_samples, o.fp32_budget = evaluator, probe_samples, fp32_budget
        o.lock_step = lock_step
        keep = []
        if lattices is not None:
            arr = (N.qmc_lattice * len(lattices))(*[make_lattice(n, z) for n, z in lattices])
            keep.append(arr)
            o.n_lattices = len(lattices)
            o.lattices = arr
        if shifts is not None:
            sh = np.ascontiguousarray(np.asarray(shifts, dtype=np.float64))
            keep.append(sh)
            o.shifts = _dptr(sh)
        return o, keep

    def submit(self, integral_id: int, invariants, order_min: int, order_max: int, **kw) -> int:
        """qmc_submit: queue a request with the serving loop; returns its id."""
        o, keep = self.options(**kw)
        inv = np.ascontiguousarray(np.asarray(invariants, dtype=np.float64))
        rid = ctypes.c_int64()
        N.check(N.lib().qmc_submit(self._c, integral_id, _dptr(inv), len(inv), order_min, order_max, ctypes.byref(o),
                                   ctypes.byref(rid)), "qmc_submit")
        return rid.value

    def poll(self, request_id: int):
        """(status, qmc_result or None): status QMC_PENDING while queued or running."""
        r = N.qmc_result()
        st = N.lib().qmc_poll(self._c, request_id, ctypes.byref(r))
        if st == N.QMC_ERR_NOT_FOUND:
            raise N.QMCError(st, "qmc_poll")
        return st, (None if st == N.QMC_PENDING else r)

    def wait(self, request_id: int, timeout: float = 600.0, interval: float = 1e-4):
        import time
        t0 = time.perf_counter()
        while True:
            st, r = self.poll(request_id)
            if st != N.QMC_PENDING:
                return r
            if time.perf_counter() - t0 > timeout:
                raise TimeoutError(f"request {request_id} still pending after {timeout} s")
            time.sleep(interval)

    def cancel(self, request_id: int):
        N.check(N.lib().qmc_cancel(self._c, request_id), "qmc_cancel")

    def serving_stats(self) -> N.qmc_serving_stats:
        st = N.qmc_serving_stats()
        N.check(N.lib().qmc_serving_stats_get(self._c, ctypes.byref(st)), "qmc_serving_stats_get")
        return st

    def integrate(self, integral_id: int, rel_tol=1e-3, **kw) -> N.qmc_result:
        """qmc_integrate (blocking); keyword arguments as in options()."""
        o, keep = self.options(rel_tol=rel_tol, **kw)
        r = N.qmc_result()
        st = N.lib().qmc_integrate(self._c, integral_id, ctypes.byref(o), ctypes.byref(r))
        if st < 0 and st not in (N.QMC_ERR_NOT_CONVERGED, N.QMC_ERR_TIMEOUT):
            raise N.QMCError(st, "qmc_integrate")
        return r


def result_arrays(r: N.qmc_result):
    n = r.n_orders
    val = np.array([complex(r.value[k][0], r.value[k][1]) for k in range(n)])
    err = np.array([[r.error[k][0], r.error[k][1]] for k in range(n)])
    return val, err
