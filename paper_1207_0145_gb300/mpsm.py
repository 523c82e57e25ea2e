"""ctypes binding of libmpsm (include/mpsm.h): argument marshalling only.

Every step of the join runs in the library's CUDA kernels; this module only
passes pointers and sizes.  Tuples are [n, 2] tensors of int64 or uint64
(key, payload) in CUDA memory, 16-byte aligned (fresh torch allocations are).
If the compiled library is missing the import fails: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import weakref
from dataclasses import dataclass
from typing import Optional, Sequence, Tuple

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmpsm.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_CAPACITY, ERR_DEVICE, ERR_STATE = range(7)
# device check bits (include/mpsm.h, MPSM_DEVERR_*)
DEVERR_LIST_OVERFLOW, DEVERR_SEGMENT_TOO_BIG, DEVERR_WAIT_TIMEOUT, DEVERR_LEVELS = 1, 2, 4, 8
DEVERR_HIST_OVERFLOW, DEVERR_LEARN, DEVERR_BOUNDS = 16, 32, 64
SPLIT_HIST, SPLIT_LEARNED, SPLIT_EQUI_HEIGHT = 0, 1, 2
SEARCH_BINARY, SEARCH_LEARNED, SEARCH_INTERP = 0, 1, 2
PART_S, PART_R, PART_SMALLER = 0, 1, 2
RUNS_RADIX, RUNS_LEARNED = 0, 1
FLAG_TIMING = 1
FLAG_KERNEL_TIMING = 2
FLAG_UNFUSED = 4
FLAG_BOUNDS_TEST = 8  # test only: one segment's recorded bounds made inexact

_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_i32 = ctypes.c_int32
_p = ctypes.c_void_p


class Options(ctypes.Structure):
    _fields_ = [("runs_r", _u32), ("partitions_s", _u32), ("fine_bits", _u32), ("radix_bits", _u32),
                ("join_tile", _u32), ("splitter_mode", _i32), ("search_mode", _i32), ("flags", _u32),
                ("seed", _u64), ("learn_steps", _u32), ("run_len", _u32), ("partition_side", _u32),
                ("run_buckets", _u32), ("reserved", _u32 * 2)]


class Tuning(ctypes.Structure):
    _fields_ = [("radix_bits", _u32), ("join_tile", _u32), ("run_len", _u32), ("partitions_s", _u32)]


class Pairs(ctypes.Structure):
    _fields_ = [("data", _p), ("capacity", _u64)]


class JobDesc(ctypes.Structure):
    _fields_ = [("R", _p), ("nR", _u64), ("S", _p), ("nS", _u64)]


class Stats(ctypes.Structure):
    _fields_ = [("ms_sort_runs", ctypes.c_float), ("ms_splitters", ctypes.c_float), ("ms_scatter", ctypes.c_float),
                ("ms_sort_partitions", ctypes.c_float), ("ms_search", ctypes.c_float), ("ms_join", ctypes.c_float),
                ("ms_learn", ctypes.c_float), ("ms_total", ctypes.c_float), ("runs_r", _u32),
                ("partitions_s", _u32), ("nfine", _u32), ("fine_shift", _u32), ("s_kept", _u64),
                ("part_max", _u64), ("imbalance", ctypes.c_double), ("mean_window", ctypes.c_double),
                ("tiles", _u64), ("levels_r", _u32), ("levels_s", _u32), ("segments_r", _u64),
                ("segments_s", _u64), ("launches", _u32), ("pad", _u32),
                ("loss_s0", ctypes.c_float), ("loss_s", ctypes.c_float), ("loss_r0", ctypes.c_float),
                ("loss_r", ctypes.c_float), ("part_probes", ctypes.c_double), ("search_probes", ctypes.c_double),
                ("search_err", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RmiInfo(ctypes.Structure):
    _fields_ = [("kmin", _u64), ("kmax", _u64), ("cshift", _u32), ("ncell", _u32), ("fit_n", _u32),
                ("train_n", _u32), ("loss0", ctypes.c_float), ("loss", ctypes.c_float)]


RMI_NPARAM, RMI_LEAVES, RMI_CELLS = 1153, 4096, 65536


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", _u32), ("ms", ctypes.c_float)]


class View(ctypes.Structure):
    _fields_ = [("r_runs", _p), ("run_offsets", _p), ("runs_r", _u32), ("key_min", _u64), ("key_max", _u64),
                ("nfine", _u32), ("fine_shift", _u32), ("fine_s", _p), ("fine_r", _p), ("splitters", _p),
                ("partitions_s", _u32), ("s_chunks", _u32), ("s_chunk_offsets", _p), ("chunk_offsets", _p),
                ("part_offsets", _p), ("s_buffer", _p), ("s_kept", _u64), ("tiles", _u64), ("join_tile", _u32),
                ("windows", _p), ("segments", _p), ("n_segments", _u32), ("window_stride", _u32),
                ("seg_windows", _p), ("pass_buffer", _p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libmpsm.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        sig = {
            "mpsm_options_default": ([P(Options)], ctypes.c_int),
            "mpsm_plan_create": ([P(_p), _u64, _u64, _u32, P(Options), _p], ctypes.c_int),
            "mpsm_plan_destroy": ([_p], None),
            "mpsm_join": ([_p, _p, _u64, _p, _u64, P(_u64), P(_u64), P(Pairs)], ctypes.c_int),
            "mpsm_join_host": ([_p, _p, _u64, _p, _u64, P(_u64), P(_u64)], ctypes.c_int),
            "mpsm_host_alloc": ([_u64, P(_p)], ctypes.c_int),
            "mpsm_host_free": ([_p, _u64], ctypes.c_int),
            "mpsm_sort_runs": ([_p, _p, _u64], ctypes.c_int),
            "mpsm_splitters": ([_p, _p, _u64], ctypes.c_int),
            "mpsm_scatter": ([_p], ctypes.c_int),
            "mpsm_sort_partitions": ([_p], ctypes.c_int),
            "mpsm_search": ([_p], ctypes.c_int),
            "mpsm_merge_join": ([_p, P(_u64), P(_u64), P(Pairs)], ctypes.c_int),
            "mpsm_join_batch": ([_p, P(JobDesc), _u32, P(_u64), P(_u64)], ctypes.c_int),
            "mpsm_plan_stats": ([_p, P(Stats)], ctypes.c_int),
            "mpsm_plan_view": ([_p, P(View)], ctypes.c_int),
            "mpsm_strerror": ([ctypes.c_int], ctypes.c_char_p),
            "mpsm_plan_device_errors": ([_p, P(_u32)], ctypes.c_int),
            "mpsm_selftest_wait_timeout": ([_p, _u32, P(_u32)], ctypes.c_int),
            "mpsm_selftest_log2_q16": ([_p, _u64, _p, _u32, _p], ctypes.c_int),
            "mpsm_plan_set_flags": ([_p, _u32], ctypes.c_int),
            "mpsm_plan_kernel_times": ([_p, P(KernelTime), _u32, P(_u32)], ctypes.c_int),
            "mpsm_sort_runs_noalloc": ([_p, _u64, _u32, _p, _p], ctypes.c_int),
            "mpsm_plan_set_tuning": ([_p, P(Tuning)], ctypes.c_int),
            "mpsm_autotune": ([_p, P(JobDesc), _u32, _u32, P(Tuning), P(ctypes.c_float)], ctypes.c_int),
            "mpsm_rmi_loss_grad": ([_p, _p, _p, _u32, _p, _p, P(ctypes.c_float)], ctypes.c_int),
            "mpsm_rmi_train": ([_p, _p, _p, _u32, _u32, ctypes.c_float, _p, P(ctypes.c_float)], ctypes.c_int),
            "mpsm_rmi_fit": ([_p, _p, _p, _u32, _u64, _u64, _u32, ctypes.c_float], ctypes.c_int),
            "mpsm_rmi_predict": ([_p, _u32, _p, _u64, _p, _p], ctypes.c_int),
            "mpsm_rmi_export": ([_p, _u32, P(RmiInfo), _p, _p, _p, _p, _p], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def host_tuples(n: int):
    """An [n, 2] uint64 numpy array in mpsm_host_alloc memory (zeroed, page-locked, on
    huge pages where the host allows) for mpsm_join_host's inputs; the memory is released
    with the last view of it."""
    import numpy as np

    rows = max(1, int(n))
    nbytes = rows * 16
    p = _p()
    _check(lib().mpsm_host_alloc(nbytes, ctypes.byref(p)), "mpsm_host_alloc")
    buf = (ctypes.c_uint64 * (2 * rows)).from_address(p.value)
    weakref.finalize(buf, lib().mpsm_host_free, p.value, nbytes)
    return np.ctypeslib.as_array(buf).reshape(rows, 2)[: int(n)]


class MPSMError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {lib().mpsm_strerror(status).decode()} (status {status})")


def _check(rc: int, what: str):
    if rc != OK:
        raise MPSMError(rc, what)


def _tuples(t) -> Tuple[int, int]:
    """(device pointer, n) of an [n, 2] 64-bit tensor."""
    if t is None:
        return 0, 0
    assert t.dim() == 2 and t.shape[1] == 2 and t.element_size() == 8, "tuples are [n, 2] 64-bit"
    assert t.is_contiguous(), "tuples must be contiguous"
    return t.data_ptr(), t.shape[0]


def make_options(runs_r=0, partitions_s=0, fine_bits=0, radix_bits=0, join_tile=0, splitter_mode=SPLIT_HIST,
                 search_mode=SEARCH_BINARY, timing=False, kernel_timing=False, flags=0,
                 seed=20120145, learn_steps=0, run_len=0, partition_side=0, run_buckets=0) -> Options:
    o = Options()
    lib().mpsm_options_default(ctypes.byref(o))
    o.runs_r, o.partitions_s, o.fine_bits, o.radix_bits, o.join_tile = runs_r, partitions_s, fine_bits, radix_bits, join_tile
    o.splitter_mode, o.search_mode = splitter_mode, search_mode
    o.flags = (FLAG_TIMING if timing else 0) | (FLAG_KERNEL_TIMING if kernel_timing else 0) | flags
    o.seed = seed
    o.learn_steps = learn_steps
    o.run_len = run_len
    o.partition_side = partition_side
    o.run_buckets = run_buckets
    return o


class _RmiMixin:
    """The learned CDF model's entry points on caller data (device float32 / uint64 tensors)."""

    def rmi_loss_grad(self, x, y, theta):
        import torch

        grad = torch.empty(RMI_NPARAM, dtype=torch.float32, device=x.device)
        loss = ctypes.c_float()
        _check(lib().mpsm_rmi_loss_grad(self.handle, x.data_ptr(), y.data_ptr(), x.numel(), theta.data_ptr(),
                                        grad.data_ptr(), ctypes.byref(loss)), "mpsm_rmi_loss_grad")
        return loss.value, grad

    def rmi_train(self, x, y, theta, steps: int, lr: float):
        """Adam steps from theta (updated in place); returns the loss before each step."""
        losses = (ctypes.c_float * max(steps, 1))()
        _check(lib().mpsm_rmi_train(self.handle, x.data_ptr(), y.data_ptr(), x.numel(), steps, lr, theta.data_ptr(),
                                    losses), "mpsm_rmi_train")
        return list(losses)[:steps]

    def rmi_fit(self, keys, y, kmin: int, kmax: int, steps: int = 200, lr: float = 3e-3):
        _check(lib().mpsm_rmi_fit(self.handle, keys.data_ptr(), y.data_ptr(), keys.numel(), kmin, kmax, steps, lr),
               "mpsm_rmi_fit")

    def rmi_predict(self, keys, slot: int = 0):
        import torch

        yhat = torch.empty(keys.numel(), dtype=torch.float32, device=keys.device)
        leaf = torch.empty(keys.numel(), dtype=torch.int32, device=keys.device)
        _check(lib().mpsm_rmi_predict(self.handle, slot, keys.data_ptr(), keys.numel(), yhat.data_ptr(), leaf.data_ptr()),
               "mpsm_rmi_predict")
        return yhat, leaf

    def rmi_export(self, slot: int = 0) -> dict:
        import numpy as np

        info = RmiInfo()
        theta = np.empty(RMI_NPARAM, dtype=np.float32)
        tab = np.empty(RMI_CELLS, dtype=np.uint16)
        base = np.empty(RMI_LEAVES, dtype=np.uint64)
        a = np.empty(RMI_LEAVES, dtype=np.float32)
        b = np.empty(RMI_LEAVES, dtype=np.float32)
        _check(lib().mpsm_rmi_export(self.handle, slot, ctypes.byref(info), theta.ctypes.data, tab.ctypes.data,
                                     base.ctypes.data, a.ctypes.data, b.ctypes.data), "mpsm_rmi_export")
        d = {k: getattr(info, k) for k, _ in info._fields_}
        d.update(theta=theta, cell_leaf=tab, leaf_base=base, leaf_a=a, leaf_b=b)
        return d


class Plan(_RmiMixin):
    """A join plan: owns the device scratch for joins up to (max_nR, max_nS)."""

    def __init__(self, max_nR: int, max_nS: int, max_jobs: int = 1, stream: Optional[int] = None, **options):
        self.options = make_options(**options)
        h = _p()
        _check(lib().mpsm_plan_create(ctypes.byref(h), max_nR, max_nS, max_jobs, ctypes.byref(self.options),
                                      stream or None), "mpsm_plan_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().mpsm_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- whole join
    def join(self, R, S, pairs=None) -> Tuple[int, int]:
        """(count, checksum); `pairs` an optional [cap, 2] CUDA tensor receiving (r_payload, s_payload)."""
        rp, nr = _tuples(R)
        sp, ns = _tuples(S)
        c, k = _u64(), _u64()
        pr = None
        if pairs is not None:
            pp, cap = _tuples(pairs)
            pr = Pairs(pp, cap)
        rc = lib().mpsm_join(self.handle, rp, nr, sp, ns, ctypes.byref(c), ctypes.byref(k),
                             ctypes.byref(pr) if pr is not None else None)
        if rc == ERR_CAPACITY:
            raise MPSMError(rc, f"mpsm_join needs {c.value} pairs")
        _check(rc, "mpsm_join")
        return c.value, k.value

    def join_host(self, R_host, S_host) -> Tuple[int, int]:
        """R_host, S_host: host tensors (pinned for speed) or numpy arrays [n, 2] of 64-bit."""
        def ptr(a):
            if hasattr(a, "data_ptr"):
                return a.data_ptr(), a.shape[0]
            return a.ctypes.data, a.shape[0]
        rp, nr = ptr(R_host)
        sp, ns = ptr(S_host)
        c, k = _u64(), _u64()
        _check(lib().mpsm_join_host(self.handle, rp, nr, sp, ns, ctypes.byref(c), ctypes.byref(k)), "mpsm_join_host")
        return c.value, k.value

    # ---- phases
    def sort_runs(self, R):
        rp, nr = _tuples(R)
        _check(lib().mpsm_sort_runs(self.handle, rp, nr), "mpsm_sort_runs")

    def splitters(self, S):
        sp, ns = _tuples(S)
        _check(lib().mpsm_splitters(self.handle, sp, ns), "mpsm_splitters")

    def scatter(self):
        _check(lib().mpsm_scatter(self.handle), "mpsm_scatter")

    def sort_partitions(self):
        _check(lib().mpsm_sort_partitions(self.handle), "mpsm_sort_partitions")

    def search(self):
        _check(lib().mpsm_search(self.handle), "mpsm_search")

    def merge_join(self, pairs=None) -> Tuple[int, int]:
        c, k = _u64(), _u64()
        pr = None
        if pairs is not None:
            pp, cap = _tuples(pairs)
            pr = Pairs(pp, cap)
        _check(lib().mpsm_merge_join(self.handle, ctypes.byref(c), ctypes.byref(k),
                                     ctypes.byref(pr) if pr is not None else None), "mpsm_merge_join")
        return c.value, k.value

    # ---- batched
    def join_batch(self, jobs: Sequence[Tuple[object, object]]):
        """jobs: sequence of (R, S) CUDA tensors -> (counts, checksums) lists."""
        n = len(jobs)
        arr = (JobDesc * n)()
        for i, (R, S) in enumerate(jobs):
            rp, nr = _tuples(R)
            sp, ns = _tuples(S)
            arr[i] = JobDesc(rp, nr, sp, ns)
        counts = (_u64 * n)()
        sums = (_u64 * n)()
        _check(lib().mpsm_join_batch(self.handle, arr, n, counts, sums), "mpsm_join_batch")
        return list(counts), list(sums)

    @staticmethod
    def _descs(jobs):
        arr = (JobDesc * len(jobs))()
        for i, (R, S) in enumerate(jobs):
            rp, nr = _tuples(R)
            sp, ns = _tuples(S)
            arr[i] = JobDesc(rp, nr, sp, ns)
        return arr

    def set_tuning(self, radix_bits=0, join_tile=0, run_len=0, partitions_s=0):
        t = Tuning(radix_bits, join_tile, run_len, partitions_s)
        _check(lib().mpsm_plan_set_tuning(self.handle, ctypes.byref(t)), "mpsm_plan_set_tuning")

    def autotune(self, jobs, reps: int = 2):
        """Times the candidate tunings on this batch; keeps and returns the fastest (dict, ms)."""
        best = Tuning()
        ms = ctypes.c_float()
        _check(lib().mpsm_autotune(self.handle, self._descs(jobs), len(jobs), reps, ctypes.byref(best),
                                   ctypes.byref(ms)), "mpsm_autotune")
        return {k: getattr(best, k) for k, _ in best._fields_}, ms.value

    # ---- introspection
    def stats(self) -> dict:
        s = Stats()
        _check(lib().mpsm_plan_stats(self.handle, ctypes.byref(s)), "mpsm_plan_stats")
        return s.as_dict()

    def set_flags(self, timing: bool = False, kernel_timing: bool = False, extra: Optional[int] = None):
        if extra is None:
            extra = 0
        flags = (FLAG_TIMING if timing else 0) | (FLAG_KERNEL_TIMING if kernel_timing else 0) | extra
        _check(lib().mpsm_plan_set_flags(self.handle, flags), "mpsm_plan_set_flags")

    def device_errors(self) -> int:
        """MPSM_DEVERR_* bits of the last call that returned MPSM_ERR_DEVICE (0 otherwise)."""
        f = _u32()
        _check(lib().mpsm_plan_device_errors(self.handle, ctypes.byref(f)), "mpsm_plan_device_errors")
        return f.value

    def kernel_times(self) -> dict:
        """{family: (launches, ms)} of the last call made with kernel timing on."""
        arr = (KernelTime * 64)()
        n = _u32()
        _check(lib().mpsm_plan_kernel_times(self.handle, arr, 64, ctypes.byref(n)), "mpsm_plan_kernel_times")
        return {arr[i].name.decode(): (arr[i].launches, arr[i].ms) for i in range(min(n.value, 64))}

    def view(self) -> View:
        v = View()
        _check(lib().mpsm_plan_view(self.handle, ctypes.byref(v)), "mpsm_plan_view")
        return v


def selftest_wait_timeout(spin_limit: int = 1000, stream: Optional[int] = None) -> Tuple[int, int]:
    """(status, MPSM_DEVERR_* bits) of the bounded-wait self-test: a kernel waits on a
    barrier nothing completes and gives up; expect (ERR_DEVICE, DEVERR_WAIT_TIMEOUT)."""
    f = _u32()
    rc = lib().mpsm_selftest_wait_timeout(stream, spin_limit, ctypes.byref(f))
    return rc, f.value


def selftest_log2_q16(n, out, wide: bool = False, stream: Optional[int] = None):
    """floor(2^16 log2 n[i]) into out[i] as the splitter kernel computes it (both 1-D
    64-bit CUDA tensors); `wide` forces the 126-bit path."""
    if n.numel() > out.numel():
        raise ValueError("out is smaller than n")
    _check(lib().mpsm_selftest_log2_q16(n.data_ptr(), n.numel(), out.data_ptr(), int(bool(wide)), stream or None),
           "mpsm_selftest_log2_q16")


def sort_runs_noalloc(R, runs: int, out, stream: Optional[int] = None):
    """Phase 1 for a small input without any device allocation (include/mpsm.h):
    the runs of R (up to 1024 runs of at most 8192 tuples) sorted into `out`."""
    rp, nr = _tuples(R)
    op, no = _tuples(out)
    if no < nr:
        raise ValueError("out is smaller than R")
    _check(lib().mpsm_sort_runs_noalloc(rp, nr, runs, op, stream or None), "mpsm_sort_runs_noalloc")


def strerror(status: int) -> str:
    return lib().mpsm_strerror(status).decode()
