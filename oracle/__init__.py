"""ctypes binding of the CPU oracle (oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg, never by the join library.  Arrays are numpy
uint64 of shape [n, 2] (key, payload) for tuples.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_p = ctypes.c_void_p


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"oracle library missing: {LIB_PATH}; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "oracle_join": ([_p, _u64, _p, _u64, _p, _p, _p, _u64], ctypes.c_int),
            "oracle_brute": ([_p, _u64, _p, _u64, _p, _p], ctypes.c_int),
            "oracle_closed_form": ([_p, ctypes.c_int, _p, _p], ctypes.c_int),
            "oracle_chunk_start": ([_u64, _u64, _u64], _u64),
            "oracle_sort_runs": ([_p, _u64, _u32, _p, _p], ctypes.c_int),
            "oracle_fine_geometry": ([_u64, _u64, _u32, _p], _u32),
            "oracle_worker_histograms": ([_p, _p, _u32, _u64, _u64, _u32, _u32, _p], ctypes.c_int),
            "oracle_run_counts": ([_p, _p, _u32, _u64, _u64, _u32, _u32, _p], ctypes.c_int),
            "oracle_log2_q16": ([_u64], _u64),
            "oracle_log2_q16_big": ([_u64], _u64),
            "oracle_log2_q16_prec": ([_u64, _u32], ctypes.c_int64),
            "oracle_splitters": ([_p, _p, _u32, _u32, _u32, _p, _p], _u32),
            "oracle_splitters_dp": ([_p, _p, _u32, _u32, _u32], _u64),
            "oracle_splitters_kind": ([_p, _p, _u32, _u32, _u32, _u32, _p, _p], _u32),
            "oracle_splitters_dp_kind": ([_p, _p, _u32, _u32, _u32, _u32], _u64),
            "oracle_prefix_sums": ([_p, _u32, _u32, _p, _p], ctypes.c_int),
            "oracle_scatter": ([_p, _p, _u32, _u64, _u64, _u32, _p, _u32, _p, _p], ctypes.c_int),
            "oracle_windows": ([_p, _p, _u64, _p, _p, _u32, _p], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _t(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint64)
    assert a.ndim == 2 and a.shape[1] == 2
    return a


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data if a.size else 0


def join(R, S, with_pairs: bool = False):
    """(count, checksum[, pairs]) of the equi-join; pairs sorted by (r_payload, s_payload)."""
    R, S = _t(R), _t(S)
    c, k = _u64(), _u64()
    if with_pairs:
        # count first, then materialise
        lib().oracle_join(_ptr(R), len(R), _ptr(S), len(S), ctypes.byref(c), ctypes.byref(k), None, 0)
        pairs = np.empty((c.value, 2), dtype=np.uint64)
        lib().oracle_join(_ptr(R), len(R), _ptr(S), len(S), ctypes.byref(c), ctypes.byref(k),
                          _ptr(pairs) or None, c.value)
        return c.value, k.value, pairs
    lib().oracle_join(_ptr(R), len(R), _ptr(S), len(S), ctypes.byref(c), ctypes.byref(k), None, 0)
    return c.value, k.value


def brute(R, S):
    R, S = _t(R), _t(S)
    c, k = _u64(), _u64()
    lib().oracle_brute(_ptr(R), len(R), _ptr(S), len(S), ctypes.byref(c), ctypes.byref(k))
    return c.value, k.value


def closed_form(workload, nthreads: int = 0):
    """(count, checksum) from the generator's bookkeeping of which R row each S tuple came from."""
    spec = workload.host_spec()
    c, k = _u64(), _u64()
    lib().oracle_closed_form(ctypes.byref(spec), nthreads, ctypes.byref(c), ctypes.byref(k))
    return c.value, k.value


def chunk_bounds(n: int, T: int) -> np.ndarray:
    return np.array([lib().oracle_chunk_start(n, T, j) for j in range(T + 1)], dtype=np.uint64)


def sort_runs(R, T: int):
    R = _t(R)
    out = np.empty_like(R)
    off = np.empty(T + 1, dtype=np.uint64)
    lib().oracle_sort_runs(_ptr(R), len(R), T, _ptr(out), off.ctypes.data)
    return out, off


def fine_geometry(kmin: int, kmax: int, B: int):
    sh = _u32()
    nb = lib().oracle_fine_geometry(kmin, kmax, B, ctypes.byref(sh))
    return nb, sh.value


def worker_histograms(S, chunk_off, kmin, kmax, shift, nb):
    S = _t(S)
    chunk_off = np.ascontiguousarray(chunk_off, dtype=np.uint64)
    W = len(chunk_off) - 1
    h = np.empty((W, nb), dtype=np.uint64)
    lib().oracle_worker_histograms(_ptr(S), chunk_off.ctypes.data, W, kmin, kmax, shift, nb, h.ctypes.data)
    return h


def run_counts(Rs, run_off, kmin, kmax, shift, nb):
    Rs = _t(Rs)
    run_off = np.ascontiguousarray(run_off, dtype=np.uint64)
    g = np.empty(nb, dtype=np.uint64)
    lib().oracle_run_counts(_ptr(Rs), run_off.ctypes.data, len(run_off) - 1, kmin, kmax, shift, nb,
                            g.ctypes.data)
    return g


def log2_q16(n: int) -> int:
    """floor(2^16 log2 n) (0 for n <= 1), the Q16 logarithm of the splitter cost."""
    return lib().oracle_log2_q16(n)


def log2_q16_prec(n: int, F: int) -> int:
    """The interval bit-by-bit method with F fractional bits alone; -1 if undecided."""
    return lib().oracle_log2_q16_prec(n, F)


def log2_q16_big(n: int) -> int:
    """The same value straight from its definition, bitlen(n^65536) - 1 (slow)."""
    return lib().oracle_log2_q16_big(n)


def splitters(H, G, P: int, T: int, kind: int = 0):
    """(sp, n_partitions, best_cost) of the contiguous grouping minimising the largest
    partition cost: kind 0 the split-relevant cost (Sec. 4.3), kind 1 equi-height
    (the partitioned side's count alone, Sec. 5.6)."""
    H = np.ascontiguousarray(H, dtype=np.uint64)
    G = np.ascontiguousarray(G, dtype=np.uint64)
    sp = np.empty(len(H), dtype=np.uint32)
    best = _u64()
    np_ = lib().oracle_splitters_kind(H.ctypes.data, G.ctypes.data, len(H), P, T, kind, sp.ctypes.data,
                                      ctypes.byref(best))
    return sp, np_, best.value


def splitters_dp(H, G, P: int, T: int, kind: int = 0) -> int:
    H = np.ascontiguousarray(H, dtype=np.uint64)
    G = np.ascontiguousarray(G, dtype=np.uint64)
    return lib().oracle_splitters_dp_kind(H.ctypes.data, G.ctypes.data, len(H), P, T, kind)


def prefix_sums(h):
    h = np.ascontiguousarray(h, dtype=np.uint64)
    W, P = h.shape
    ps = np.empty((W, P), dtype=np.uint64)
    part_off = np.empty(P + 1, dtype=np.uint64)
    lib().oracle_prefix_sums(h.ctypes.data, W, P, ps.ctypes.data, part_off.ctypes.data)
    return ps, part_off


def scatter(S, chunk_off, kmin, kmax, shift, sp, ps):
    S = _t(S)
    chunk_off = np.ascontiguousarray(chunk_off, dtype=np.uint64)
    sp = np.ascontiguousarray(sp, dtype=np.uint32)
    ps = np.ascontiguousarray(ps, dtype=np.uint64)
    W, P = ps.shape
    kept = int(np.count_nonzero((S[:, 0] >= np.uint64(kmin)) & (S[:, 0] <= np.uint64(kmax))))
    out = np.zeros((kept, 2), dtype=np.uint64)
    lib().oracle_scatter(_ptr(S), chunk_off.ctypes.data, W, kmin, kmax, shift, sp.ctypes.data, P,
                         ps.ctypes.data, _ptr(out))
    return out


def windows(Ss, tile_off, Rs, run_off):
    Ss, Rs = _t(Ss), _t(Rs)
    tile_off = np.ascontiguousarray(tile_off, dtype=np.uint64)
    run_off = np.ascontiguousarray(run_off, dtype=np.uint64)
    nt, T = len(tile_off) - 1, len(run_off) - 1
    win = np.empty((nt, T, 2), dtype=np.uint64)
    lib().oracle_windows(_ptr(Ss), tile_off.ctypes.data, nt, _ptr(Rs), run_off.ctypes.data, T, win.ctypes.data)
    return win
