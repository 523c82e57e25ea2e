"""P-MPSM on the host's cores (Sec. 3.2 and 4 of the paper): the multithreaded CPU
baseline that bench.py times beside the GPU library.  It shares no code with the
GPU path or the oracle.  R is cut into sorted runs and S is range-partitioned, as
in the GPU library; the result is (count, wrapping u64 sum of r.payload +
s.payload) and the milliseconds of phases 1, 2, 3, 4 and their total."""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpmpsm_cpu.so")
_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CPU baseline library missing: {LIB_PATH}; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.pmpsm_join.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                 ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.pmpsm_join.restype = ctypes.c_int
        _lib = L
    return _lib


def join(R, S, threads: int = 0, fine_bits: int = 10):
    """(count, checksum, [ms phase 1, 2, 3, 4, total]) for uint64 [n, 2] arrays (key, payload)."""
    R = np.ascontiguousarray(R, dtype=np.uint64)
    S = np.ascontiguousarray(S, dtype=np.uint64)
    c, k = ctypes.c_uint64(), ctypes.c_uint64()
    ms = (ctypes.c_double * 5)()
    rc = lib().pmpsm_join(R.ctypes.data if len(R) else None, len(R), S.ctypes.data if len(S) else None, len(S),
                          threads, fine_bits, ctypes.byref(c), ctypes.byref(k), ms)
    if rc != 0:
        raise RuntimeError(f"pmpsm_join failed ({rc})")
    return c.value, k.value, list(ms)
