"""Seeded synthetic workloads for the MPSM join (inputs only).

The paper evaluates on synthetic relations of 16-byte tuples, a 64-bit join key
and a 64-bit payload (Sec. 5.1): R with unique keys, S drawn from R's keys at a
multiplicity (1, 4, 8 or 16), and skewed variants (Sec. 5.5, 5.6).  This module
builds those shapes, plus the sparse clustered 64-bit domain and the batched
job mix used for the larger configurations.  It holds none of the join's
arithmetic.  Every value is a pure function of (seed, stream, index), evaluated
by ``gen_core.h`` on the host or on the device with identical results; the small
inverse-CDF tables (Zipf ranks, cluster spacing) are built here in FP64 once
and shared byte-for-byte by both sides.

Sizes use the paper's unit M = 2**20 (Sec. 1).
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

M = 1 << 20
DEFAULT_SEED = 20120145

KIND_UNIFORM, KIND_ZIPF, KIND_SPARSE, KIND_NEGCORR, KIND_LOCSKEW = 0, 1, 2, 3, 4
GEN_NONE = (1 << 64) - 1

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmpsm_gen.so")


class GenSpec(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("hR", ctypes.c_uint32),
        ("hS", ctypes.c_uint32),
        ("pad0", ctypes.c_uint32),
        ("nR", ctypes.c_uint64),
        ("nS", ctypes.c_uint64),
        ("seed", ctypes.c_uint64),
        ("zthr", ctypes.c_void_p),
        ("zlo", ctypes.c_void_p),
        ("nz", ctypes.c_uint64),
        ("cl", ctypes.c_void_p),
        ("qtab", ctypes.c_void_p),
        ("ncl", ctypes.c_uint32),
        ("nq", ctypes.c_uint32),
        ("n_fk", ctypes.c_uint64),
    ]


_lib = None


def lib():
    """The compiled generator library (built by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"generator library missing: {LIB_PATH}; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER(GenSpec)
        for name in ("gen_fill_r", "gen_fill_s", "gen_s_rows"):
            fn = getattr(L, name)
            fn.argtypes = [P, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                           ctypes.c_void_p, ctypes.c_int]
            fn.restype = ctypes.c_int
        L.gen_half_width.argtypes = [ctypes.c_uint64]
        L.gen_half_width.restype = ctypes.c_uint32
        L.gen_sorted_key.argtypes = [P, ctypes.c_uint64]
        L.gen_sorted_key.restype = ctypes.c_uint64
        for name in ("gen_permute", "gen_permute_inv"):
            fn = getattr(L, name)
            fn.argtypes = [ctypes.c_uint64] * 4
            fn.restype = ctypes.c_uint64
        L.gen_draw.argtypes = [ctypes.c_uint64] * 3
        L.gen_draw.restype = ctypes.c_uint64
        _lib = L
    return _lib


# ---------------------------------------------------------------- tables


def zipf_table(n: int, theta: float, head: int = 16384, ratio: float = 1.001):
    """Inverse-CDF table of Zipf(theta) over ranks [0, n): P(rank k) ~ (k+1)^-theta.

    The first ``head`` ranks are exact entries; the tail is cut into buckets whose
    end/start ratio is at most ``ratio`` and drawn uniformly within a bucket, with
    bucket mass from the integral of x^-theta over [a+0.5, b+0.5).  Returns
    (thresholds u64[nz], starts u64[nz+1]); a draw u picks the first entry e with
    u < thresholds[e].
    """
    if n <= 0:
        raise ValueError("zipf table needs n >= 1")
    h = min(n, head)
    starts = list(range(h))
    a = h
    while a < n:
        starts.append(a)
        a = min(n, max(a + 1, int(math.ceil(a * ratio))))
    starts.append(n)
    zlo = np.array(starts, dtype=np.uint64)
    nz = len(starts) - 1
    w = np.empty(nz, dtype=np.float64)
    w[:h] = np.arange(1, h + 1, dtype=np.float64) ** (-theta)
    if nz > h:
        lo = zlo[h:-1].astype(np.float64) + 0.5
        hi = zlo[h + 1:].astype(np.float64) + 0.5
        if abs(theta - 1.0) < 1e-12:
            w[h:] = np.log(hi) - np.log(lo)
        else:
            w[h:] = (hi ** (1.0 - theta) - lo ** (1.0 - theta)) / (1.0 - theta)
    cdf = np.cumsum(w) / w.sum()
    thr = np.floor(np.minimum(cdf * 2.0 ** 64, 2.0 ** 64 - 4096.0)).astype(np.uint64)
    thr[-1] = np.uint64(GEN_NONE)
    return thr, zlo


CLUSTER_DTYPE = np.dtype([("g0", "<u8"), ("n", "<u8"), ("lo", "<u8"), ("spread", "<u8")])


def sparse_tables(n_r: int, seed: int, ncl: int = 64, nq: int = 1024):
    """64 clusters over the full uint64 range with log-normal key spacing.

    Cluster c lives in slot [c*2^58, (c+1)*2^58) at a random base.  Its n_c keys
    are lo + 2j + Q_c(j): the 2j term keeps neighbours at least 2 apart (so every
    gap holds a non-key), and Q_c is the normalised quantile function of a signed
    log-normal X = +-exp(sigma Z), sigma ~ U[0.5, 2], scaled to a spread drawn
    log-uniformly in [16 n_c, 2^56] -- dense cores, heavy tails, widely varying
    scales.  The quantile is tabulated at nq+1 points and interpolated in integer
    arithmetic, so keys are exact and strictly increasing.
    """
    from scipy.special import ndtri

    if n_r < 1:
        raise ValueError("sparse workload needs nR >= 1")
    ncl = int(min(ncl, n_r))
    rng = np.random.default_rng([seed & 0xFFFFFFFF, seed >> 32, 0x5A5E])
    w = rng.uniform(0.5, 1.5, ncl)
    n_c = np.floor(n_r * w / w.sum()).astype(np.int64)
    n_c = np.maximum(n_c, 1)
    diff = n_r - int(n_c.sum())
    n_c[int(np.argmax(n_c))] += diff
    assert n_c.min() >= 1 and int(n_c.sum()) == n_r
    cl = np.zeros(ncl, dtype=CLUSTER_DTYPE)
    q = np.zeros((ncl, nq + 1), dtype=np.uint64)
    g0 = 0
    slot = 1 << 58
    u = np.arange(nq + 1, dtype=np.float64) / nq
    for c in range(ncl):
        nc = int(n_c[c])
        e = rng.uniform(math.log2(nc) + 4.0, 56.0)
        spread = int(2.0 ** e)
        base = c * slot + (1 << 50) + int(rng.integers(0, slot - (1 << 57) - (1 << 51)))
        sigma = rng.uniform(0.5, 2.0)
        v = 2.0 * u - 1.0
        p = np.clip(np.abs(v), 1e-9, 1.0 - 1e-9)
        x = np.sign(v) * np.exp(sigma * ndtri(p))
        norm = (x - x[0]) / (x[-1] - x[0])
        d = np.floor(norm * float(spread))
        d = np.clip(d, 0.0, float(spread))
        dq = np.array([int(t) for t in d], dtype=object)
        dq[0] = 0
        dq[-1] = spread
        run = 0
        for i in range(nq + 1):  # non-decreasing, exact integers
            run = max(run, int(dq[i]))
            q[c, i] = run
        cl[c] = (g0, nc, base, spread)
        g0 += nc
    return cl, q


# ---------------------------------------------------------------- workloads


@dataclass
class Workload:
    """One join's inputs: R (nR unique keys) and S (nS tuples).

    kind = KIND_UNIFORM: R keys are a random permutation of 1..nR; S keys are
    uniform foreign keys into R.  KIND_NEGCORR: R's keys are 1..4nR/5 and then every
    16th key (80 % in the low fifth of the domain), in random order; 80 % of S's
    foreign keys fall in the high fifth.  KIND_LOCSKEW: R's keys are 1..nR stored in
    64 row clusters of ascending key ranges, shuffled inside each cluster.  KIND_ZIPF: S rows follow Zipf(theta) over R's
    rows, hot rows at random positions.  KIND_SPARSE: R keys from the clustered
    64-bit domain; round(fk_share * nS) S tuples are foreign keys, the rest fall
    strictly inside gaps between R keys and match nothing.
    """

    kind: int
    n_r: int
    n_s: int
    seed: int = DEFAULT_SEED
    theta: float = 0.9
    fk_share: float = 0.7
    _tables: dict = field(default_factory=dict, repr=False)
    _dev: dict = field(default_factory=dict, repr=False)

    def __post_init__(self):
        if self.kind == KIND_ZIPF and self.n_r > 0:
            self._tables["zthr"], self._tables["zlo"] = zipf_table(self.n_r, self.theta)
        if self.kind == KIND_SPARSE and self.n_r > 0:
            self._tables["cl"], self._tables["qtab"] = sparse_tables(self.n_r, self.seed)

    @property
    def n_fk(self) -> int:
        if self.kind == KIND_SPARSE:
            return int(round(self.fk_share * self.n_s))
        return self.n_s

    def _spec(self, ptrs) -> GenSpec:
        L = lib()
        s = GenSpec()
        s.kind = self.kind
        s.hR = L.gen_half_width(max(self.n_r, 1))
        s.hS = L.gen_half_width(max(self.n_s, 1))
        s.nR, s.nS, s.seed = self.n_r, self.n_s, self.seed & GEN_NONE
        s.n_fk = self.n_fk
        if self.kind == KIND_ZIPF:
            s.zthr, s.zlo = ptrs["zthr"], ptrs["zlo"]
            s.nz = len(self._tables["zthr"])
        if self.kind == KIND_SPARSE:
            s.cl, s.qtab = ptrs["cl"], ptrs["qtab"]
            s.ncl = len(self._tables["cl"])
            s.nq = self._tables["qtab"].shape[1] - 1
        return s

    def host_spec(self) -> GenSpec:
        ptrs = {k: v.ctypes.data for k, v in self._tables.items()}
        return self._spec(ptrs)

    def device_spec(self, device="cuda") -> GenSpec:
        import torch

        if not self._dev and self._tables:
            for k, v in self._tables.items():
                raw = np.ascontiguousarray(v).view(np.uint8)
                self._dev[k] = torch.from_numpy(raw.copy()).to(device)
        ptrs = {k: v.data_ptr() for k, v in self._dev.items()}
        return self._spec(ptrs)

    # host fills (numpy uint64 [n, 2])
    def r_host(self, nthreads: int = 0) -> np.ndarray:
        out = np.empty((self.n_r, 2), dtype=np.uint64)
        spec = self.host_spec()
        _check(lib().gen_fill_r(ctypes.byref(spec), out.ctypes.data, 0, self.n_r, 0, None, nthreads))
        return out

    def s_host(self, nthreads: int = 0) -> np.ndarray:
        out = np.empty((self.n_s, 2), dtype=np.uint64)
        spec = self.host_spec()
        _check(lib().gen_fill_s(ctypes.byref(spec), out.ctypes.data, 0, self.n_s, 0, None, nthreads))
        return out

    def s_rows_host(self, nthreads: int = 0) -> np.ndarray:
        out = np.empty(self.n_s, dtype=np.uint64)
        spec = self.host_spec()
        _check(lib().gen_s_rows(ctypes.byref(spec), out.ctypes.data, 0, self.n_s, 0, None, nthreads))
        return out

    # device fills into caller-owned buffers (pointer to n x 16 bytes)
    def fill_r_device(self, ptr: int, stream: Optional[int] = None):
        spec = self.device_spec()
        _check(lib().gen_fill_r(ctypes.byref(spec), ptr, 0, self.n_r, 1, stream, 0))

    def fill_s_device(self, ptr: int, stream: Optional[int] = None):
        spec = self.device_spec()
        _check(lib().gen_fill_s(ctypes.byref(spec), ptr, 0, self.n_s, 1, stream, 0))


def _check(rc: int):
    if rc != 0:
        raise RuntimeError(f"generator call failed with status {rc}")


# ---------------------------------------------------------------- named workloads


def plain(n_r: int, n_s: int, seed: int = DEFAULT_SEED) -> Workload:
    return Workload(KIND_UNIFORM, n_r, n_s, seed)


def zipf(n_r: int, n_s: int, theta: float = 0.9, seed: int = DEFAULT_SEED) -> Workload:
    return Workload(KIND_ZIPF, n_r, n_s, seed, theta=theta)


def sparse(n_r: int, n_s: int, fk_share: float = 0.7, seed: int = DEFAULT_SEED) -> Workload:
    return Workload(KIND_SPARSE, n_r, n_s, seed, fk_share=fk_share)


def locskew(n_r: int, n_s: int, seed: int = DEFAULT_SEED) -> Workload:
    """Location skew (Sec. 5.5): R stored in 64 row clusters of ascending key ranges,
    each cluster's keys in random order; S uniform foreign keys."""
    return Workload(KIND_LOCSKEW, n_r, n_s, seed)


def negcorr(n_r: int, n_s: int, seed: int = DEFAULT_SEED) -> Workload:
    """Negatively correlated 80:20 skew (Sec. 5.6): 80 % of R's unique keys in the low
    fifth of the key domain, 80 % of S's foreign keys in the high fifth."""
    return Workload(KIND_NEGCORR, n_r, n_s, seed)


def batch_jobs(n_jobs: int = 256, lo: int = 10 * 1024, hi: int = 20 * M, seed: int = DEFAULT_SEED,
               theta: float = 0.8) -> List[Workload]:
    """Independent joins of uneven sizes: |R_i| log-uniform in [lo, hi], |S_i| = m_i |R_i|
    with m_i uniform in {1, 2, 4, 8, 16}; half the jobs uniform foreign keys, half
    Zipf(theta)."""
    rng = np.random.default_rng([seed & 0xFFFFFFFF, 0xBA7C])
    n_r = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), n_jobs))).astype(np.int64)
    mult = rng.choice(np.array([1, 2, 4, 8, 16]), n_jobs)
    kinds = np.array([KIND_UNIFORM] * (n_jobs // 2) + [KIND_ZIPF] * (n_jobs - n_jobs // 2))
    rng.shuffle(kinds)
    jobs = []
    for i in range(n_jobs):
        nr = int(n_r[i])
        jobs.append(Workload(int(kinds[i]), nr, nr * int(mult[i]), seed=(seed * 1000003 + i) & GEN_NONE,
                             theta=theta))
    return jobs


CONFIGS = {
    # name: (builder, description)
    "plain-1M-4M": lambda seed=DEFAULT_SEED: plain(1 * M, 4 * M, seed),
    "plain-400M-1600M": lambda seed=DEFAULT_SEED: plain(400 * M, 1600 * M, seed),
    "pairs-100M-400M": lambda seed=DEFAULT_SEED: plain(100 * M, 400 * M, seed),
    "plain-25M-100M": lambda seed=DEFAULT_SEED: plain(25 * M, 100 * M, seed),
    "plain-12M-48M": lambda seed=DEFAULT_SEED: plain(12 * M, 48 * M, seed),
    # multiplicities 1 and 16 beside the headline's 4 (role reversal, Sec. 5.4)
    "plain-800M-800M": lambda seed=DEFAULT_SEED: plain(800 * M, 800 * M, seed),
    "plain-200M-3200M": lambda seed=DEFAULT_SEED: plain(200 * M, 3200 * M, seed),
    "plain-283M-2263M": lambda seed=DEFAULT_SEED: plain(283 * M, 2263 * M, seed),  # multiplicity 8
    "zipf0.9-200M-800M": lambda seed=DEFAULT_SEED: zipf(200 * M, 800 * M, 0.9, seed),
    "sparse-1600M-1600M": lambda seed=DEFAULT_SEED: sparse(1600 * M, 1600 * M, 0.7, seed),
    # Sec. 5.6 (multiplicity 4, at a quarter of the paper's 1600M x 6400M)
    "negcorr-400M-1600M": lambda seed=DEFAULT_SEED: negcorr(400 * M, 1600 * M, seed),
    # Sec. 5.5, location skew of the run side (multiplicity 4)
    "locskew-400M-1600M": lambda seed=DEFAULT_SEED: locskew(400 * M, 1600 * M, seed),
}
