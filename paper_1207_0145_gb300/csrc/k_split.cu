// k_split.cu -- phase 2 of MPSM: skew-aware splitters for range-partitioning S.
//
// Sec. 4 computes global partition bounds from both inputs' key distributions:
//  - the run side's distribution comes from its sorted runs (Sec. 4.1: sorted
//    runs give a CDF "en passant"); here the number of R tuples below each fine
//    radix boundary is read off every sorted run by binary search, i.e. the
//    run-side CDF evaluated exactly at the boundaries;
//  - the partitioned side's distribution is a fine B-bit radix histogram
//    (Sec. 4.2), produced by the MODE_FINE pass in k_pass.cu;
//  - splitters group the 2^B fine buckets into at most P contiguous partitions
//    so that the largest split-relevant cost (Sec. 4.3) is minimal.
// The cost of a partition holding n tuples of S and r tuples of R, in units of
// 2^-16 tuples, is n*log2(n) + T*n + r with log2 in Q16 fixed point (integer
// arithmetic only, so the choice of splitters is reproducible bit for bit).
// The equi-height baseline of Sec. 5.6 (Fig. 16b) uses the cost n alone.
// The paper leaves the optimiser open; this one bisects the integer bound C and
// tests feasibility with the left-to-right greedy grouping, whose group count
// after P greedy jumps is found by repeated squaring of the jump function.
#include "mpsm_internal.cuh"
#include "mpsm_launch.h"

namespace mpsm {

namespace {

__device__ __forceinline__ u64 lower_bound_key(const Tuple* a, u64 n, u64 key) {
  u64 lo = 0;
  while (n > 0) {
    const u64 h = n >> 1;
    if (a[lo + h].key < key) {
      lo += h + 1;
      n -= h + 1;
    } else {
      n = h;
    }
  }
  return lo;
}

// Fractional part of log2(1 + i/1024) in Q16 by the bit-by-bit method:
// normalise to [1, 2) in Q31, square 16 times, one fractional bit per squaring.
__device__ __forceinline__ u32 log2_frac_entry(u32 i) {
  u64 x = (u64)(1024u + i) << 21;
  u32 r = 0;
#pragma unroll
  for (int b = 15; b >= 0; --b) {
    x = (x * x) >> 31;
    if (x >= (1ull << 32)) {
      x >>= 1;
      r |= 1u << b;
    }
  }
  return r;
}

// log2(n) in Q16 from n's leading 11 significant bits (0 for n <= 1)
__device__ __forceinline__ u64 log2_q16(u64 n, const u32* frac) {
  if (n <= 1) return 0;
  const u32 k = 63u - (u32)__clzll((long long)n);
  const u32 m = (k >= 10) ? (u32)(n >> (k - 10)) : (u32)(n << (10 - k));
  return ((u64)k << 16) + frac[m - 1024u];
}

// split-relevant cost of n partitioned-side and r run-side tuples; with `height`
// set, the partitioned side's count alone (equi-height partitions, Sec. 5.6)
__device__ __forceinline__ u64 split_cost(u64 n, u64 r, u32 T, const u32* frac, bool height) {
  if (height) return n << 16;
  return n * log2_q16(n, frac) + (((u64)T * n + r) << 16);
}

__device__ __forceinline__ u64 part_cost(const u64* PH, const u64* PG, u32 a, u32 b, u32 T, const u32* frac,
                                         bool height) {
  return split_cost(PH[b] - PH[a], PG[b] - PG[a], T, frac, height);
}

__global__ void k_run_bounds(Job* jobs, u32 njobs, const Run* runs, const Tuple* xr) {
  __shared__ u64 s_mn[8], s_mx[8];
  const u32 job = blockIdx.x;
  if (job >= njobs) return;
  const Job J = jobs[job];
  u64 mn = ~0ull, mx = 0;
  for (u32 j = threadIdx.x; j < J.runs; j += blockDim.x) {
    const Run r = runs[J.run_base + j];
    if (!r.len) continue;
    const u64 a = xr[r.off].key, b = xr[r.off + r.len - 1].key;
    mn = a < mn ? a : mn;
    mx = b > mx ? b : mx;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const u64 a = __shfl_xor_sync(0xffffffffu, mn, d), b = __shfl_xor_sync(0xffffffffu, mx, d);
    mn = a < mn ? a : mn;
    mx = b > mx ? b : mx;
  }
  if (lane_id() == 0) {
    s_mn[warp_id()] = mn;
    s_mx[warp_id()] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (u32 w = 1; w < blockDim.x / 32; ++w) {
      mn = s_mn[w] < mn ? s_mn[w] : mn;
      mx = s_mx[w] > mx ? s_mx[w] : mx;
    }
    Job& O = jobs[job];
    if (J.nR && mn <= mx) {
      O.kmin = mn;
      O.kmax = mx;
      O.has_range = 1;
      const u32 bits = bitlen64(mx - mn);
      O.fine_shift = bits > J.fine_bits ? bits - J.fine_bits : 0u;
      O.nfine = (u32)((mx - mn) >> O.fine_shift) + 1u;
    } else {
      O.kmin = ~0ull;  // empty range: every key is dropped
      O.kmax = 0;
      O.has_range = 0;
      O.fine_shift = 0;
      O.nfine = 0;
    }
    O.parts = 0;
    O.s_kept = 0;
    O.count = 0;
    O.checksum = 0;
  }
}

// rc[f] = number of R tuples with key < kmin + (f << shift), for 0 < f < nfine
__global__ void k_run_cdf(const Job* jobs, u32 njobs, const Run* runs, const Tuple* xr, u64* rc) {
  const u32 job = blockIdx.y;
  const Job J = jobs[job];
  if (J.nfine < 2 || J.runs == 0) return;
  const u64 total = (u64)(J.nfine - 1) * J.runs;
  for (u64 q = (u64)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (u64)gridDim.x * blockDim.x) {
    const u32 f = 1u + (u32)(q / J.runs);
    const u32 j = (u32)(q % J.runs);
    const u64 bound = J.kmin + ((u64)f << J.fine_shift);
    const Run r = runs[J.run_base + j];
    const u64 lb = lower_bound_key(xr + r.off, r.len, bound);
    atomicAdd(&rc[(u64)job * (FINE_MAX + 1) + f], lb);
  }
}

__global__ void __launch_bounds__(1024) k_splitters(Job* jobs, const u64* fine_s, const u64* rc, u64* fine_r, u32* sp,
                                                    u32* part_fstart, u32* err, bool height) {
  constexpr u32 NT = 1024;
  // dynamic shared memory: PH, PG (u64, FINE_MAX + 1 each), frac (u32, 1024), A, B (u16, FINE_MAX + 8 each)
  extern __shared__ __align__(128) unsigned char sm_raw[];
  u64* PH = reinterpret_cast<u64*>(sm_raw);
  u64* PG = PH + (FINE_MAX + 1);
  u32* frac = reinterpret_cast<u32*>(PG + (FINE_MAX + 1));
  u16* A = reinterpret_cast<u16*>(frac + 1024);
  u16* B = A + (FINE_MAX + 8);
  __shared__ u64 s_red[2 * (NT / 32)];
  __shared__ u64 s_warp[NT / 32 + 1];
  __shared__ u64 s_lo;
  __shared__ u64 s_hi;
  __shared__ u32 s_parts;
  const u32 job = blockIdx.x;
  const Job J = jobs[job];
  const u32 nb = J.nfine;
  const u32 tid = threadIdx.x;
  if (nb > FINE_MAX) {
    if (tid == 0) atomicOr(err, (u32)DERR_BOUNDS);
    return;
  }
  if (nb == 0) {
    if (tid == 0) {
      jobs[job].parts = 0;
      part_fstart[J.part_base] = 0;
    }
    return;
  }
  const u32 P = J.parts_req < nb ? J.parts_req : nb;
  const u32 T = J.runs;
  frac[tid] = log2_frac_entry(tid);  // one entry per thread: NT == 1024 entries
  const u64* rcj = rc + (u64)job * (FINE_MAX + 1);
  // per-bucket counts, then prefix sums PH, PG over nb + 1 entries
  for (u32 f = tid; f < nb; f += NT) {
    const u64 r0 = f == 0 ? 0ull : rcj[f];
    const u64 r1 = (f + 1 == nb) ? J.nR : rcj[f + 1];
    PH[f] = fine_s[J.fine_base + f];
    PG[f] = r1 - r0;
    fine_r[J.fine_base + f] = r1 - r0;
  }
  __syncthreads();
  // lower bound of the optimum: the largest single bucket, and the per-bucket
  // costs spread over P partitions (merging buckets never lowers the cost)
  u64 mx = 0, sm = 0;
  for (u32 f = tid; f < nb; f += NT) {
    const u64 c = split_cost(PH[f], PG[f], T, frac, height);
    mx = c > mx ? c : mx;
    sm += c;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const u64 o = __shfl_xor_sync(0xffffffffu, mx, d);
    mx = o > mx ? o : mx;
    sm += __shfl_xor_sync(0xffffffffu, sm, d);
  }
  if (lane_id() == 0) {
    s_red[warp_id()] = mx;
    s_red[NT / 32 + warp_id()] = sm;
  }
  __syncthreads();
  if (tid == 0) {
    u64 m = 0, z = 0;
    for (u32 w = 0; w < NT / 32; ++w) {
      m = s_red[w] > m ? s_red[w] : m;
      z += s_red[NT / 32 + w];
    }
    const u64 mean = (z + P - 1) / P;
    s_lo = m > mean ? m : mean;
  }
  __syncthreads();
  const u64 totH = smem_exclusive_scan<u64, NT, FINE_MAX / NT>(PH, nb, s_warp);
  const u64 totG = smem_exclusive_scan<u64, NT, FINE_MAX / NT>(PG, nb, s_warp);
  if (tid == 0) {
    PH[nb] = totH;
    PG[nb] = totG;
    const u64 h = split_cost(totH, totG, T, frac, height);
    s_hi = h > s_lo ? h : s_lo;
  }
  __syncthreads();
  // bisection on the largest admissible cost C
  for (;;) {
    const u64 lo = s_lo;
    const u64 hi = s_hi;
    const bool last = !(lo < hi);
    const u64 C = last ? lo : lo + (hi - lo) / 2;
    // greedy jump: A[a] = furthest end b with cost(a, b) <= C (>= a+1 since C >= single costs)
    for (u32 a = tid; a < nb; a += NT) {
      u32 l = a + 1, h = nb;
      while (l < h) {
        const u32 m = (l + h + 1) >> 1;
        if (part_cost(PH, PG, a, m, T, frac, height) <= C) l = m; else h = m - 1;
      }
      A[a] = (u16)l;
    }
    if (tid == 0) A[nb] = (u16)nb;
    __syncthreads();
    if (last) break;
    // position after P greedy jumps from bucket 0, by squaring the jump function
    u16* base = A;
    u16* tmp = B;
    u32 pos = 0, k = P;
    for (;;) {
      if (k & 1u) pos = base[pos];
      k >>= 1;
      if (k == 0 || pos == nb) break;
      for (u32 a = tid; a <= nb; a += NT) tmp[a] = base[base[a]];
      __syncthreads();
      u16* t = base;
      base = tmp;
      tmp = t;
    }
    __syncthreads();
    if (tid == 0) {
      if (pos == nb) s_hi = C; else s_lo = C + 1;
    }
    __syncthreads();
  }
  // leftmost greedy grouping at the optimum
  u32* fst = part_fstart + J.part_base;
  if (tid == 0) {
    u32 g = 0, a = 0;
    while (a < nb) {
      if (g >= P_MAX || A[a] <= a) {  // more groups than allowed, or no progress
        atomicOr(err, (u32)DERR_BOUNDS);
        break;
      }
      fst[g++] = a;
      a = A[a];
    }
    fst[g] = nb;
    s_parts = g;
    jobs[job].parts = g;
  }
  __syncthreads();
  const u32 parts = s_parts;
  for (u32 g = tid; g < parts; g += NT)
    for (u32 f = fst[g]; f < fst[g + 1] && f < nb; ++f) sp[J.fine_base + f] = g;
}

// per chunk: partition histogram = sum of the chunk's fine histogram over each partition's buckets
__global__ void k_fold(const Seg* segs, const u32* nseg_ptr, const LSeg* ls_fine, const LSeg* ls_split,
                       const u64* totals, const Job* jobs, const u32* hist_fine, const u32* part_fstart,
                       u32* hist_split) {
  __shared__ u32 s_seg;
  const u64 nch = totals[0];
  const u32 nseg = *nseg_ptr;
  for (u64 c = blockIdx.x; c < nch; c += gridDim.x) {
    if (threadIdx.x == 0) {
      u32 lo = 0, hi = nseg;
      while (hi - lo > 1) {
        const u32 mid = (lo + hi) >> 1;
        if (ls_fine[mid].chunk_base <= c) lo = mid; else hi = mid;
      }
      s_seg = lo;
    }
    __syncthreads();
    const u32 s = s_seg;
    const LSeg Lf = ls_fine[s], Ls = ls_split[s];
    const Job& J = jobs[segs[s].job];
    const u64 ci = c - Lf.chunk_base;
    const u32* hf = hist_fine + Lf.hist_base + ci * Lf.F;
    u32* hs = hist_split + Ls.hist_base + ci * Ls.F;
    for (u32 p = threadIdx.x; p < Ls.F; p += blockDim.x) {
      const u32 fa = part_fstart[J.part_base + p], fb = part_fstart[J.part_base + p + 1];
      u32 sum = 0;
      for (u32 f = fa; f < fb; ++f) sum += hf[f];
      hs[p] = sum;
    }
    __syncthreads();
  }
}

constexpr size_t SMEM_SPLITTERS = 2 * (FINE_MAX + 1) * sizeof(u64) + 1024 * sizeof(u32) + 2 * (FINE_MAX + 8) * sizeof(u16);

}  // namespace

void init_attrs_split() {
  cudaFuncSetAttribute(k_splitters, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_SPLITTERS);
  cudaFuncSetAttribute(k_splitters, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

void launch_run_bounds(Job* jobs, u32 njobs, const Run* runs, const Tuple* xr, cudaStream_t st) {
  k_run_bounds<<<njobs, 256, 0, st>>>(jobs, njobs, runs, xr);
}

void launch_run_cdf(const Job* jobs, u32 njobs, const Run* runs, const Tuple* xr, u64* rc, cudaStream_t st) {
  k_run_cdf<<<dim3(64, njobs), 256, 0, st>>>(jobs, njobs, runs, xr, rc);
}

void launch_splitters(Job* jobs, u32 njobs, const u64* fine_s, const u64* rc, u64* fine_r, u32* sp,
                      u32* part_fstart, u32* err, cudaStream_t st, bool equi_height) {
  k_splitters<<<njobs, 1024, SMEM_SPLITTERS, st>>>(jobs, fine_s, rc, fine_r, sp, part_fstart, err, equi_height);
}

void launch_fold(const Seg* segs, const u32* nseg, const LSeg* ls_fine, const LSeg* ls_split, const u64* totals,
                 const Job* jobs, const u32* hist_fine, const u32* part_fstart, u32* hist_split, cudaStream_t st,
                 int nsm) {
  k_fold<<<nsm * 4, 256, 0, st>>>(segs, nseg, ls_fine, ls_split, totals, jobs, hist_fine, part_fstart, hist_split);
}

}  // namespace mpsm
