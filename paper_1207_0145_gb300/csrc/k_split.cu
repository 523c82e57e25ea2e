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
// 2^-16 tuples, is n*L(n) + 2^16 (T*n + r) with L(n) = floor(2^16 log2 n), the
// exact Q16 logarithm (integer arithmetic only, so the choice of splitters is
// reproducible bit for bit).
// The equi-height baseline of Sec. 5.6 (Fig. 16b) uses the cost n alone.
// The paper leaves the optimiser open; this one bisects the integer bound C and
// tests feasibility with the left-to-right greedy grouping, whose group count
// after P greedy jumps is found by repeated squaring of the jump function; the
// jumps found at earlier bounds bracket the search for each later one.
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

// ---------------------------------------------------------------- the Q16 logarithm
// L(n) = floor(2^16 log2 n) for n >= 2, 0 below.  Sec. 4.3 charges a partition
// of n tuples n log n for its sort; here that term is n * L(n), in integers, so
// the splitters are reproducible bit for bit.  Bit-by-bit method: with n = 2^k x,
// x in [1, 2), log2 n = k + log2 x, and squaring x doubles log2 x, so every
// squaring gives the next fractional bit (1 when the square reaches 2, which is
// then halved).  x is carried as an interval [lo, hi] that holds the true value
// (lo's squares rounded down, hi's up), and a bit is taken only when the squares
// of both ends lie on the same side of 2, so every bit is certain.  Fixed point
// with 62 fraction bits first; a bit it cannot decide (an interval that straddles
// 2, which takes an n whose 2^16 log2 n lies within about 2^-38 of an integer)
// is retried with 126 fraction bits.

// (h:l) >> s rounded down or up, s = 62 or 63, for results below 2^64
__device__ __forceinline__ u64 shr128(u64 h, u64 l, u32 s, bool up) {
  const u64 q = (h << (64u - s)) | (l >> s);
  return q + ((up && (l & ((1ull << s) - 1ull)) != 0ull) ? 1ull : 0ull);
}

// the 256-bit square of the 128-bit number (xh:xl), r[0] lowest
__device__ __forceinline__ void sq256(u64 xh, u64 xl, u64* r) {
  const u64 ll = xl * xl, llh = __umul64hi(xl, xl);
  const u64 hl = xh * xl, hlh = __umul64hi(xh, xl);
  const u64 hh = xh * xh, hhh = __umul64hi(xh, xh);
  // x^2 = hh 2^128 + 2 hl 2^64 + ll, with 2 hl = (c2 : d1 : d0)
  const u64 d0 = hl << 1, d1 = (hlh << 1) | (hl >> 63), c2 = hlh >> 63;
  r[0] = ll;
  r[1] = llh + d0;
  const u64 cy1 = r[1] < d0 ? 1ull : 0ull;
  u64 s2 = hh + d1;
  u64 cy2 = s2 < d1 ? 1ull : 0ull;
  s2 += cy1;
  cy2 += (s2 < cy1) ? 1ull : 0ull;
  r[2] = s2;
  r[3] = hhh + c2 + cy2;
}

// r >> (64 + w) rounded down or up as 128 bits (h:l), w = 62 or 63, r[3] < 2^w
__device__ __forceinline__ void shr256(const u64* r, u32 w, bool up, u64& h, u64& l) {
  l = (r[2] << (64u - w)) | (r[1] >> w);
  h = (r[3] << (64u - w)) | (r[2] >> w);
  if (up && ((r[1] & ((1ull << w) - 1ull)) | r[0]) != 0ull) {
    ++l;
    if (l == 0ull) ++h;
  }
}

// L(n) with 126 fraction bits (n >= 2); ~0 if a bit stays undecided even here
__device__ __noinline__ u64 log2_q16_wide(u64 n) {
  const u32 k = 63u - (u32)__clzll((long long)n);
  const u32 s = 126u - k;  // x = n 2^s in [2^126, 2^127)
  u64 loh = s >= 64u ? n << (s - 64u) : n >> (64u - s);
  u64 lol = s >= 64u ? 0ull : n << s;
  u64 hih = loh, hil = lol;
  u64 res = (u64)k << 16;
  u64 a[4], b[4];
  for (int i = 15; i >= 0; --i) {
    sq256(loh, lol, a);
    sq256(hih, hil, b);
    const bool one = a[3] >= (1ull << 61);  // lo^2 >= 2 (2^253 in these units)
    if (!one && b[3] >= (1ull << 61)) return ~0ull;
    const u32 w = one ? 63u : 62u;          // square, halved when it reached 2
    shr256(a, w, false, loh, lol);
    shr256(b, w, true, hih, hil);
    if (one) res |= 1ull << i;
  }
  return res;
}

// L(n); ~0 only if neither precision decides (not seen for any n tried)
__device__ __forceinline__ u64 log2_q16(u64 n) {
  if (n <= 1) return 0;
  const u32 k = 63u - (u32)__clzll((long long)n);
  u64 lo, hi;
  if (k <= 62u) {
    lo = hi = n << (62u - k);  // exact
  } else {
    lo = n >> 1;
    hi = lo + (n & 1ull);
  }
  u64 res = (u64)k << 16;
  for (int i = 15; i >= 0; --i) {
    const u64 ah = __umul64hi(lo, lo), al = lo * lo;
    const u64 bh = __umul64hi(hi, hi), bl = hi * hi;
    const bool one = ah >= (1ull << 61);  // lo^2 >= 2 (2^125 in Q124)
    if (!one && bh >= (1ull << 61)) return log2_q16_wide(n);
    const u32 s = one ? 63u : 62u;
    lo = shr128(ah, al, s, false);
    hi = shr128(bh, bl, s, true);
    if (one) res |= 1ull << i;
  }
  return res;
}

// split-relevant cost of n partitioned-side and r run-side tuples, in units of
// 2^-16 tuples: n L(n) + (T n + r) 2^16; with `height` set, the partitioned
// side's count alone (equi-height partitions, Sec. 5.6).  *bad is set if L(n)
// stayed undecided.
__device__ __forceinline__ u64 split_cost(u64 n, u64 r, u32 T, bool height, bool& bad) {
  if (height) return n << 16;
  const u64 L = log2_q16(n);
  if (L == ~0ull) bad = true;
  return n * L + (((u64)T * n + r) << 16);
}

// split_cost(n, r) <= C, settled without L(n) unless C lies within a few units of
// the cost.  Bounds on L(n): 2^16 k <= L(n) < 2^16 (k + 1) for k = floor(log2 n), and
// L(n) within 64 of 2^16 log2f(n): CUDA's log2f is within 1 ulp (at most 2^-18 for
// results below 64, i.e. 1/4 unit after the scaling) and float(n) is within 2^-24 of
// n (0.006 units), so 64 units is far more than the error.
__device__ __forceinline__ bool cost_le(u64 n, u64 r, u32 T, u64 C, bool height, bool& bad) {
  if (height) return (n << 16) <= C;
  const u64 base = ((u64)T * n + r) << 16;
  if (n <= 1) return base <= C;
  const u64 k = 63u - (u32)__clzll((long long)n);
  const float lf = log2f((float)n) * 65536.0f;
  u64 llo = lf > 64.0f ? (u64)(lf - 64.0f) : 0ull;
  u64 lhi = (u64)(lf + 64.0f) + 1ull;
  llo = llo > (k << 16) ? llo : (k << 16);
  lhi = lhi < (k << 16) + 65535ull ? lhi : (k << 16) + 65535ull;
  if (base + n * llo > C) return false;
  if (base + n * lhi <= C) return true;
  const u64 L = log2_q16(n);
  if (L == ~0ull) {
    bad = true;
    return false;
  }
  return base + n * L <= C;
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

constexpr u32 KCAND = 2048;  // candidate costs the splitter solve sorts in shared memory (a power of two)

__global__ void __launch_bounds__(1024) k_splitters(Job* jobs, const u64* fine_s, const u64* rc, u64* fine_r, u32* sp,
                                                    u32* part_fstart, u32* err, bool height) {
  constexpr u32 NT = 1024;
  constexpr u32 AW = FINE_MAX + 8;
  // dynamic shared memory: PH, PG (u64, FINE_MAX + 1 each), then five u16 arrays of AW
  // entries: the greedy jumps at the bound being tested, at the largest bound known to be
  // infeasible and at the smallest known to be feasible, and two buffers for squaring
  extern __shared__ __align__(128) unsigned char sm_raw[];
  u64* PH = reinterpret_cast<u64*>(sm_raw);
  u64* PG = PH + (FINE_MAX + 1);
  u16* jarr = reinterpret_cast<u16*>(PG + (FINE_MAX + 1));
  __shared__ u64 s_red[2 * (NT / 32)];
  __shared__ u64 s_warp[NT / 32 + 1];
  __shared__ u64 s_lo;
  __shared__ u64 s_hi;
  __shared__ u32 s_parts;
  __shared__ u32 s_bad;
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
  bool bad = false;
  if (tid == 0) s_bad = 0;
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
    const u64 c = split_cost(PH[f], PG[f], T, height, bad);
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
    const u64 h = split_cost(totH, totG, T, height, bad);
    s_hi = h > s_lo ? h : s_lo;
  }
  // The greedy jump A_C[a] (furthest end b with cost(a, b) <= C) grows with C, so
  // the jumps at the largest bound found infeasible (Alo) and at the smallest found
  // feasible (Ahi) bracket those of every bound the bisection tests later.
  u16* Acur = jarr;
  u16* Alo = jarr + AW;
  u16* Ahi = jarr + 2 * AW;
  u16* B1 = jarr + 3 * AW;
  u16* B2 = jarr + 4 * AW;
  for (u32 a = tid; a < nb; a += NT) {
    Alo[a] = (u16)(a + 1);  // every tested C is at least the largest single-bucket cost
    Ahi[a] = (u16)nb;
  }
  __syncthreads();
  // Bisection on the largest admissible cost C.  Feasibility changes only at costs
  // cost(a, b) of some bucket range, so the optimum is lo itself or the cost of a range
  // b in (Alo[a], Ahi[a]] for some a (the jumps at a cost below lo and at hi).  Once there
  // are fewer than KCAND such ranges, the optimum is the smallest feasible value among
  // lo and their costs: they are sorted and the bisection continues over their indices
  // (candidate mode), with the same feasibility test.
  u64* cand = reinterpret_cast<u64*>(jarr + 5 * AW);  // KCAND
  bool cmode = false;
  u32 ci_lo = 0, ci_hi = 0;
  for (;;) {
    bool last;
    u64 C;
    u32 cmid = 0;
    if (!cmode) {
      const u64 lo = s_lo;
      const u64 hi = s_hi;
      last = !(lo < hi);
      C = last ? lo : lo + (hi - lo) / 2;
    } else {
      last = !(ci_lo < ci_hi);
      cmid = last ? ci_lo : ci_lo + (ci_hi - ci_lo) / 2;
      C = cand[cmid];
    }
    for (u32 a = tid; a < nb; a += NT) {
      u32 l = Alo[a], h = Ahi[a];  // cost(a, l) <= C, and A_C[a] <= h
      const u64 ha = PH[a], ga = PG[a];
      while (l < h) {
        const u32 m = (l + h + 1) >> 1;
        if (cost_le(PH[m] - ha, PG[m] - ga, T, C, height, bad)) l = m; else h = m - 1;
      }
      Acur[a] = (u16)l;
    }
    if (tid == 0) Acur[nb] = (u16)nb;
    __syncthreads();
    if (last) break;
    // position after P greedy jumps from bucket 0, by squaring the jump function
    // (into B1 / B2, so Acur is kept)
    const u16* base = Acur;
    u16* tmp = B1;
    u32 pos = 0, k = P;
    for (;;) {
      if (k & 1u) pos = base[pos];
      k >>= 1;
      if (k == 0 || pos == nb) break;
      for (u32 a = tid; a <= nb; a += NT) tmp[a] = base[base[a]];
      __syncthreads();
      base = tmp;
      tmp = (tmp == B1) ? B2 : B1;
    }
    __syncthreads();
    const bool feasible = pos == nb;
    if (!cmode) {
      if (tid == 0) {
        if (feasible) s_hi = C; else s_lo = C + 1;
      }
    } else if (feasible) {
      ci_hi = cmid;  // every thread keeps the same indices
    } else {
      ci_lo = cmid + 1;
    }
    u16* t = Acur;
    if (feasible) {
      Acur = Ahi;
      Ahi = t;
    } else {
      Acur = Alo;
      Alo = t;
    }
    __syncthreads();
    if (!cmode) {
      // the ranges whose cost lies in the bracket (block-uniform count)
      u64 k = 0;
      for (u32 a = tid; a < nb; a += NT) k += (u64)(Ahi[a] - Alo[a]);
      k = warp_sum(k);
      if (lane_id() == 0) s_red[warp_id()] = k;
      __syncthreads();
      u64 K = 0;
      for (u32 w = 0; w < NT / 32; ++w) K += s_red[w];
      __syncthreads();
      if (K + 1 <= KCAND) {
        if (tid == 0) {
          s_parts = 1;
          cand[0] = s_lo;
        }
        __syncthreads();
        for (u32 a = tid; a < nb; a += NT) {
          const u64 ha = PH[a], ga = PG[a];
          for (u32 b = Alo[a] + 1u; b <= Ahi[a]; ++b) {
            const u32 at = atomicAdd(&s_parts, 1u);
            cand[at] = split_cost(PH[b] - ha, PG[b] - ga, T, height, bad);
          }
        }
        const u32 KC = (u32)K + 1u;
        u32 KP = 1;
        while (KP < KC) KP <<= 1;
        for (u32 i = KC + tid; i < KP; i += NT) cand[i] = ~0ull;
        __syncthreads();
        // bitonic sort of the KP <= KCAND candidates
        for (u32 sz = 2; sz <= KP; sz <<= 1) {
          for (u32 st = sz >> 1; st > 0; st >>= 1) {
            for (u32 i = tid; i < KP; i += NT) {
              const u32 j = i ^ st;
              if (j > i) {
                const bool up = (i & sz) == 0;
                const u64 x = cand[i], y = cand[j];
                if ((x > y) == up) {
                  cand[i] = y;
                  cand[j] = x;
                }
              }
            }
            __syncthreads();
          }
        }
        cmode = true;
        // costs below lo (ranges the first jumps admit without a test) cannot be the
        // optimum; starting at lo keeps every tested cost inside the jumps' bracket
        const u64 lo = s_lo;
        ci_lo = 0;
        u32 m = KC;
        while (m > 0) {
          const u32 h = m >> 1;
          if (cand[ci_lo + h] < lo) {
            ci_lo += h + 1;
            m -= h + 1;
          } else {
            m = h;
          }
        }
        ci_hi = KC - 1u;  // the largest candidate is at least the optimum, so feasible
      }
    }
  }
  if (bad) atomicOr(&s_bad, 1u);
  // leftmost greedy grouping at the optimum
  u32* fst = part_fstart + J.part_base;
  __syncthreads();
  if (tid == 0) {
    if (s_bad) atomicOr(err, (u32)DERR_BOUNDS);  // a logarithm stayed undecided
    u32 g = 0, a = 0;
    while (a < nb) {
      if (g >= P_MAX || Acur[a] <= a) {  // more groups than allowed, or no progress
        atomicOr(err, (u32)DERR_BOUNDS);
        break;
      }
      fst[g++] = a;
      a = Acur[a];
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

// floor(2^16 log2 n[i]) as the splitters compute it (wide: the 126-bit path for every value)
__global__ void k_log2_selftest(const u64* n, u64 count, u64* out, u32 wide) {
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (u64)gridDim.x * blockDim.x) {
    const u64 v = n[i];
    out[i] = v <= 1 ? 0ull : (wide ? log2_q16_wide(v) : log2_q16(v));
  }
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

constexpr size_t SMEM_SPLITTERS = 2 * (FINE_MAX + 1) * sizeof(u64) + 5 * (FINE_MAX + 8) * sizeof(u16) +
                                  KCAND * sizeof(u64);

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

void launch_log2_selftest(const u64* n, u64 count, u64* out, u32 wide, cudaStream_t st, int nsm) {
  if (count) k_log2_selftest<<<nsm * 4, 256, 0, st>>>(n, count, out, wide);
}

void launch_fold(const Seg* segs, const u32* nseg, const LSeg* ls_fine, const LSeg* ls_split, const u64* totals,
                 const Job* jobs, const u32* hist_fine, const u32* part_fstart, u32* hist_split, cudaStream_t st,
                 int nsm) {
  k_fold<<<nsm * 4, 256, 0, st>>>(segs, nseg, ls_fine, ls_split, totals, jobs, hist_fine, part_fstart, hist_split);
}

}  // namespace mpsm
