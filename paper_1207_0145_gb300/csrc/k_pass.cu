// k_pass.cu -- the partitioning machinery shared by phases 1-3 of MPSM.
//
// A pass takes a list of "big" segments (contiguous, key-ordered slices too large
// to sort in one block's shared memory) and splits each into F key-ordered
// buckets, the paper's radix clustering (Sec. 3.2.1):
//   k_level_plan : per segment, the bucket function and the chunking (one chunk
//                  = one "worker" W_i of the paper, a contiguous piece of input)
//   k_hist       : per chunk, the histogram h_i over the F buckets (+ exact
//                  per-bucket key min/max)
//   k_scan       : per segment, the prefix sums ps_i[b] = start of bucket b +
//                  sum over chunks k < i of h_k[b] (the ps equation under Fig. 6),
//                  and the children segments for the next pass
//   k_scatter    : per chunk, every tuple copied to ps_i[bucket]++ (Sec. 4.3) --
//                  synchronisation-free, since each chunk owns its ranges
// The same kernels run three bucket functions: MODE_RADIX (top bits of key -
// segment min, or F equal-width key ranges before the fused sort-and-join; the sort
// passes of phases 1 and 3), MODE_FINE (the fine
// B-bit histogram of S over R's key range, Sec. 4.2) and MODE_SPLIT (fine bucket
// -> partition through the splitter vector sp, Sec. 4.3).
// Segments that fit NMAX tuples are finished by k_seg_sort: one block loads the
// segment with a bulk async copy (TMA) into shared memory and radix-sorts it
// there (first digit by an unstable counting pass, further digits by stable
// warp-ballot ranking), then writes it out in order.
#include <algorithm>
#include <mutex>

#include "mpsm.h"
#include "mpsm_internal.cuh"
#include "learn.cuh"
#include "mpsm_launch.h"

namespace mpsm {

namespace {

constexpr u32 NT_PASS = 512;
constexpr u32 SCAN_UNROLL = 8;  // histogram rows read per group in k_scan
// scatter geometry (measured): the first radix pass over runs or partitions (fan-out
// up to 2048) and the range-partition scatter run one 1024-thread block per SM on
// two 5120-tuple buffers, so the next tile loads while the current one is ranked and
// written (long write runs per bucket and no idle SM while a lone block waits for its
// tile); the later radix passes over smaller segments and the learned partitioning
// are fastest with 4096-tuple tiles and two 512-thread blocks
constexpr u32 RX_TILE = 5120, RX_NT = 1024, RX_MINB = 1, RX_STAGES = 2;
constexpr u32 SP_TILE = 4096, SP_NT = 512, SP_MINB = 2;
constexpr u32 NT_SORT = 512;
constexpr u32 NW_SORT = NT_SORT / 32;

// floor(a * 2^64 / d) for a < d, by binary long division (the remainder stays below d)
__device__ __forceinline__ u64 frac64(u64 a, u64 d) {
  u64 rem = a, q = 0;
  for (int i = 0; i < 64; ++i) {
    const bool carry = (rem >> 63) != 0;  // 2 rem >= 2^64 > d
    rem <<= 1;
    q <<= 1;
    if (carry || rem >= d) {
      rem -= d;
      q |= 1ull;
    }
  }
  return q;
}

// MODE_RADIX bucket of a key before the clamp to F - 1 (see k_level_plan)
__device__ __forceinline__ u64 radix_bucket(const LSeg& L, u64 key) {
  const u64 d = key < L.lo ? 0ull : key - L.lo;
  return L.mul ? __umul64hi(d, L.mul) : d >> L.shift;
}

// smallest key offset (key - lo) of MODE_RADIX bucket b (0 < b < F): b << shift, or
// with mul the smallest d with mulhi(d, mul) >= b, i.e. ceil(b 2^64 / mul)
__device__ __forceinline__ u64 bucket_start(const LSeg& L, u32 b) {
  if (!L.mul) return (u64)b << L.shift;
  const unsigned __int128 num = ((unsigned __int128)b) << 64;
  u64 q = (u64)(num / L.mul);
  if ((unsigned __int128)q * L.mul < num) ++q;
  return q;
}

__device__ __forceinline__ u64 ld_key_stream(const Tuple* p) {
  return (u64)__ldcs(reinterpret_cast<const long long*>(&p->key));
}

__device__ __forceinline__ void emit(Seg* out, u32* cnt, u32 cap, const Seg& s, u32* err) {
  const u32 i = atomicAdd(cnt, 1u);
  if (i < cap) out[i] = s; else atomicOr(err, (u32)DERR_SEG_OVERFLOW);
}

// last s in [0, n) with ls[s].chunk_base <= c (ls[0].chunk_base is 0): a 32-way search
// by one whole warp, so a chunk's segment costs about log32(n) dependent loads
__device__ __forceinline__ u32 find_seg_warp(const LSeg* ls, u32 n, u64 c) {
  const u32 lane = lane_id();
  u32 lo = 0, len = n;  // the answer lies in [lo, lo + len), and ls[lo].chunk_base <= c
  while (len > 1) {
    const u32 step = (len + 31u) / 32u;
    const u32 idx = lo + lane * step;
    const bool ok = lane * step < len && ls[idx].chunk_base <= c;
    const u32 m = __ballot_sync(0xffffffffu, ok);  // lane 0 always holds
    const u32 k = 31u - (u32)__clz(m);
    const u32 end = lo + len;
    lo += k * step;
    len = end - lo < step ? end - lo : step;
  }
  return lo;
}

// ---------------------------------------------------------------- bounds by sampling
__global__ void k_sample_bounds(Seg* segs, const u32* nseg_ptr, Bufs bufs, const Job* jobs) {
  const u32 n = *nseg_ptr;
  const u32 lane = lane_id();
  const u32 gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u32 nw = (gridDim.x * blockDim.x) >> 5;
  for (u32 s = gw; s < n; s += nw) {
    const Seg sg = segs[s];
    const Tuple* src = seg_src(bufs, jobs, sg.flags & 7u, sg.job, sg.off);
    u64 mn = ~0ull, mx = 0;
    for (u32 i = lane; i < 1024; i += 32) {
      const u64 p = (sg.len - 1) * (u64)i / 1023ull;
      const u64 k = src[p].key;
      mn = k < mn ? k : mn;
      mx = k > mx ? k : mx;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      const u64 a = __shfl_xor_sync(0xffffffffu, mn, d), b = __shfl_xor_sync(0xffffffffu, mx, d);
      mn = a < mn ? a : mn;
      mx = b > mx ? b : mx;
    }
    // 1024 evenly spaced samples of uniform keys miss an extreme by more than range/64
    // with probability about e^-16; widen by that much so the edge buckets, which take
    // every key beyond the bounds, stay as small as the others
    const u64 pad = (mx - mn) >> 6;
    mn = mn > pad ? mn - pad : 0ull;
    mx = (~0ull - mx) > pad ? mx + pad : ~0ull;
    if (lane == 0) {
      segs[s].kmin = mn;
      segs[s].kmax = mx;
    }
  }
}

// ---------------------------------------------------------------- level plan
__global__ void __launch_bounds__(1024) k_level_plan(const Seg* segs, u32* nseg_ptr, u32 seg_cap, LSeg* ls,
                                                     u64* totals, u32 mode, u64 chunk, u32 radix_bits, u64 fill,
                                                     const Job* jobs, u64 hist_cap, u64 bucket_cap, u32* err,
                                                     LearnCtx lc) {
  __shared__ u64 s_warp[33];
  __shared__ u64 carry[3];
  u32 n = *nseg_ptr;
  if (n > seg_cap) n = seg_cap;
  __syncthreads();
  if (threadIdx.x == 0) {
    *nseg_ptr = n;
    carry[0] = carry[1] = carry[2] = 0;
  }
  __syncthreads();
  const u32 fmax = 1u << radix_bits;
  for (u32 base = 0; base < n; base += 1024) {
    const u32 i = base + threadIdx.x;
    u64 nch = 0, nh = 0, nb = 0;
    LSeg L{};
    if (i < n) {
      const Seg s = segs[i];
      u32 F, shift;
      u64 lo;
      if (mode == MODE_RADIX) {
        const u64 range = s.kmax - s.kmin;
        shift = 0;
        if (fill) {
          // F buckets of equal key width over [kmin, kmax], F chosen so that a bucket of
          // uniform keys holds `fill` tuples and its child fits the fused kernel's tile
          // in one piece.  bucket = floor((key - kmin) * F / (range + 1)), computed as the
          // high word of (key - kmin) * mul, mul = floor(2^64 F / (range + 1)), which stays
          // below F and is monotone in the key.
          const u64 want = (s.len + fill - 1) / fill;
          F = want < F_MIN ? F_MIN : (want > fmax ? fmax : (u32)want);
          if (range >= (u64)F) L.mul = range == ~0ull ? (u64)F : frac64(F, range + 1u);
        } else {
          // top bits of key - kmin: the smallest power of two >= len / N_LEAF buckets
          // (at most fmax), of which the key range may fill only a part
          const u64 want = (s.len + N_LEAF - 1) / N_LEAF;
          u32 f = F_MIN;
          while (f < want && f < fmax) f <<= 1;
          const u32 d = 31u - (u32)__clz(f);
          const u32 bits = bitlen64(range);
          shift = bits > d ? bits - d : 0u;
          F = (u32)(range >> shift) + 1u;
        }
        // few distinct key values in many tuples (a hot key among few others): one
        // bucket per value, so every child is constant or small after this pass; at
        // most one bucket per 64 tuples keeps the histogram and bucket arrays in bounds
        if (range < (u64)F || (range < (u64)fmax && range + 1u <= s.len / 64u)) {
          shift = 0;
          L.mul = 0;
          F = (u32)range + 1u;
        }
        lo = s.kmin;
      } else if (mode == MODE_RLEARN) {
        // the job's learned bucket function: lo and shift give the cell of a key
        const RunLearn& RL = lc.rl[s.job];
        lo = RL.lo;
        shift = RL.shift;
        F = RL.F;
      } else {
        const Job& J = jobs[s.job];
        lo = J.kmin;
        shift = J.fine_shift;
        F = (mode == MODE_FINE) ? J.nfine : J.parts;
      }
      nch = F ? (s.len + chunk - 1) / chunk : 0;
      nh = nch * F;
      nb = F;
      L.lo = lo;
      L.shift = shift;
      L.F = F;
      L.nchunks = (u32)nch;
      // dense keys (at most 64 key values per tuple): a bucket's keys fill its key range
      // closely, so that range serves as the child's bounds, and the histogram keeps
      // exact extremes only for the two edge buckets, which take every key beyond a
      // sampled range
      L.nominal = (mode == MODE_RADIX && (s.kmax - s.kmin) / 64u <= s.len) ? 1u : 0u;
      L.bucket_base = (mode == MODE_FINE) ? jobs[s.job].fine_base : 0ull;
    }
    u64 t0, t1, t2;
    const u64 p0 = block_exclusive_scan<u64, 1024>(nch, &t0, s_warp);
    const u64 p1 = block_exclusive_scan<u64, 1024>(nh, &t1, s_warp);
    const u64 p2 = block_exclusive_scan<u64, 1024>(nb, &t2, s_warp);
    if (i < n) {
      L.chunk_base = carry[0] + p0;
      L.hist_base = carry[1] + p1;
      if (mode != MODE_FINE) L.bucket_base = carry[2] + p2;  // fine buckets sit at the job's fixed slot
      ls[i] = L;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      carry[0] += t0;
      carry[1] += t1;
      carry[2] += t2;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (carry[1] > hist_cap || carry[2] > bucket_cap) {
      atomicOr(err, (u32)DERR_HIST_OVERFLOW);
      carry[0] = carry[1] = carry[2] = 0;
      *nseg_ptr = 0;
    }
    totals[0] = carry[0];
    totals[1] = carry[1];
    totals[2] = carry[2];
  }
}

__global__ void k_init_buckets(u64* bmin, u64* bmax, u64* btot, const u64* totals) {
  const u64 n = totals[2];
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
    bmin[i] = ~0ull;
    bmax[i] = 0;
    if (btot) btot[i] = 0;
  }
}

// ---------------------------------------------------------------- histograms
template <u32 MODE, u32 FCAP>
__global__ void __launch_bounds__(NT_PASS) k_hist(const Seg* segs, const u32* nseg_ptr, const LSeg* ls,
                                                  const u64* totals, u64 chunk, Bufs bufs, const Job* jobs,
                                                  u32 src_where, u32* hist, u64* bmin, u64* bmax, u64* btot,
                                                  LearnCtx lc) {
  extern __shared__ __align__(128) unsigned char sm_raw[];
  u64* smin = reinterpret_cast<u64*>(sm_raw);
  u64* smax = smin + FCAP;
  u32* scnt = reinterpret_cast<u32*>(smax + FCAP);
  u32* scell = scnt + FCAP;                              // MODE_LEARN: fine-cell table (FINE_MAX)
  u64* sbnd = reinterpret_cast<u64*>(scell + FINE_MAX);  // MODE_LEARN: partition boundaries (P_MAX)
  u32* srank = reinterpret_cast<u32*>(sbnd + P_MAX);     // MODE_LEARN: their sample ranks (2 P_MAX)
  __shared__ u32 s_seg;
  const u64 nch = totals[0];
  const u32 nseg = *nseg_ptr;
  for (u64 c = blockIdx.x; c < nch; c += gridDim.x) {
    if (threadIdx.x < 32) {
      const u32 sg = find_seg_warp(ls, nseg, c);
      if (threadIdx.x == 0) s_seg = sg;
    }
    __syncthreads();
    const LSeg L = ls[s_seg];
    const Seg S = segs[s_seg];
    const u32 F = L.F;
    for (u32 b = threadIdx.x; b < F; b += NT_PASS) {
      scnt[b] = 0;
      smin[b] = ~0ull;
      smax[b] = 0;
    }
    __syncthreads();
    const u64 ci = c - L.chunk_base;
    const u64 a = ci * chunk;
    const u64 e = (a + chunk < S.len) ? a + chunk : S.len;
    const Tuple* src = seg_src(bufs, jobs, src_where, S.job, S.off);
    u64 kmin = 0, kmax = ~0ull;
    if (MODE == MODE_FINE || MODE == MODE_LEARN) {
      kmin = jobs[S.job].kmin;
      kmax = jobs[S.job].kmax;
    }
    const u64 row0 = S.off - jobs[S.job].s_base;  // MODE_LEARN: row of the tuple in the job's S
    u32 probes = 0, keys = 0;
    u32 fit_n = 0;
    RunLearn RL{};
    // learned partitions of a dense job (at most 64 key values per S tuple) take their
    // boundaries as bounds: only the counts are needed here.  Likewise the interior fine
    // buckets of a dense job: a partition's bounds then come from its buckets' key ranges,
    // and only the two edge buckets keep exact extremes
    const bool ldense = MODE == MODE_LEARN && (kmax - kmin) / 64u <= jobs[S.job].nS;
    const bool fdense = MODE == MODE_FINE && (kmax - kmin) / 64u <= jobs[S.job].nS;
    if (MODE == MODE_LEARN) {
      const Job& J = jobs[S.job];
      for (u32 f = threadIdx.x; f < J.nfine; f += NT_PASS) scell[f] = lc.cell[J.fine_base + f];
      for (u32 q = threadIdx.x; q + 1u < F; q += NT_PASS) {
        sbnd[q] = lc.bnd[(u64)S.job * P_MAX + q];
        srank[2 * q] = lc.brank[(u64)S.job * 2 * P_MAX + 2 * q];
        srank[2 * q + 1] = lc.brank[(u64)S.job * 2 * P_MAX + 2 * q + 1];
      }
      fit_n = lc.models[2 * S.job].fit_n;
      __syncthreads();
    }
    if (MODE == MODE_RLEARN) {
      RL = lc.rl[S.job];
      for (u32 f = threadIdx.x; f < RL.ncell; f += NT_PASS) scell[f] = lc.rcell[(u64)S.job * FINE_MAX + f];
      for (u32 q = threadIdx.x; q + 1u < F; q += NT_PASS) sbnd[q] = lc.rbnd[(u64)S.job * P_MAX + q];
      __syncthreads();
    }
    for (u64 t0 = a + threadIdx.x; t0 < e; t0 += NT_PASS * 4) {
      u64 k[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const u64 t = t0 + (u64)i * NT_PASS;
        k[i] = t < e ? ld_key_stream(src + t) : 0;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const u64 t = t0 + (u64)i * NT_PASS;
        if (t >= e) continue;
        u32 b;
        if (MODE == MODE_RADIX) {
          const u64 d = radix_bucket(L, k[i]);
          b = d >= F ? F - 1u : (u32)d;
        } else if (MODE == MODE_LEARN) {
          if (k[i] < kmin || k[i] > kmax) continue;
          b = learned_cell_part(scell[(k[i] - kmin) >> L.shift], sbnd, srank, F, fit_n, k[i], row0 + t, lc.seed,
                                probes);
          ++keys;
        } else if (MODE == MODE_RLEARN) {
          b = run_learn_bucket(scell[run_learn_cell(RL, k[i])], sbnd, k[i]);
          b = b < F ? b : F - 1u;
        } else {
          if (k[i] < kmin || k[i] > kmax) continue;
          b = (u32)((k[i] - kmin) >> L.shift);
        }
        atomicAdd(&scnt[b], 1u);
        if (MODE == MODE_RADIX && L.nominal && b - 1u < F - 2u) continue;  // an interior bucket of a dense level
        if (fdense && b - 1u < F - 2u) continue;                            // an interior fine bucket of a dense job
        if (ldense) continue;
        atomicMin(&smin[b], k[i]);
        atomicMax(&smax[b], k[i]);
      }
    }
    if (MODE == MODE_LEARN && lc.stat) {
      const u32 wp = warp_sum(probes), wk = warp_sum(keys);
      if (lane_id() == 0 && wk) {
        atomicAdd(&lc.stat[0], (u64)wp);
        atomicAdd(&lc.stat[1], (u64)wk);
      }
      probes = keys = 0;
    }
    __syncthreads();
    u32* hrow = hist + L.hist_base + ci * F;
    for (u32 b = threadIdx.x; b < F; b += NT_PASS) {
      const u32 cnt = scnt[b];
      hrow[b] = cnt;
      if (cnt && !ldense && !(MODE == MODE_RADIX && L.nominal && b - 1u < F - 2u)) {
        if (!(fdense && b - 1u < F - 2u)) {
          atomicMin(&bmin[L.bucket_base + b], smin[b]);
          atomicMax(&bmax[L.bucket_base + b], smax[b]);
        }
        if (btot) atomicAdd(&btot[L.bucket_base + b], (u64)cnt);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- prefix sums + children
template <u32 MODE>
__global__ void __launch_bounds__(NT_PASS) k_scan(const Seg* segs, const u32* nseg_ptr, const LSeg* ls, u32* hist,
                                                  const u64* bmin, const u64* bmax, const u32* part_fstart,
                                                  Seg* big_out, u32* big_cnt, u32 big_cap, Seg* fin_out,
                                                  u32* fin_cnt, u32 fin_cap, u32 dst_where, u32 final_where,
                                                  Job* jobs, u64* part_off, u32* err, const u64* lbnd) {
  extern __shared__ __align__(128) unsigned char sm_raw[];
  u64* start = reinterpret_cast<u64*>(sm_raw);  // F_MAX + 1
  u64* bkmin = start + (F_MAX + 1);             // F_MAX
  u64* bkmax = bkmin + F_MAX;                   // F_MAX
  __shared__ u64 s_warp[NT_PASS / 32 + 1];
  const u32 nseg = *nseg_ptr;
  constexpr u64 HALF = NMAX / 4;  // packed groups stay <= NMAX/2 (the two-blocks-per-SM sort class)
  for (u32 s = blockIdx.x; s < nseg; s += gridDim.x) {
    const LSeg L = ls[s];
    const Seg S = segs[s];
    const u32 F = L.F;
    const u64 C = L.nchunks;
    u32* h = hist + L.hist_base;
    const Job J = jobs[S.job];
    for (u32 b = threadIdx.x; b < F; b += NT_PASS) {
      // the bucket's total over the chunks; its per-chunk offsets are written below,
      // once the bucket's start is known (loads issued in groups, not one per round trip)
      u64 run = 0, c = 0;
      for (; c + SCAN_UNROLL <= C; c += SCAN_UNROLL) {
        u32 v[SCAN_UNROLL];
#pragma unroll
        for (u32 q = 0; q < SCAN_UNROLL; ++q) v[q] = h[(c + q) * F + b];
#pragma unroll
        for (u32 q = 0; q < SCAN_UNROLL; ++q) run += v[q];
      }
      for (; c < C; ++c) run += h[c * F + b];
      start[b] = run;
      if (MODE == MODE_SPLIT) {
        const u32 fa = part_fstart[J.part_base + b], fb = part_fstart[J.part_base + b + 1];
        // a dense job's interior fine buckets contribute their key ranges (the fine
        // histogram kept exact extremes only for the edge buckets, as k_hist says)
        const bool dense = (J.kmax - J.kmin) / 64u <= J.nS;
        u64 mn = ~0ull, mx = 0;
        for (u32 f = fa; f < fb; ++f) {
          u64 a = bmin[J.fine_base + f], z = bmax[J.fine_base + f];
          if (dense && f - 1u < J.nfine - 2u) {
            a = J.kmin + ((u64)f << J.fine_shift);
            z = J.kmin + ((u64)(f + 1u) << J.fine_shift) - 1ull;
          }
          mn = a < mn ? a : mn;
          mx = z > mx ? z : mx;
        }
        bkmin[b] = mn;
        bkmax[b] = mx;
      } else if (MODE == MODE_LEARN && lbnd && (J.kmax - J.kmin) / 64u <= J.nS) {
        // a dense job's learned partition b holds keys in [bnd[b - 1], bnd[b]] (a hot key
        // equal to boundaries is spread over the partitions it bounds)
        const u64* bj = lbnd + (u64)S.job * P_MAX;
        bkmin[b] = b == 0 ? J.kmin : bj[b - 1];
        bkmax[b] = b + 1 == F ? J.kmax : bj[b];
      } else if (MODE == MODE_RADIX && L.nominal && b - 1u < F - 2u) {
        bkmin[b] = L.lo + bucket_start(L, b);
        bkmax[b] = L.lo + bucket_start(L, b + 1u) - 1ull;
      } else {
        bkmin[b] = bmin[L.bucket_base + b];
        bkmax[b] = bmax[L.bucket_base + b];
      }
    }
    __syncthreads();
    const u64 total = smem_exclusive_scan<u64, NT_PASS, F_MAX / NT_PASS>(start, F, s_warp);
    if (threadIdx.x == 0) start[F] = total;
    __syncthreads();
    // ps_i[b] = start of bucket b + the counts of chunks k < i (u32: offsets within the segment)
    for (u32 b = threadIdx.x; b < F; b += NT_PASS) {
      u32 run = (u32)start[b];
      u64 c = 0;
      for (; c + SCAN_UNROLL <= C; c += SCAN_UNROLL) {
        u32 v[SCAN_UNROLL];
#pragma unroll
        for (u32 q = 0; q < SCAN_UNROLL; ++q) v[q] = h[(c + q) * F + b];
#pragma unroll
        for (u32 q = 0; q < SCAN_UNROLL; ++q) {
          h[(c + q) * F + b] = run;
          run += v[q];
        }
      }
      for (; c < C; ++c) {
        const u32 v = h[c * F + b];
        h[c * F + b] = run;
        run += v;
      }
    }
    if (MODE == MODE_SPLIT || MODE == MODE_LEARN) {
      for (u32 b = threadIdx.x; b <= F; b += NT_PASS) part_off[J.part_base + b] = start[b];
      if (threadIdx.x == 0) jobs[S.job].s_kept = total;
    }
    // children: buckets of at most NMAX/4 tuples whose starts share a NMAX/4 window
    // are packed into one final segment (<= NMAX/2); larger ones stand alone.
    for (u32 b = threadIdx.x; b < F; b += NT_PASS) {
      const u64 st = start[b], len = start[b + 1] - st;
      const bool pk = len <= HALF;
      const u64 grp = st / HALF;
      if (pk) {
        if (b > 0 && (start[b] - start[b - 1]) <= HALF && start[b - 1] / HALF == grp) continue;  // not a leader
        u64 end = start[b + 1], mn = bkmin[b], mx = bkmax[b];
        for (u32 e = b + 1; e < F; ++e) {
          const u64 le = start[e + 1] - start[e];
          if (le > HALF || start[e] / HALF != grp) break;
          end = start[e + 1];
          if (le) {
            mn = bkmin[e] < mn ? bkmin[e] : mn;
            mx = bkmax[e] > mx ? bkmax[e] : mx;
          }
        }
        const u64 glen = end - st;
        if (glen == 0) continue;
        if (mn == mx && dst_where == final_where) continue;  // constant keys already in place
        Seg c{S.off + st, glen, mn, mx, S.job, dst_where | SEG_EXACT};
        emit(fin_out, fin_cnt, fin_cap, c, err);
      } else {
        const u64 mn = bkmin[b], mx = bkmax[b];
        if (len > NMAX && mn < mx) {
          Seg c{S.off + st, len, mn, mx, S.job, dst_where | SEG_EXACT};
          emit(big_out, big_cnt, big_cap, c, err);
        } else if (mn == mx) {
          if (dst_where == final_where) continue;
          for (u64 p = 0; p < len; p += NMAX) {
            const u64 l = (len - p < NMAX) ? len - p : NMAX;
            Seg c{S.off + st + p, l, mn, mx, S.job, dst_where | SEG_EXACT};
            emit(fin_out, fin_cnt, fin_cap, c, err);
          }
        } else {
          Seg c{S.off + st, len, mn, mx, S.job, dst_where | SEG_EXACT};
          emit(fin_out, fin_cnt, fin_cap, c, err);
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- scatter
// Per chunk (worker): tiles of SC_TILE tuples arrive by bulk async copy into
// shared memory (with two buffers the next tile's copy overlaps this tile's work;
// with one, two blocks per SM overlap each other's).  Each tuple gets
// (bucket, rank) from a shared-memory counter; an exclusive scan gives the
// tile's bucket starts; a permutation index orders the tile by bucket so the
// write-out stores runs of consecutive destinations (coalesced 16-byte stores).
// Each thread owns F_MAX / NT_SC buckets in the scan and keeps their write
// offsets in registers, so one pass over the counters per tile scans them,
// publishes each bucket's offset and clears the counts.
template <u32 MODE, u32 SC_TILE, u32 NT_SC, u32 SC_MINB, u32 STAGES, u32 LPCAP = P_MAX>
__global__ void __launch_bounds__(NT_SC, SC_MINB) k_scatter(const Seg* segs, const u32* nseg_ptr, const LSeg* ls,
                                                        const u64* totals, u64 chunk, Bufs bufs, const Job* jobs,
                                                        u32 src_where, u32 dst_where, const u32* hist, const u32* sp,
                                                        u32* err, LearnCtx lc) {
  static_assert(STAGES == 1 || STAGES == 2, "one or two tile buffers");
  constexpr u32 IT = SC_TILE / NT_SC;
  constexpr u32 DROP = 0xFFFFFFFFu;
  extern __shared__ __align__(128) unsigned char sm_raw[];
  Tuple* stages = reinterpret_cast<Tuple*>(sm_raw);                // STAGES x SC_TILE
  u32* hcnt = reinterpret_cast<u32*>(stages + STAGES * SC_TILE);   // F_MAX
  u32* hb = hcnt + F_MAX;                                          // F_MAX
  u32* gb = hb + F_MAX;                                            // F_MAX
  u16* sidx = reinterpret_cast<u16*>(gb + F_MAX);                  // SC_TILE
  u16* sb = sidx + SC_TILE;                                        // SC_TILE
  // MODE_LEARN keeps the fine-cell table as u32 entries, or -- with LPCAP < P_MAX, for at
  // most LPCAP partitions -- as u16 (start partition, LCELL_SPLIT and LCELL_HOT in bits 15
  // and 14) with the end partition of each cut cell in sphi[start] (cut cells start at
  // different partitions)
  constexpr bool LCOMPACT = LPCAP < P_MAX;
  u16* spl = sb + SC_TILE;                                         // FINE_MAX u16 (MODE_SPLIT) or
  u32* spl32 = reinterpret_cast<u32*>(spl);                        //   the MODE_LEARN cell table
  u64* sbnd = reinterpret_cast<u64*>(LCOMPACT ? (void*)(spl + FINE_MAX) : (void*)(spl32 + FINE_MAX));  // LPCAP
  u32* srank = reinterpret_cast<u32*>(sbnd + LPCAP);               // 2 LPCAP (MODE_LEARN)
  u16* sphi = reinterpret_cast<u16*>(srank + 2 * LPCAP);           // LPCAP (compact MODE_LEARN)
  __shared__ __align__(8) u64 mbar[STAGES];
  __shared__ u32 s_seg;
  __shared__ u32 s_warp[NT_SC / 32 + 1];
  const u32 tid = threadIdx.x;
  if (tid == 0)
    for (u32 q = 0; q < STAGES; ++q) mbar_init(&mbar[q], 1);
  __syncthreads();
  u32 phases = 0;  // bit q: the parity buffer q's barrier completes next
  const u64 nch = totals[0];
  const u32 nseg = *nseg_ptr;
  Tuple* dbase = dst_where == W_XR ? bufs.xr : (dst_where == W_XS ? bufs.xs : bufs.y);
  for (u64 c = blockIdx.x; c < nch; c += gridDim.x) {
    if (tid < 32) {
      const u32 sg = find_seg_warp(ls, nseg, c);
      if (tid == 0) s_seg = sg;
    }
    __syncthreads();
    const LSeg L = ls[s_seg];
    const Seg S = segs[s_seg];
    const u32 F = L.F;
    const u64 ci = c - L.chunk_base;
    const u32* orow = hist + L.hist_base + ci * F;
    constexpr u32 PER = F_MAX / NT_SC;
    u32 curv[PER];  // write offset (within the segment) of owned bucket tid * PER + i
#pragma unroll
    for (u32 i = 0; i < PER; ++i) {
      const u32 b = tid * PER + i;
      curv[i] = b < F ? orow[b] : 0u;
    }
    for (u32 b = tid; b < F; b += NT_SC) hcnt[b] = 0;
    u64 kmin = 0, kmax = ~0ull;
    if (MODE == MODE_SPLIT || MODE == MODE_LEARN) {
      const Job& J = jobs[S.job];
      kmin = J.kmin;
      kmax = J.kmax;
      if (MODE == MODE_SPLIT) {
        for (u32 f = tid; f < J.nfine; f += NT_SC) spl[f] = (u16)sp[J.fine_base + f];
      } else if (LCOMPACT) {
        for (u32 f = tid; f < J.nfine; f += NT_SC) {
          const u32 e = lc.cell[J.fine_base + f];
          spl[f] = (u16)((e & 0x3FFFu) | ((e & LCELL_SPLIT) ? 0x8000u : 0u) | ((e & LCELL_HOT) ? 0x4000u : 0u));
          if (e & LCELL_SPLIT) sphi[e & 0x3FFFu] = (u16)((e >> 16) & 0x3FFFu);
        }
      } else {
        for (u32 f = tid; f < J.nfine; f += NT_SC) spl32[f] = lc.cell[J.fine_base + f];
      }
    }
    u32 fit_n = 0;
    if (MODE == MODE_LEARN) {
      for (u32 q = tid; q + 1u < F; q += NT_SC) {
        sbnd[q] = lc.bnd[(u64)S.job * P_MAX + q];
        srank[2 * q] = lc.brank[(u64)S.job * 2 * P_MAX + 2 * q];
        srank[2 * q + 1] = lc.brank[(u64)S.job * 2 * P_MAX + 2 * q + 1];
      }
      fit_n = lc.models[2 * S.job].fit_n;
    }
    RunLearn RL{};
    if (MODE == MODE_RLEARN) {  // the job's learned run bucket function (k_hist reads the same tables)
      RL = lc.rl[S.job];
      for (u32 f = tid; f < RL.ncell; f += NT_SC) spl32[f] = lc.rcell[(u64)S.job * FINE_MAX + f];
      for (u32 q = tid; q + 1u < F; q += NT_SC) sbnd[q] = lc.rbnd[(u64)S.job * P_MAX + q];
    }
    const u64 row0 = S.off - jobs[S.job].s_base;  // MODE_LEARN: row of the segment's first tuple in the job's S
    u32 probes = 0;
    const u64 a = ci * chunk;
    const u64 e = (a + chunk < S.len) ? a + chunk : S.len;
    const Tuple* src = seg_src(bufs, jobs, src_where, S.job, S.off);
    Tuple* dst = dbase + S.off;
    const u32 ntile = (u32)((e - a + SC_TILE - 1) / SC_TILE);
    auto tile_len = [&](u32 k) {
      const u64 t0 = a + (u64)k * SC_TILE;
      return (u32)((e - t0) < SC_TILE ? (e - t0) : SC_TILE);
    };
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    // with two buffers, tile k + 1 of the chunk loads while tile k is ranked and written
    if (STAGES == 2 && tid == 0 && ntile)
      tma_load_1d(stages, src + a, tile_len(0) * (u32)sizeof(Tuple), &mbar[0]);
    for (u32 k = 0; k < ntile; ++k) {
      const u64 t0 = a + (u64)k * SC_TILE;
      const u32 n = tile_len(k);
      const u32 q = STAGES == 2 ? (k & 1u) : 0u;
      if (STAGES == 1 && tid == 0) tma_load_1d(stages, src + t0, n * (u32)sizeof(Tuple), &mbar[0]);
      const bool ok = mbar_wait(&mbar[q], (phases >> q) & 1u, SPIN_LIMIT);
      phases ^= 1u << q;
      if (!__syncthreads_and(ok)) {
        if (tid == 0) atomicOr(err, (u32)DERR_TMA_TIMEOUT);
        return;
      }
      // the other buffer's last readers (tile k - 1) passed their fence and this barrier
      if (STAGES == 2 && tid == 0 && k + 1 < ntile)
        tma_load_1d(stages + (q ^ 1u) * SC_TILE, src + t0 + SC_TILE, tile_len(k + 1) * (u32)sizeof(Tuple), &mbar[q ^ 1u]);
      const Tuple* T = stages + q * SC_TILE;
      u32 br[IT];
#pragma unroll
      for (u32 i = 0; i < IT; ++i) {
        const u32 x = i * NT_SC + tid;
        br[i] = DROP;
        if (x >= n) continue;
        const u64 key = T[x].key;
        u32 b;
        if (MODE == MODE_RADIX) {
          const u64 d = radix_bucket(L, key);
          b = d >= F ? F - 1u : (u32)d;
        } else if (MODE == MODE_LEARN) {
          if (key < kmin || key > kmax) continue;
          u32 e;
          if (LCOMPACT) {
            const u32 c = spl[(key - kmin) >> L.shift];
            e = (c & 0x3FFFu) | ((c & 0x4000u) ? LCELL_HOT : 0u) |
                ((c & 0x8000u) ? (LCELL_SPLIT | ((u32)sphi[c & 0x3FFFu] << 16)) : 0u);
          } else {
            e = spl32[(key - kmin) >> L.shift];
          }
          b = learned_cell_part(e, sbnd, srank, F, fit_n, key, row0 + t0 + x, lc.seed, probes);
        } else if (MODE == MODE_RLEARN) {
          b = run_learn_bucket(spl32[run_learn_cell(RL, key)], sbnd, key);
          b = b < F ? b : F - 1u;
        } else {
          if (key < kmin || key > kmax) continue;
          b = spl[(key - kmin) >> L.shift];
        }
        br[i] = (b << 16) | atomicAdd(&hcnt[b], 1u);
      }
      __syncthreads();
      // hb = exclusive scan of hcnt; position p of bucket b goes to offset gb[b] + p
      // (mod 2^32: gb[b] is the bucket's offset minus hb[b]); counts cleared for the next tile
      u32 kept;
      {
        u32 loc[PER], sum = 0;
#pragma unroll
        for (u32 i = 0; i < PER; ++i) {
          const u32 b = tid * PER + i;
          loc[i] = b < F ? hcnt[b] : 0u;
          sum += loc[i];
        }
        u32 pre = block_exclusive_scan_1b<u32, NT_SC>(sum, &kept, s_warp);
#pragma unroll
        for (u32 i = 0; i < PER; ++i) {
          const u32 b = tid * PER + i;
          if (b < F) {
            hb[b] = pre;
            gb[b] = curv[i] - pre;
            hcnt[b] = 0;
          }
          curv[i] += loc[i];
          pre += loc[i];
        }
      }
      __syncthreads();
#pragma unroll
      for (u32 i = 0; i < IT; ++i) {
        if (br[i] == DROP) continue;
        const u32 b = br[i] >> 16;
        const u32 p = hb[b] + (br[i] & 0xFFFFu);
        sidx[p] = (u16)(i * NT_SC + tid);
        sb[p] = (u16)b;
      }
      __syncthreads();
      for (u32 p = tid; p < kept; p += NT_SC) {
        const u32 off = gb[sb[p]] + p;
        st_tuple(dst + off, T[sidx[p]]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      // one buffer: the next tile's copy is issued before its wait, so every reader of
      // this one must be done first.  Two buffers: the next tile's barrier (and the
      // chunk's, after the last tile) comes before any write to this tile's buffer,
      // counters or index arrays
      if (STAGES == 1) __syncthreads();
    }
  }
}

// ---------------------------------------------------------------- final in-SMEM sort
// One block per final segment: a bulk async copy stages the segment in shared
// memory, its exact key range sets the number of radix digits, the lowest digit
// is a counting pass (order within a digit is free there) and every further
// 8-bit digit a stable pass ranked with warp ballots.  Only a permutation of
// indices moves; the write-out reads tuples in sorted order from shared memory
// and stores them coalesced.  Two instantiations share the work list: CAP =
// 4096 (two blocks per SM, so one block's copy overlaps the other's sort)
// takes segments of at most 4096 tuples and all constant-key segments; CAP =
// 8192 (one block per SM) takes the rest.  The fused instantiation (phases 3
// and 4 in one kernel) takes every final S segment, in 4096-tuple pieces, and
// joins it in shared memory instead of writing it out.  A block fetches its next
// segment one ahead and asks L2 for that segment's data, so the next bulk copy
// finds it there.
// sum of one u64 per thread over the block (result valid in thread 0)
template <u32 NT>
__device__ __forceinline__ u64 block_sum_u64(u64 v, u64* s_red) {
  v = warp_sum(v);
  if (lane_id() == 0) s_red[warp_id()] = v;
  __syncthreads();
  u64 t = 0;
  if (threadIdx.x == 0)
    for (u32 w = 0; w < NT / 32; ++w) t += s_red[w];
  __syncthreads();
  return t;
}

// Join of a segment or piece whose keys all equal `key` (n tuples at s, global or
// shared): every R tuple of its windows with that key matches every S tuple.
// Each matching R tuple r adds n pairs and n r.pay + (sum of the S payloads) to
// the calling thread's running count and checksum.  The windows of up to RCH runs at a
// time are staged in rtab (free shared memory) with their prefix sums, so the block's
// threads share every window position: a hot key's long window in one run is read by
// all of them, not walked by one thread.
constexpr u32 RCH = 128;
// shared memory the fused kernel adds after the counting array, so that the u16
// directory of a segment covers 2^14 keys (two blocks per SM still fit)
constexpr u32 DIR_EXT_BYTES = 16384;

template <u32 NT>
__device__ __forceinline__ void seg_join_const(const Tuple* s, u32 n, u64 key, const Seg& sg, u32 item,
                                               const FuseCtx& fc, u64* s_red, u32* rtab, u64& acc_cnt,
                                               u64& acc_chk) {
  const u32 tid = threadIdx.x;
  const Job& J = fc.jobs[sg.job];
  u64 ssum = 0;
  for (u32 i = tid; i < n; i += NT) ssum += s[i].pay;
  ssum = block_sum_u64<NT>(ssum, s_red);
  if (tid == 0) s_red[0] = ssum;
  __syncthreads();
  ssum = s_red[0];
  u32* wl = rtab;                                            // RCH window starts
  u32* wpre = rtab + RCH;                                    // RCH + 1 window prefix
  u64* roff = reinterpret_cast<u64*>(rtab + 2 * RCH + 8);    // RCH run offsets
  const u32 T = J.runs;
  for (u32 j0 = 0; j0 < T; j0 += RCH) {
    const u32 nr = T - j0 < RCH ? T - j0 : RCH;
    __syncthreads();  // ssum read; the previous chunk's readers are done
    if (tid < nr) {
      const u32* w = fc.swin + 2ull * ((u64)item * fc.maxT + j0 + tid);
      wl[tid] = w[0];
      wpre[tid] = w[1] > w[0] ? w[1] - w[0] : 0u;
      roff[tid] = fc.runs[J.run_base + j0 + tid].off;
    }
    __syncthreads();
    if (tid < 32) {  // exclusive scan of the window lengths, 4 per lane
      u32 v[4], sum = 0;
#pragma unroll
      for (u32 k = 0; k < 4; ++k) {
        const u32 idx = tid * 4 + k;
        v[k] = idx < nr ? wpre[idx] : 0u;
        sum += v[k];
      }
      u32 inc = sum;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const u32 y = __shfl_up_sync(0xffffffffu, inc, d);
        if (tid >= (u32)d) inc += y;
      }
      u32 run = inc - sum;
#pragma unroll
      for (u32 k = 0; k < 4; ++k) {
        const u32 idx = tid * 4 + k;
        if (idx < nr) wpre[idx] = run;
        run += v[k];
      }
      const u32 tot = __shfl_sync(0xffffffffu, inc, 31);
      if (tid == 0) wpre[nr] = tot;
    }
    __syncthreads();
    const u32 W = wpre[nr];
    for (u32 q = tid; q < W; q += NT) {
      u32 lo = 0, hi = nr;  // run: last with wpre[lo] <= q
      while (hi - lo > 1) {
        const u32 mid = (lo + hi) >> 1;
        if (wpre[mid] <= q) lo = mid;
        else hi = mid;
      }
      // the windows cover the segment's bounds, which may exceed `key`
      const Tuple t = ld_stream(fc.xr + roff[lo] + wl[lo] + (q - wpre[lo]));
      if (t.key == key) {
        acc_cnt += n;
        acc_chk += ssum + (u64)n * t.pay;
      }
    }
  }
}

// Adds the block's running count and checksum to job `job`'s totals (every thread calls it).
template <u32 NT>
__device__ __forceinline__ void flush_job_result(u64& acc_cnt, u64& acc_chk, u32 job, const FuseCtx& fc, u64* s_red) {
  const u64 c = block_sum_u64<NT>(acc_cnt, s_red);
  const u64 k = block_sum_u64<NT>(acc_chk, s_red);
  if (threadIdx.x == 0 && job != 0xFFFFFFFFu && c) {
    atomicAdd(&fc.jobs[job].count, c);
    atomicAdd(&fc.jobs[job].checksum, k);
  }
  acc_cnt = 0;
  acc_chk = 0;
}

// Join of a sorted segment (tup in the order ia, n tuples, keys in [mn, mx])
// against its R windows, added to the calling thread's running count and
// checksum.  dir (free shared memory, 2^DIRB u16 entries) becomes an
// order-preserving directory of at most 2^DIRB - 1 key buckets -- one key per
// bucket when the segment's key range allows -- unless cdir gives the exact per-key
// starts; rtab (free shared memory) stages up to RCH runs' windows and their prefix
// sums at a time, so every thread takes any window position.

// The window of run tid (< RCH) of the block's segment, read by thread tid when the
// segment starts, so that its latency hides behind the sort; the first RCH runs'
// windows are staged from these registers.
struct WinReg {
  u32 lo, hi;  // window [lo, hi) in the run
  u64 off;     // the run's first position in xr
};

template <u32 CAP, u32 NT, u32 DIRB>
__device__ __forceinline__ void seg_join(const Tuple* tup, const u16* ia, u16* dir, u32* rtab, const u32* cdir, u32 n,
                                         u64 mn, u64 mx, const Seg& sg, u32 item, const FuseCtx& fc, const WinReg& wr,
                                         u64& cnt, u64& chk) {
  const u32 tid = threadIdx.x, lane = tid & 31u, wid = tid >> 5;
  const Job& J = fc.jobs[sg.job];
  const u32 T = J.runs, run_base = J.run_base;
  const u64 range = mx - mn;
  const u32 rbits = bitlen64(range);
  u32 dsh = rbits > DIRB ? rbits - DIRB : 0u;
  if ((range >> dsh) + 2u > (u64)(1u << DIRB)) ++dsh;  // nbk + 1 entries fit
  const u32 nbk = (u32)(range >> dsh) + 1u;
  if (!cdir) {
    // the caller checked every key against [mn, mx]; the clamp keeps the writes inside
    // the nbk + 1 directory entries regardless
    auto bucket = [&](u32 i) {
      const u64 b = (tup[ia[i]].key - mn) >> dsh;
      return b < (u64)nbk ? (u32)b : nbk - 1u;
    };
    for (u32 i = tid; i < n; i += NT) {
      const u32 b = bucket(i);
      const u32 x0 = i ? bucket(i - 1) + 1u : 0u;
      for (u32 x = x0; x <= b; ++x) dir[x] = (u16)i;
      if (i == n - 1)
        for (u32 x = b + 1u; x <= nbk; ++x) dir[x] = (u16)n;
    }
  }
  // wpre: RCH + 1 window prefix sums; rbase: per run, the xr index of window position
  // q is rbase + q (the window's first tuple minus its prefix, modulo 2^64)
  u32* wpre = rtab;
  u64* rbase = reinterpret_cast<u64*>(rtab + RCH + 8);
  for (u32 j0 = 0; j0 < T; j0 += RCH) {
    const u32 nr = T - j0 < RCH ? T - j0 : RCH;
    // directory built; the previous chunk's readers are done (with cdir, the caller's
    // barrier after the placement comes right before the first chunk)
    if (j0 || !cdir) __syncthreads();
    if (tid < nr) {
      u32 lo, hi;
      u64 off;
      if (j0 == 0) {
        lo = wr.lo;
        hi = wr.hi;
        off = wr.off;
      } else {
        const u32* w = fc.swin + 2ull * ((u64)item * fc.maxT + j0 + tid);
        lo = w[0];
        hi = w[1];
        off = fc.runs[run_base + j0 + tid].off;
      }
      wpre[tid] = hi > lo ? hi - lo : 0u;  // empty unless the run was sorted (a failed check)
      rbase[tid] = off + lo;
    }
    __syncthreads();
    if (tid < 32) {  // exclusive scan of the window lengths, 4 per lane
      u32 v[4], sum = 0;
#pragma unroll
      for (u32 k = 0; k < 4; ++k) {
        const u32 idx = tid * 4 + k;
        v[k] = idx < nr ? wpre[idx] : 0u;
        sum += v[k];
      }
      u32 inc = sum;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const u32 y = __shfl_up_sync(0xffffffffu, inc, d);
        if (tid >= (u32)d) inc += y;
      }
      u32 run = inc - sum;
#pragma unroll
      for (u32 k = 0; k < 4; ++k) {
        const u32 idx = tid * 4 + k;
        if (idx < nr) {
          wpre[idx] = run;
          rbase[idx] -= run;
        }
        run += v[k];
      }
      const u32 tot = __shfl_sync(0xffffffffu, inc, 31);
      if (tid == 0) wpre[nr] = tot;
    }
    __syncthreads();
    const u32 W = wpre[nr];
    constexpr u32 U = 4;  // most R loads in flight per thread
    // each warp takes 32 Ub consecutive window positions per step, Ub loads of 32
    // consecutive positions, so a warp's positions span few runs: one search finds the
    // run of its first position, and each lane walks on from there.  Ub grows with the
    // windows (1 to U), so that short windows still spread over every warp.
    const u32 Ub = W >= NT * U ? U : (W + NT - 1u) / NT;
    for (u32 q0 = wid * (32u * Ub); q0 < W; q0 += NT * Ub) {
      u32 j = 0, hi = nr;  // the last run whose prefix is <= q0
      while (hi - j > 1) {
        const u32 mid = (j + hi) >> 1;
        if (wpre[mid] <= q0) j = mid;
        else hi = mid;
      }
      Tuple r[U];
#pragma unroll
      for (u32 u = 0; u < U; ++u) {
        const u32 q = q0 + u * 32u + lane;
        r[u].key = 0;
        r[u].pay = 0;
        if (u < Ub && q < W) {
          while (wpre[j + 1] <= q) ++j;  // wpre[nr] = W > q ends the walk
          r[u] = ld_stream(fc.xr + (rbase[j] + q));
        }
      }
#pragma unroll
      for (u32 u = 0; u < U; ++u) {
        const u32 q = q0 + u * 32u + lane;
        if (u >= Ub || q >= W) continue;
        const u64 key = r[u].key;
        if (key < mn || key > mx) continue;
        u32 lb, ub;
        if (cdir) {  // exact per-key starts
          const u32 d = (u32)(key - mn);
          lb = cdir[d];
          ub = cdir[d + 1];
        } else {
          const u32 bi = (u32)((key - mn) >> dsh);
          lb = dir[bi];
          ub = dir[bi + 1];
        }
        if (!cdir && dsh) {  // a bucket spans several keys: narrow [lb, ub) to `key`
          u32 a = lb, m = ub - lb;
          while (m > 0) {
            const u32 h = m >> 1;
            if (tup[ia[a + h]].key < key) {
              a += h + 1;
              m -= h + 1;
            } else {
              m = h;
            }
          }
          u32 e = a;
          while (e < ub && tup[ia[e]].key == key) ++e;
          lb = a;
          ub = e;
        }
        if (lb >= ub) continue;
        u64 ssum = 0;
        for (u32 i = lb; i < ub; ++i) ssum += tup[ia[i]].pay;
        cnt += ub - lb;
        chk += (u64)(ub - lb) * r[u].pay + ssum;
      }
    }
  }
}

template <u32 CAP, u32 MINB, bool FUSE, u32 NT>
__global__ void __launch_bounds__(NT, MINB) k_seg_sort(const Seg* segs, const u32* nseg_ptr, u32 cap, u32* work,
                                                            Bufs bufs, const Job* jobs, u32 dst_where, u32* err,
                                                            FuseCtx fc) {
  constexpr u32 IT = CAP / NT;
  constexpr u32 NW = NT / 32;
  constexpr bool SMALL = CAP <= NMAX / 2;
  extern __shared__ __align__(128) unsigned char sm_raw[];
  Tuple* tup = reinterpret_cast<Tuple*>(sm_raw);        // CAP
  u16* ia = reinterpret_cast<u16*>(tup + CAP);          // CAP
  u16* ib = ia + CAP;                                   // CAP
  u32* cnt = reinterpret_cast<u32*>(ib + CAP);          // NW * 256 (>= 2048); fused: DIR_EXT_BYTES after it
  __shared__ __align__(8) u64 mbar;
  __shared__ u32 s_item[2];
  __shared__ u32 s_warp[NT / 32 + 1];
  __shared__ u64 s_mn[NW], s_mx[NW];
  __shared__ u64 s_red[NW];
  const u32 tid = threadIdx.x, lane = lane_id(), wid = warp_id();
  if (tid == 0) {
    mbar_init(&mbar, 1);
    s_item[0] = atomicAdd(work, 1u);
  }
  u32 slot = 0;
  u32 phase = 0;
  u32 n_items = *nseg_ptr;
  if (n_items > cap) n_items = cap;
  Tuple* dstb = dst_where == W_XR ? bufs.xr : bufs.xs;
  // fused: each thread's count and checksum run on across the segments of one job;
  // the block adds them to the job's totals when the job changes and at the end
  u64 acc_cnt = 0, acc_chk = 0;
  u32 acc_job = 0xFFFFFFFFu;
  for (;;) {
    // order this block's earlier generic-proxy use of the buffers before the next bulk copy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();  // publishes the item thread 0 fetched during the previous one
    const u32 item = s_item[slot];
    if (item >= n_items) break;
    u32 nxt = 0;
    if (tid == 0) nxt = atomicAdd(work, 1u);  // the next item; its value is needed only below
    const u32 nslot = slot ^ 1u;
    slot ^= 1u;
    // thread 0 publishes the next item (read after the barrier that ends this one) and
    // asks L2 for the start of its data, so its bulk copy finds it there
    auto publish_next = [&]() {
      if (tid == 0) {
        s_item[nslot] = nxt;
        if (nxt < n_items) {
          const Seg ns = segs[nxt];
          const bool nconst = (ns.flags & SEG_EXACT) && ns.kmin == ns.kmax;
          // only a segment of this class (the same test as the skip below)
          const bool mine = SMALL ? !(!FUSE && !nconst && ns.len > CAP) : !(nconst || ns.len <= NMAX / 2);
          const Tuple* nsrc = seg_src(bufs, jobs, ns.flags & 7u, ns.job, ns.off);
          const u32 nbytes = (u32)((ns.len < CAP ? ns.len : (u64)CAP) * sizeof(Tuple));
          if (mine && nbytes)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(nsrc), "r"(nbytes) : "memory");
        }
      }
    };
    bool published = false;
    const Seg sg = segs[item];
    const bool constant = (sg.flags & SEG_EXACT) && sg.kmin == sg.kmax;
    // the other class (the fused small class takes every segment, big ones in pieces)
    if (SMALL ? (!FUSE && !constant && sg.len > CAP) : (constant || sg.len <= NMAX / 2)) {
      publish_next();
      continue;
    }
    if (FUSE && sg.job != acc_job) {  // block-uniform: sg is the block's segment
      flush_job_result<NT>(acc_cnt, acc_chk, acc_job, fc, s_red);
      acc_job = sg.job;
    }
    const Tuple* src = seg_src(bufs, jobs, sg.flags & 7u, sg.job, sg.off);
    Tuple* dst = dstb + sg.off;
    const u32 n = (u32)sg.len;
    const bool inplace = (src == dst);
    if (constant) {
      publish_next();
      if (FUSE) {
        seg_join_const<NT>(src, n, sg.kmin, sg, item, fc, s_red, reinterpret_cast<u32*>(ib), acc_cnt, acc_chk);
      } else if (!inplace) {
        for (u32 i = tid; i < n; i += NT) st_tuple(dst + i, src[i]);
      }
      continue;
    }
    if (!FUSE && sg.len > CAP) {
      if (tid == 0) atomicOr(err, (u32)DERR_SEG_TOO_BIG);
      publish_next();
      continue;
    }
    WinReg wr{0u, 0u, 0ull};
    // The fused join is exact for any split of S into pieces joined against windows
    // that cover their keys, so a segment above CAP is sorted and joined in pieces.
    bool failed = false;
    for (u32 p0 = 0; p0 < n; p0 += CAP) {
    const u32 n = (sg.len - p0 < CAP) ? (u32)(sg.len - p0) : CAP;  // this piece
    if (tid == 0) tma_load_1d(tup, src + p0, n * (u32)sizeof(Tuple), &mbar);
    if (!published) {
      publish_next();
      published = true;
      // fused: run tid's window of this segment, read while the copy is in flight and
      // used by the join after the sort
      if (FUSE) {
        const Job& J = fc.jobs[sg.job];
        if (tid < J.runs && tid < RCH) {
          const u32* w = fc.swin + 2ull * ((u64)item * fc.maxT + tid);
          wr.lo = w[0];
          wr.hi = w[1];
          wr.off = fc.runs[J.run_base + tid].off;
        }
      }
    }
    // the counting pass's counters, cleared while the copy is in flight (their last
    // readers passed the barrier before this piece; the one after the wait orders it)
    for (u32 b = tid; b < 2048u; b += NT) cnt[b] = 0;
    const bool ok = mbar_wait(&mbar, phase, SPIN_LIMIT);
    phase ^= 1u;
    if (!__syncthreads_and(ok)) {
      if (tid == 0) atomicOr(err, (u32)DERR_TMA_TIMEOUT);
      failed = true;
      break;
    }
    // key range: the segment's exact bounds from the pass that made it, else a reduction
    u64 mn = ~0ull, mx = 0;
    if (sg.flags & SEG_EXACT) {
      mn = sg.kmin;
      mx = sg.kmax;
    } else {
      for (u32 i = tid; i < n; i += NT) {
        const u64 k = tup[i].key;
        mn = k < mn ? k : mn;
        mx = k > mx ? k : mx;
      }
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {
        const u64 a = __shfl_xor_sync(0xffffffffu, mn, d), b = __shfl_xor_sync(0xffffffffu, mx, d);
        mn = a < mn ? a : mn;
        mx = b > mx ? b : mx;
      }
      if (lane == 0) {
        s_mn[wid] = mn;
        s_mx[wid] = mx;
      }
      __syncthreads();
      mn = s_mn[0];
      mx = s_mx[0];
#pragma unroll
      for (u32 w = 1; w < NW; ++w) {
        mn = s_mn[w] < mn ? s_mn[w] : mn;
        mx = s_mx[w] > mx ? s_mx[w] : mx;
      }
    }
    const u32 bits = bitlen64(mx - mn);
    if (bits == 0) {
      if (FUSE) {
        seg_join_const<NT>(tup, n, mn, sg, item, fc, s_red, reinterpret_cast<u32*>(ib), acc_cnt, acc_chk);
      } else if (!inplace) {
        for (u32 i = tid; i < n; i += NT) st_tuple(dst + i, tup[i]);
      }
      __syncthreads();
      continue;
    }
    // pass 1: counting sort on the low digit (order within a digit is free here)
    const u32 w1 = bits < 11u ? bits : 11u;
    const u32 F1 = 1u << w1;
    u32 dr[IT];
    bool outside = false;  // a key beyond the segment's recorded bounds
#pragma unroll
    for (u32 i = 0; i < IT; ++i) {
      const u32 e = tid + i * NT;
      if (e < n) {
        const u64 key = tup[e].key;
        outside |= key < mn || key > mx;
        const u32 d = (u32)((key - mn) & (u64)(F1 - 1u));
        const u32 r = atomicAdd(&cnt[d], 1u);
        dr[i] = (d << 16) | r;
      }
    }
    // Every shared-memory index below is masked to its digit or checked against
    // [mn, mx]; the recorded bounds are exact by construction, and if they ever were
    // not, the piece is reported and left instead of being sorted or joined wrongly.
    if (__syncthreads_or(outside)) {
      if (tid == 0) atomicOr(err, (u32)DERR_BOUNDS);
      failed = true;
      break;
    }
    // fused: ask L2 for this thread's R window (by 128-byte line), so the join's loads
    // find it there
    if (FUSE && p0 == 0 && wr.hi > wr.lo) {
      const char* wp = reinterpret_cast<const char*>(fc.xr + wr.off + wr.lo);
      const char* we = reinterpret_cast<const char*>(fc.xr + wr.off + wr.hi);
      for (const char* q = (const char*)((size_t)wp & ~(size_t)127); q < we; q += 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
    }
    smem_exclusive_scan<u32, NT, 2048 / NT>(cnt, F1, s_warp);
    if (tid == 0) cnt[F1] = n;  // with bits <= 11, cnt is then the start of every key value
#pragma unroll
    for (u32 i = 0; i < IT; ++i) {
      const u32 e = tid + i * NT;
      if (e < n) ia[cnt[dr[i] >> 16] + (dr[i] & 0xFFFFu)] = (u16)e;
    }
    __syncthreads();
    // further digits: stable ranking, 8 bits per pass
    u32 sh = w1;
    const u32 per = (((n + NW - 1) / NW) + 31u) & ~31u;
    const u32 wb = wid * per;
    const u32 we = (wb + per < n) ? wb + per : n;
    const u32 nb = per / 32u;
    const u32 lt = (1u << lane) - 1u;
    while (sh < bits) {
      const u32 w = (bits - sh) < 8u ? (bits - sh) : 8u;
      const u32 FB = 1u << w;
      for (u32 i = tid; i < NW * 256u; i += NT) cnt[i] = 0;
      __syncthreads();
      u32 rec[IT];
      u16 ee[IT];
#pragma unroll
      for (u32 k = 0; k < IT; ++k) {
        if (k < nb) {
          const u32 pos = wb + k * 32u + lane;
          const bool valid = pos < we;
          const u32 e = valid ? ia[pos] : 0u;
          const u32 d = valid ? (u32)(((tup[e].key - mn) >> sh) & (u64)(FB - 1u)) : 0u;
          u32 peers = __ballot_sync(0xffffffffu, valid);
          for (u32 bit = 0; bit < w; ++bit) {
            const u32 bb = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
            peers &= ((d >> bit) & 1u) ? bb : ~bb;
          }
          const u32 rank_in = __popc(peers & lt);
          const u32 leader = __ffs(peers) - 1u;
          u32 base = 0;
          if (valid) base = cnt[wid * 256u + d];
          __syncwarp();
          if (valid && lane == leader) cnt[wid * 256u + d] = base + __popc(peers);
          __syncwarp();
          rec[k] = (d << 16) | (base + rank_in);
          ee[k] = (u16)e;
        }
      }
      __syncthreads();
      {
        u32 tot_d = 0;
        if (tid < FB)
          for (u32 ww = 0; ww < NW; ++ww) tot_d += cnt[ww * 256u + tid];
        u32 total;
        const u32 dbase = block_exclusive_scan<u32, NT>(tid < FB ? tot_d : 0u, &total, s_warp);
        if (tid < FB) {
          u32 run = dbase;
          for (u32 ww = 0; ww < NW; ++ww) {
            const u32 c = cnt[ww * 256u + tid];
            cnt[ww * 256u + tid] = run;
            run += c;
          }
        }
      }
      __syncthreads();
#pragma unroll
      for (u32 k = 0; k < IT; ++k) {
        if (k < nb) {
          const u32 pos = wb + k * 32u + lane;
          if (pos < we) ib[cnt[wid * 256u + (rec[k] >> 16)] + (rec[k] & 0xFFFFu)] = ee[k];
        }
      }
      __syncthreads();
      u16* t = ia;
      ia = ib;
      ib = t;
      sh += w;
    }
    if (FUSE) {
      // the free index array stages the windows; the counting pass's digit starts are an
      // exact per-key directory after one pass, else the counters and the extension
      // after them hold a u16 directory
      constexpr u32 DIRB = 14;
      static_assert((1u << DIRB) * sizeof(u16) <= NW * 256u * sizeof(u32) + DIR_EXT_BYTES,
                    "the u16 directory fits the counting array and its extension");
      if (bits <= 11u)
        seg_join<CAP, NT, DIRB>(tup, ia, nullptr, reinterpret_cast<u32*>(ib), cnt, n, mn, mx, sg, item, fc, wr,
                                acc_cnt, acc_chk);
      else
        seg_join<CAP, NT, DIRB>(tup, ia, reinterpret_cast<u16*>(cnt), reinterpret_cast<u32*>(ib), nullptr, n, mn, mx,
                                sg, item, fc, wr, acc_cnt, acc_chk);
    } else {
      for (u32 i = tid; i < n; i += NT) st_tuple(dst + i, tup[ia[i]]);
    }
    // every reader of this piece is done before the next bulk copy overwrites it: a
    // barrier here before the segment's next piece, the loop's own before the next segment
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if ((u64)p0 + CAP < sg.len) __syncthreads();
    }
    if (failed) break;
  }
  if (FUSE) flush_job_result<NT>(acc_cnt, acc_chk, acc_job, fc, s_red);
}

// ---------------------------------------------------------------- fused-path search
// Fences: every 64th key of the sorted runs (one array over xr), small enough to
// stay in L2, so a run bound costs a fence search plus one 64-tuple block.
__global__ void k_fences(const Tuple* xr, u64 n, u64* fence) {
  const u64 nf = (n + 63) / 64;
  for (u64 g = (u64)blockIdx.x * blockDim.x + threadIdx.x; g < nf; g += (u64)gridDim.x * blockDim.x)
    fence[g] = xr[g * 64].key;
}

// Every gs-th fence of one run [g0, g1), staged in shared memory by the block that
// searches that run: a fence search then bisects ntop shared entries and at most
// gs - 1 fences instead of all g1 - g0.
constexpr u32 TOP_CAP = 2048;
struct TopFences {
  const u64* top;  // top[t] = fence[g0 + t * gs], t < ntop
  u32 ntop;
  u64 gs;
};

// first position of run [off, off + len) whose key is >= key (upper: > key), minus off;
// the fences are searched by bisection (narrowed first by `tf`, the run's staged
// top-level fences, when given) or (interp) by interpolation search.  With
// `from` (an upper bound after the lower bound of a key <= this one), the fence search
// gallops forward from the fence the lower bound stopped at, *from, instead: a window
// is short, so its end is a fence or two on, in lines the lower bound brought into L2.
// `at` receives the fence the search stopped at.
__device__ __forceinline__ u64 run_bound(const Tuple* xr, const u64* fence, u64 off, u64 len, u64 key, bool upper,
                                         u32& probes, bool interp = false, const u64* from = nullptr,
                                         u64* at = nullptr, TopFences tf = TopFences{nullptr, 0u, 1ull}) {
  const u64 end = off + len;
  u64 lo = off, hi = end;
  const u64 g0 = (off + 63) / 64, g1 = len ? (end - 1) / 64 + 1 : g0;
  if (g0 < g1) {
    u64 a = g0, m = g1 - g0;
    if (from && *from >= g0 && *from <= g1) {
      // every fence before *from is below the earlier key, so not past this one
      a = *from;
      u64 step = 1;
      for (;;) {
        if (a >= g1) {
          m = 0;
          break;
        }
        ++probes;
        const u64 f = fence[a];
        if (upper ? f > key : f >= key) {
          m = 0;
          break;
        }
        const u64 next = a + step;
        if (next >= g1) {  // the answer is in (a, g1]
          m = g1 - (a + 1);
          a = a + 1;
          break;
        }
        ++probes;
        const u64 fn = fence[next];
        if (upper ? fn > key : fn >= key) {  // the answer is in (a, next]
          m = next - (a + 1);
          a = a + 1;
          break;
        }
        a = next + 1;
        step <<= 1;
      }
    } else if (tf.top) {
      // first staged fence past the key: the answer lies in the gs fences up to it
      u32 t = 0, tm = tf.ntop;
      while (tm > 0) {
        const u32 h = tm >> 1;
        const u64 f = tf.top[t + h];
        if (!(upper ? f > key : f >= key)) {
          t += h + 1;
          tm -= h + 1;
        } else {
          tm = h;
        }
      }
      if (t == 0) {
        m = 0;  // the run's first fence is already past the key
      } else {
        a = g0 + (u64)(t - 1) * tf.gs + 1;
        const u64 b = g0 + (u64)t * tf.gs;
        m = (b < g1 ? b : g1) - a;
      }
    } else if (interp) {
      if (upper && key == ~0ull) {
        a = g1;
      } else {
        auto at = [&](u64 i) { return fence[g0 + i]; };
        a = g0 + interp_lower_bound(at, g1 - g0, upper ? key + 1ull : key, probes);
      }
      m = 0;
    }
    while (m > 0) {
      const u64 h = m >> 1;
      ++probes;
      const u64 f = fence[a + h];
      if (!(upper ? f > key : f >= key)) {
        a += h + 1;
        m -= h + 1;
      } else {
        m = h;
      }
    }
    if (at) *at = a;
    if (a > g0) lo = (a - 1) * 64 + 1;
    if (a < g1) hi = a * 64;
  } else if (at) {
    *at = g0;
  }
  u64 m = hi - lo;
  while (m > 0) {
    const u64 h = m >> 1;
    ++probes;
    const u64 k = xr[lo + h].key;
    if (!(upper ? k > key : k >= key)) {
      lo += h + 1;
      m -= h + 1;
    } else {
      m = h;
    }
  }
  return lo - off;
}

// windows of every (final S segment, R run) pair from the segment's key bounds:
// fence search for the start and a gallop over the fences to the end (or the
// paper's interpolation search over the fences), or with the learned R-side
// model its predicted position times the run length followed by an exact
// exponential + binary search.  Block (x, j) takes run j of every segment
// x, x + gridDim.x, ... (in blockDim-sized groups); for the fence search it stages
// run j's top-level fences (of the job its first segment belongs to) in shared
// memory, and a segment of another job searches the fences alone.
constexpr u32 NT_SEARCH = 256;

__global__ void __launch_bounds__(NT_SEARCH, 6) k_seg_search(const Seg* segs, const u32* nseg_ptr, u32 cap,
                                                          const Job* jobs, const Run* runs, const Tuple* xr,
                                                          const u64* fence, u32* swin, u32 maxT, LearnCtx lc) {
  __shared__ u64 s_top[TOP_CAP];
  __shared__ u32 s_run;
  __shared__ u32 s_ntop;
  __shared__ u64 s_gs;
  u32 nseg = *nseg_ptr;
  if (nseg > cap) nseg = cap;
  const u32 j = blockIdx.y;
  const u32 tid = threadIdx.x;
  u32 probes = 0, nsearch = 0;
  u64 err_sum = 0;
  const bool staged = !lc.models && !lc.interp;
  if (staged) {
    if (tid == 0) {
      s_run = 0xFFFFFFFFu;
      s_ntop = 0;
      s_gs = 1;
      const u32 first = blockIdx.x * NT_SEARCH;
      if (first < nseg) {
        const Job& J = jobs[segs[first].job];
        if (j < J.runs) {
          const Run r = runs[J.run_base + j];
          const u64 g0 = (r.off + 63) / 64, g1 = r.len ? (r.off + r.len - 1) / 64 + 1 : g0;
          const u64 nf = g1 - g0;
          const u64 gs = nf > TOP_CAP ? (nf + TOP_CAP - 1) / TOP_CAP : 1ull;
          s_run = J.run_base + j;
          s_gs = gs;
          s_ntop = (u32)((nf + gs - 1) / gs);
        }
      }
    }
    __syncthreads();
    if (s_run != 0xFFFFFFFFu) {
      const Run r = runs[s_run];
      const u64 g0 = (r.off + 63) / 64;
      for (u32 t = tid; t < s_ntop; t += NT_SEARCH) s_top[t] = fence[g0 + (u64)t * s_gs];
    }
    __syncthreads();
  }
  const TopFences none{nullptr, 0u, 1ull};
  const TopFences tf = staged ? TopFences{s_top, s_ntop, s_gs} : none;
  for (u64 item = (u64)blockIdx.x * NT_SEARCH + tid; item < nseg; item += (u64)gridDim.x * NT_SEARCH) {
    const Seg sg = segs[item];
    const Job& J = jobs[sg.job];
    if (j >= J.runs) continue;
    const u64 idx = item * maxT + j;
    const u32 ri = J.run_base + j;
    const Run r = runs[ri];
    if (lc.models) {
      const RmiModel* M = &lc.models[2 * sg.job + 1];
      const Tuple* a = xr + r.off;
      auto at = [&](u64 i) { return a[i].key; };
      u64 g = (u64)(rmi_predict(M, sg.kmin) * (float)r.len);
      g = g > r.len ? r.len : g;
      const u64 lo = gallop_from(at, r.len, g, sg.kmin, probes);
      err_sum += g > lo ? g - lo : lo - g;
      u64 hi = r.len;
      if (sg.kmax != ~0ull) {
        u64 h = (u64)(rmi_predict(M, sg.kmax) * (float)r.len);
        h = h < lo ? lo : (h > r.len ? r.len : h);
        hi = gallop_from(at, r.len, h, sg.kmax + 1ull, probes);
      }
      swin[2 * idx] = (u32)lo;
      swin[2 * idx + 1] = (u32)hi;
    } else {  // fences by bisection, or by interpolation search (Sec. 3.2.2)
      u64 a = 0;
      const TopFences t = (staged && ri == s_run) ? tf : none;
      swin[2 * idx] = (u32)run_bound(xr, fence, r.off, r.len, sg.kmin, false, probes, lc.interp, nullptr, &a, t);
      swin[2 * idx + 1] = (u32)run_bound(xr, fence, r.off, r.len, sg.kmax, true, probes, lc.interp, &a);
    }
    nsearch += 2;
  }
  if (lc.stat) {
    const u32 wp = warp_sum(probes), wn = warp_sum(nsearch);
    const u64 we = warp_sum(err_sum);
    if (lane_id() == 0 && wn) {
      atomicAdd(&lc.stat[2], (u64)wp);
      atomicAdd(&lc.stat[3], (u64)wn);
      atomicAdd(&lc.stat[4], we);
    }
  }
}

// Test only: narrows the recorded upper bound of the first exact final segment that
// spans at least three keys to the middle of its range, so its largest key lies
// beyond it; the sort kernels must report DERR_BOUNDS for that segment.
__global__ void k_narrow_bounds_test(Seg* segs, const u32* nseg_ptr, u32 cap) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  u32 n = *nseg_ptr;
  if (n > cap) n = cap;
  for (u32 i = 0; i < n; ++i) {
    Seg& s = segs[i];
    if ((s.flags & SEG_EXACT) && s.len >= 2 && s.kmax - s.kmin >= 2) {
      s.kmax = s.kmin + (s.kmax - s.kmin) / 2;
      return;
    }
  }
}

// Points job 0's partitioned input at the next piece of it (the host-buffer join
// copies that input in pieces and joins each against the sorted runs while the
// next one is in flight); its count and checksum keep accumulating.
__global__ void k_set_part(Job* jobs, Seg* split, const Tuple* S, u64 nS) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  jobs[0].S = S;
  jobs[0].nS = nS;
  split[0] = Seg{jobs[0].s_base, nS, 0ull, 0ull, 0u, W_SIN};
}

__global__ void k_check_empty(const u32* cnt, u32* err, u32 flag) {
  if (threadIdx.x == 0 && *cnt != 0) atomicOr(err, flag);
}

constexpr size_t smem_scatter(u32 tile, u32 stages = 1, bool learn = false, u32 lpcap = P_MAX) {
  return stages * tile * sizeof(Tuple) + 3 * F_MAX * sizeof(u32) + 2 * tile * sizeof(u16) +
         FINE_MAX * ((learn && lpcap == P_MAX) ? sizeof(u32) : sizeof(u16)) +
         (learn ? lpcap * (sizeof(u64) + 2 * sizeof(u32) + (lpcap < P_MAX ? sizeof(u16) : 0)) : 0);
}
// the learned partitioning of jobs with at most LN_SMALL partitions: two 5120-tuple buffers
constexpr u32 LN_SMALL = 512;
// the learned partitioning pass: two 4096-tuple buffers per block (one block per SM), so
// the partition boundaries and their ranks fit beside them in shared memory
constexpr u32 LN_TILE = 4096, LN_NT = 1024;
constexpr size_t SMEM_HIST_LEARN = F_MAX * 20 + FINE_MAX * 4 + P_MAX * (sizeof(u64) + 2 * sizeof(u32));
constexpr size_t smem_sort(u32 cap, u32 nt) { return cap * sizeof(Tuple) + 2 * cap * sizeof(u16) + (nt / 32) * 256 * sizeof(u32); }
// the fused kernel's shared memory: the sort's, then the directory's extension
constexpr size_t smem_sort_join(u32 cap, u32 nt) { return smem_sort(cap, nt) + DIR_EXT_BYTES; }
constexpr u32 NT_BIG = 512;  // threads of the 8192-tuple class (one block per SM; 1024 measured slower)
constexpr size_t SMEM_SCAN = (3 * F_MAX + 1) * sizeof(u64);


template <class K>
void set_smem(K kernel, size_t bytes) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  // ask for the largest shared-memory carveout so several blocks fit per SM
  cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

}  // namespace

void init_attrs_pass() {

  set_smem(k_hist<MODE_RADIX, F_MAX>, F_MAX * 20);
  set_smem(k_hist<MODE_FINE, FINE_MAX>, FINE_MAX * 20);
  set_smem(k_hist<MODE_LEARN, F_MAX>, SMEM_HIST_LEARN);
  set_smem(k_hist<MODE_RLEARN, F_MAX>, SMEM_HIST_LEARN);
  set_smem(k_scatter<MODE_RLEARN, LN_TILE, LN_NT, 1, 2>, smem_scatter(LN_TILE, 2, true));
  set_smem(k_scan<MODE_LEARN>, SMEM_SCAN);
  set_smem(k_scatter<MODE_LEARN, LN_TILE, LN_NT, 1, 2>, smem_scatter(LN_TILE, 2, true));
  set_smem(k_scatter<MODE_LEARN, RX_TILE, RX_NT, RX_MINB, RX_STAGES, LN_SMALL>,
           smem_scatter(RX_TILE, RX_STAGES, true, LN_SMALL));
  set_smem(k_scan<MODE_RADIX>, SMEM_SCAN);
  set_smem(k_scan<MODE_SPLIT>, SMEM_SCAN);
  set_smem(k_scatter<MODE_RADIX, RX_TILE, RX_NT, RX_MINB, RX_STAGES>, smem_scatter(RX_TILE, RX_STAGES));
  set_smem(k_scatter<MODE_RADIX, SP_TILE, SP_NT, SP_MINB, 1>, smem_scatter(SP_TILE));
  set_smem(k_scatter<MODE_SPLIT, RX_TILE, RX_NT, RX_MINB, RX_STAGES>, smem_scatter(RX_TILE, RX_STAGES));
  set_smem(k_seg_sort<NMAX / 2, 2, false, NT_SORT>, smem_sort(NMAX / 2, NT_SORT));
  set_smem(k_seg_sort<NMAX, 1, false, NT_BIG>, smem_sort(NMAX, NT_BIG));
  set_smem(k_seg_sort<NMAX / 2, 2, true, NT_SORT>, smem_sort_join(NMAX / 2, NT_SORT));
}

namespace {

}  // namespace

void launch_sample_bounds(Seg* segs, const u32* nseg, u32 max_segs, Bufs bufs, const Job* jobs, cudaStream_t st) {
  if (!max_segs) return;
  const u32 blocks = (max_segs + 7) / 8;
  k_sample_bounds<<<blocks < 1024 ? blocks : 1024, 256, 0, st>>>(segs, nseg, bufs, jobs);
}

void launch_level_plan(const Seg* segs, u32* nseg, u32 seg_cap, LSeg* ls, u64* totals, u32 mode, u64 chunk,
                       u32 radix_bits, const Job* jobs, u64 hist_cap, u64 bucket_cap, u32* err, cudaStream_t st,
                       u64 fill, const LearnCtx* lc) {
  k_level_plan<<<1, 1024, 0, st>>>(segs, nseg, seg_cap, ls, totals, mode, chunk, radix_bits, fill, jobs, hist_cap,
                                   bucket_cap, err, lc ? *lc : LearnCtx{});
}

void launch_init_buckets(u64* bmin, u64* bmax, u64* btot, const u64* totals, cudaStream_t st, int nsm) {
  k_init_buckets<<<nsm * 2, 512, 0, st>>>(bmin, bmax, btot, totals);
}

void launch_hist(u32 mode, const Seg* segs, const u32* nseg, const LSeg* ls, const u64* totals, u64 chunk,
                 Bufs bufs, const Job* jobs, u32 src_where, u32* hist, u64* bmin, u64* bmax, u64* btot,
                 const LearnCtx& lc, cudaStream_t st, int nsm) {
  if (mode == MODE_RADIX) {
    const size_t sm = F_MAX * 20;
    k_hist<MODE_RADIX, F_MAX><<<nsm * 2, NT_PASS, sm, st>>>(segs, nseg, ls, totals, chunk, bufs, jobs, src_where,
                                                             hist, bmin, bmax, btot, lc);
  } else if (mode == MODE_RLEARN) {
    k_hist<MODE_RLEARN, F_MAX><<<nsm * 2, NT_PASS, SMEM_HIST_LEARN, st>>>(segs, nseg, ls, totals, chunk, bufs, jobs,
                                                                        src_where, hist, bmin, bmax, btot, lc);

  } else if (mode == MODE_LEARN) {
    k_hist<MODE_LEARN, F_MAX><<<nsm * 2, NT_PASS, SMEM_HIST_LEARN, st>>>(segs, nseg, ls, totals, chunk, bufs, jobs,
                                                                       src_where, hist, bmin, bmax, btot, lc);
  } else {
    const size_t sm = FINE_MAX * 20;
    k_hist<MODE_FINE, FINE_MAX><<<nsm * 2, NT_PASS, sm, st>>>(segs, nseg, ls, totals, chunk, bufs, jobs,
                                                               src_where, hist, bmin, bmax, btot, lc);
  }
}

void launch_scan(u32 mode, const Seg* segs, const u32* nseg, const LSeg* ls, u32* hist, const u64* bmin,
                 const u64* bmax, const u32* part_fstart, Seg* big_out, u32* big_cnt, u32 big_cap, Seg* fin_out,
                 u32* fin_cnt, u32 fin_cap, u32 dst_where, Job* jobs, u64* part_off, u32* err, cudaStream_t st,
                 int nsm, bool keep_const, const u64* lbnd) {
  // constant-key children already at their final place are skipped unless the
  // fused sort-and-join must still see them
  const u32 final_where = (!keep_const && (dst_where == W_XR || dst_where == W_XS)) ? dst_where : 0xFFu;
  if (mode == MODE_SPLIT) {
    k_scan<MODE_SPLIT><<<nsm * 2, NT_PASS, SMEM_SCAN, st>>>(segs, nseg, ls, hist, bmin, bmax, part_fstart, big_out,
                                                            big_cnt, big_cap, fin_out, fin_cnt, fin_cap, dst_where,
                                                            final_where, jobs, part_off, err, lbnd);
  } else if (mode == MODE_LEARN) {
    k_scan<MODE_LEARN><<<nsm * 2, NT_PASS, SMEM_SCAN, st>>>(segs, nseg, ls, hist, bmin, bmax, part_fstart, big_out,
                                                            big_cnt, big_cap, fin_out, fin_cnt, fin_cap, dst_where,
                                                            final_where, jobs, part_off, err, lbnd);
  } else {
    k_scan<MODE_RADIX><<<nsm * 2, NT_PASS, SMEM_SCAN, st>>>(segs, nseg, ls, hist, bmin, bmax, part_fstart, big_out,
                                                            big_cnt, big_cap, fin_out, fin_cnt, fin_cap, dst_where,
                                                            final_where, jobs, part_off, err, lbnd);
  }
}

void launch_scatter(u32 mode, const Seg* segs, const u32* nseg, const LSeg* ls, const u64* totals, u64 chunk,
                    Bufs bufs, const Job* jobs, u32 src_where, u32 dst_where, const u32* hist, const u32* sp,
                    u32* err, const LearnCtx& lc, cudaStream_t st, int nsm, bool big_tiles) {
  if (mode == MODE_SPLIT) {
    k_scatter<MODE_SPLIT, RX_TILE, RX_NT, RX_MINB, RX_STAGES><<<nsm * RX_MINB, RX_NT, smem_scatter(RX_TILE, RX_STAGES), st>>>(
        segs, nseg, ls, totals, chunk, bufs, jobs, src_where, dst_where, hist, sp, err, lc);
  } else if (mode == MODE_LEARN && big_tiles) {  // every job has at most LN_SMALL partitions
    k_scatter<MODE_LEARN, RX_TILE, RX_NT, RX_MINB, RX_STAGES, LN_SMALL>
        <<<nsm * RX_MINB, RX_NT, smem_scatter(RX_TILE, RX_STAGES, true, LN_SMALL), st>>>(
            segs, nseg, ls, totals, chunk, bufs, jobs, src_where, dst_where, hist, sp, err, lc);
  } else if (mode == MODE_LEARN) {
    k_scatter<MODE_LEARN, LN_TILE, LN_NT, 1, 2><<<nsm, LN_NT, smem_scatter(LN_TILE, 2, true), st>>>(
        segs, nseg, ls, totals, chunk, bufs, jobs, src_where, dst_where, hist, sp, err, lc);
  } else if (mode == MODE_RLEARN) {  // the learned run bucket tables take the learned pass's layout
    k_scatter<MODE_RLEARN, LN_TILE, LN_NT, 1, 2><<<nsm, LN_NT, smem_scatter(LN_TILE, 2, true), st>>>(
        segs, nseg, ls, totals, chunk, bufs, jobs, src_where, dst_where, hist, sp, err, lc);

  } else if (big_tiles) {
    k_scatter<MODE_RADIX, RX_TILE, RX_NT, RX_MINB, RX_STAGES><<<nsm * RX_MINB, RX_NT, smem_scatter(RX_TILE, RX_STAGES), st>>>(
        segs, nseg, ls, totals, chunk, bufs, jobs, src_where, dst_where, hist, sp, err, lc);
  } else {
    k_scatter<MODE_RADIX, SP_TILE, SP_NT, SP_MINB, 1><<<nsm * SP_MINB, SP_NT, smem_scatter(SP_TILE), st>>>(
        segs, nseg, ls, totals, chunk, bufs, jobs, src_where, dst_where, hist, sp, err, lc);
  }
}

void launch_seg_sort(const Seg* segs, const u32* nseg, u32 cap, u32* work, Bufs bufs, const Job* jobs,
                     u32 dst_where, u32* err, cudaStream_t st, int nsm) {
  // small segments first (two blocks per SM), then the large ones; each kernel
  // walks the whole list with its own work counter and skips the other class
  const FuseCtx none{};
  k_seg_sort<NMAX / 2, 2, false, NT_SORT><<<nsm * 2, NT_SORT, smem_sort(NMAX / 2, NT_SORT), st>>>(
      segs, nseg, cap, work, bufs, jobs, dst_where, err, none);
  k_seg_sort<NMAX, 1, false, NT_BIG><<<nsm, NT_BIG, smem_sort(NMAX, NT_BIG), st>>>(segs, nseg, cap, work + 1, bufs, jobs,
                                                                                 dst_where, err, none);
}

void launch_seg_sort_join(const Seg* segs, const u32* nseg, u32 cap, u32* work, Bufs bufs, const Job* jobs, u32* err,
                          const FuseCtx& fc, cudaStream_t st, int nsm) {
  // one size class: segments above 4096 tuples are sorted and joined in pieces
  k_seg_sort<NMAX / 2, 2, true, NT_SORT><<<nsm * 2, NT_SORT, smem_sort_join(NMAX / 2, NT_SORT), st>>>(
      segs, nseg, cap, work, bufs, jobs, W_XS, err, fc);
}

void launch_fences(const Tuple* xr, u64 n, u64* fence, cudaStream_t st, int nsm) {
  if (n) k_fences<<<nsm * 4, 256, 0, st>>>(xr, n, fence);
}

void launch_seg_search(const Seg* segs, const u32* nseg, u32 cap, const Job* jobs, const Run* runs, const Tuple* xr,
                       const u64* fence, u32* swin, u32 maxT, const LearnCtx& lc, cudaStream_t st, int nsm) {
  if (!maxT) return;
  // one wave of six blocks per SM over all runs (gridDim.y = maxT <= RUNS_MAX)
  const u32 bx = std::max<u32>(1u, (u32)((nsm * 6 + maxT - 1) / maxT));
  k_seg_search<<<dim3(bx, maxT), NT_SEARCH, 0, st>>>(segs, nseg, cap, jobs, runs, xr, fence, swin, maxT, lc);
}

void launch_narrow_bounds_test(Seg* segs, const u32* nseg, u32 cap, cudaStream_t st) {
  k_narrow_bounds_test<<<1, 32, 0, st>>>(segs, nseg, cap);
}

void launch_set_part(Job* jobs, Seg* split, const Tuple* S, u64 nS, cudaStream_t st) {
  k_set_part<<<1, 32, 0, st>>>(jobs, split, S, nS);
}

void launch_check_empty(const u32* cnt, u32* err, u32 flag, cudaStream_t st) {
  k_check_empty<<<1, 32, 0, st>>>(cnt, err, flag);
}


// ---------------------------------------------------------------- allocation-free run sort
// Sorts the runs of R into a caller buffer with all scratch -- the job record,
// the list of runs, the two work counters of the sort kernels and the error
// flag -- in one file-scope device array instead of cudaMalloc'ed memory.

namespace {

constexpr u32 NOALLOC_MAX_RUNS = 1024;

struct NoAllocScratch {
  Job job;
  u32 counters[8];  // [0] runs listed, [1] [2] work counters, [3] error flags
  Seg segs[NOALLOC_MAX_RUNS];
};

// Shared by every call on this device; it keeps the last call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

__global__ void k_noalloc_init(NoAllocScratch* sc, const Tuple* R, u64 nR, u32 runs) {
  if (threadIdx.x == 0) {
    Job J{};
    J.R = R;
    J.nR = nR;
    J.runs = runs;
    sc->job = J;
    sc->counters[1] = 0;
    sc->counters[2] = 0;
    sc->counters[3] = 0;
  }
  __syncthreads();
  for (u32 j = threadIdx.x; j < runs; j += blockDim.x) {
    const u64 a = (u64)(((unsigned __int128)nR * j) / runs);
    const u64 b = (u64)(((unsigned __int128)nR * (j + 1)) / runs);
    if (b > a)
      sc->segs[j] = Seg{a, b - a, 0ull, ~0ull, 0u, W_RIN};
    else
      sc->segs[j] = Seg{a, 0ull, 0ull, 0ull, 0u, W_RIN | SEG_EXACT};  // empty run: nothing to move
  }
  if (threadIdx.x == 0) sc->counters[0] = runs;
}

std::mutex g_noalloc_mu;
void* g_noalloc_addr[128];  // device address of the scratch array, per device ordinal

}  // namespace

}  // namespace mpsm

/* See include/mpsm.h.  The first call on a device looks up the scratch array's
 * device address (cudaGetSymbolAddress, with that device current) and sets the
 * sort kernels' shared-memory limits.  Every call reads the error flag back and
 * synchronises its stream, so none can run inside a stream capture.  Calls whose
 * work overlaps on the GPU share the array and race. */
extern "C" __attribute__((visibility("default"))) int mpsm_sort_runs_noalloc(const mpsm_tuple_t* R, uint64_t nR,
                                                                             uint32_t runs, mpsm_tuple_t* out,
                                                                             void* stream) {
  using namespace mpsm;
  if (runs == 0 || runs > NOALLOC_MAX_RUNS) return MPSM_ERR_INVALID_ARG;
  if (nR && (!R || !out)) return MPSM_ERR_INVALID_ARG;
  if ((((uintptr_t)R) | ((uintptr_t)out)) & 15u) return MPSM_ERR_INVALID_ARG;
  if ((nR + runs - 1) / runs > NMAX) return MPSM_ERR_INVALID_ARG;  // every run must fit one block
  if (nR == 0) return MPSM_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
    cudaGetLastError();
    return MPSM_ERR_CUDA;
  }
  NoAllocScratch* sc = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return MPSM_ERR_CUDA;
      }
      init_attrs_pass();
      g_noalloc_addr[dev] = ptr;
    }
    sc = reinterpret_cast<NoAllocScratch*>(g_noalloc_addr[dev]);
  }
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (nsm <= 0) nsm = 1;
  cudaStream_t st = (cudaStream_t)stream;
  k_noalloc_init<<<1, 1024, 0, st>>>(sc, reinterpret_cast<const Tuple*>(R), nR, runs);
  Bufs b{reinterpret_cast<Tuple*>(out), nullptr, nullptr};
  launch_seg_sort(sc->segs, &sc->counters[0], NOALLOC_MAX_RUNS, &sc->counters[1], b, &sc->job, W_XR,
                  &sc->counters[3], st, nsm);
  if (cudaGetLastError() != cudaSuccess) return MPSM_ERR_CUDA;
  u32 err = 0;
  if (cudaMemcpyAsync(&err, &sc->counters[3], sizeof(u32), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return MPSM_ERR_CUDA;
  }
  return err ? MPSM_ERR_DEVICE : MPSM_OK;
}
