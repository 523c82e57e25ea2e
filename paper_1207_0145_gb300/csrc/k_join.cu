// k_join.cu -- phase 4 of MPSM: locate each run's relevant part, then join.
//
// After phase 3 the kept S tuples of a job are sorted (partitions are disjoint
// key ranges in key order, each sorted).  They are cut into tiles of `tile`
// tuples.  For every (tile, R run) pair the search step finds the run's window
// [first key >= tile's first key, first key > tile's last key) (Sec. 3.2.2: the
// search for the start of the merge; binary search here, the learned model in
// k_learn.cu).  The join step stages one S tile in shared memory (bulk async
// copy), turns its payloads into prefix sums, and streams every run window
// through it: each R tuple r finds its equal-key range [lb, ub) in the tile by
// binary search, contributing ub - lb pairs and (ub - lb) * r.payload + (sum of
// S payloads in [lb, ub)) to the checksum.  Each R tuple is read once per tile
// whose key range covers it and each S tuple once, so the S side is never
// rescanned per run (the T*|S| term of the paper's cost is avoided by staging).
#include "mpsm_internal.cuh"
#include "learn.cuh"
#include "mpsm_launch.h"

namespace mpsm {

namespace {

constexpr u32 NT_JOIN = 512;

__device__ __forceinline__ u64 lower_bound_g(const Tuple* a, u64 n, u64 key) {
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

__device__ __forceinline__ u64 upper_bound_g(const Tuple* a, u64 n, u64 key) {
  u64 lo = 0;
  while (n > 0) {
    const u64 h = n >> 1;
    if (a[lo + h].key <= key) {
      lo += h + 1;
      n -= h + 1;
    } else {
      n = h;
    }
  }
  return lo;
}

// last job i with field(i) <= q
template <typename F>
__device__ __forceinline__ u32 find_job(const Job* jobs, u32 njobs, u64 q, F field) {
  u32 lo = 0, hi = njobs;
  while (hi - lo > 1) {
    const u32 mid = (lo + hi) >> 1;
    if (field(jobs[mid]) <= q) lo = mid; else hi = mid;
  }
  return lo;
}

// A device check that failed earlier in the call (err != 0) may have left S or the
// runs unsorted: then no tile is searched or joined (the call reports the error).
__global__ void __launch_bounds__(1024) k_tiles(Job* jobs, u32 njobs, u32 tile, u64* totals, const u32* err) {
  __shared__ u64 s_warp[33];
  __shared__ u64 carry[3];
  if (threadIdx.x == 0) carry[0] = carry[1] = carry[2] = 0;
  if (*err) {
    if (threadIdx.x == 0) totals[0] = totals[1] = totals[2] = 0;
    return;
  }
  __syncthreads();
  for (u32 base = 0; base < njobs; base += 1024) {
    const u32 i = base + threadIdx.x;
    u64 nt = 0, nw = 0, ns = 0;
    if (i < njobs) {
      nt = (jobs[i].s_kept + tile - 1) / tile;
      nw = nt * jobs[i].runs;
      ns = ((nt + SEARCH_TB - 1) / SEARCH_TB) * jobs[i].runs;
    }
    u64 t0, t1, t2;
    const u64 p0 = block_exclusive_scan<u64, 1024>(nt, &t0, s_warp);
    const u64 p1 = block_exclusive_scan<u64, 1024>(nw, &t1, s_warp);
    const u64 p2 = block_exclusive_scan<u64, 1024>(ns, &t2, s_warp);
    if (i < njobs) {
      jobs[i].ntiles = nt;
      jobs[i].tile_base = carry[0] + p0;
      jobs[i].win_base = carry[1] + p1;
      jobs[i].search_base = carry[2] + p2;
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
    totals[0] = carry[0];
    totals[1] = carry[1];
    totals[2] = carry[2];
  }
}

// first i >= from with a[i].key >= key; the answer is known to be >= from
__device__ __forceinline__ u64 gallop_lower(const Tuple* a, u64 n, u64 from, u64 key) {
  if (from >= n || a[from].key >= key) return from;
  u64 lo = from, step = 1;  // a[lo].key < key
  while (lo + step < n && a[lo + step].key < key) {
    lo += step;
    step <<= 1;
  }
  const u64 hi = (lo + step < n) ? lo + step : n;
  return lo + 1 + lower_bound_g(a + lo + 1, hi - lo - 1, key);
}

// first i >= from with a[i].key > key; the answer is known to be >= from
__device__ __forceinline__ u64 gallop_upper(const Tuple* a, u64 n, u64 from, u64 key) {
  if (from >= n || a[from].key > key) return from;
  u64 lo = from, step = 1;  // a[lo].key <= key
  while (lo + step < n && a[lo + step].key <= key) {
    lo += step;
    step <<= 1;
  }
  const u64 hi = (lo + step < n) ? lo + step : n;
  return lo + 1 + upper_bound_g(a + lo + 1, hi - lo - 1, key);
}

// One thread per (job, run, block of SEARCH_TB consecutive tiles): a full binary
// search for the block's first tile, then galloping forward from the previous
// window, since tile key ranges are increasing (Sec. 3.2.2's start search,
// reusing each result as the next one's lower limit).
__global__ void k_search(const Job* jobs, u32 njobs, const Run* runs, const Tuple* xr, const Tuple* xs, u32 tile,
                         const u64* totals, u32* win, LearnCtx lc) {
  const u64 nitems = totals[2];
  u32 probes = 0, nsearch = 0;
  u64 err_sum = 0;
  for (u64 q = (u64)blockIdx.x * blockDim.x + threadIdx.x; q < nitems; q += (u64)gridDim.x * blockDim.x) {
    const u32 ji = find_job(jobs, njobs, q, [](const Job& j) { return j.search_base; });
    const Job& J = jobs[ji];
    const u64 nblk = (J.ntiles + SEARCH_TB - 1) / SEARCH_TB;
    const u64 local = q - J.search_base;
    const u32 j = (u32)(local / nblk);
    const u64 k = local - (u64)j * nblk;
    const u64 t0 = k * SEARCH_TB;
    const u64 t1 = (t0 + SEARCH_TB < J.ntiles) ? t0 + SEARCH_TB : J.ntiles;
    const Run r = runs[J.run_base + j];
    const Tuple* a = xr + r.off;
    const u64 s_end = J.s_base + J.s_kept;
    u64 lb = 0;
    for (u64 t = t0; t < t1; ++t) {
      const u64 s0 = J.s_base + t * tile;
      const u64 s1 = (s0 + tile < s_end ? s0 + tile : s_end) - 1;
      const u64 klo = xs[s0].key, khi = xs[s1].key;
      if (t != t0) {
        lb = gallop_lower(a, r.len, lb, klo);
      } else if (lc.models) {
        // learned start: the R-side model's CDF value times the run length, then an
        // exact exponential + binary search from there
        u64 g = (u64)(rmi_predict(&lc.models[2 * ji + 1], klo) * (float)r.len);
        if (g > r.len) g = r.len;
        auto at = [&](u64 i) { return a[i].key; };
        lb = gallop_from(at, r.len, g, klo, probes);
        err_sum += g > lb ? g - lb : lb - g;
        ++nsearch;
      } else if (lc.interp) {
        auto at = [&](u64 i) { return a[i].key; };
        lb = interp_lower_bound(at, r.len, klo, probes);
        ++nsearch;
      } else {
        lb = lower_bound_g(a, r.len, klo);
        probes += bitlen64(r.len);
        ++nsearch;
      }
      const u64 ub = gallop_upper(a, r.len, lb, khi);
      const u64 w = J.win_base + t * J.runs + j;
      win[2 * w] = (u32)lb;
      win[2 * w + 1] = (u32)ub;
    }
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

// first index in [lb, n) whose key differs from `key` (keys[lb] == key): a short
// forward scan, four independent probes at a time, then binary search for long runs
__device__ __forceinline__ u32 equal_run_end(const u64* keys, u32 n, u32 lb, u64 key) {
  u32 ub = lb + 1;
#pragma unroll
  for (int rep = 0; rep < 2; ++rep) {
    const bool m0 = ub < n && keys[ub] == key;
    const bool m1 = ub + 1 < n && keys[ub + 1] == key;
    const bool m2 = ub + 2 < n && keys[ub + 2] == key;
    const bool m3 = ub + 3 < n && keys[ub + 3] == key;
    if (!m0) return ub;
    if (!m1) return ub + 1;
    if (!m2) return ub + 2;
    if (!m3) return ub + 3;
    ub += 4;
  }
  u32 m = n - ub;  // long run of equal keys: binary search for its end
  while (m > 0) {
    const u32 h = m >> 1;
    if (keys[ub + h] <= key) {
      ub += h + 1;
      m -= h + 1;
    } else {
      m = h;
    }
  }
  return ub;
}

__device__ __forceinline__ u32 lower_bound_s(const u64* keys, u32 n, u64 key) {
  u32 a = 0, m = n;
  while (m > 0) {
    const u32 h = m >> 1;
    if (keys[a + h] < key) {
      a += h + 1;
      m -= h + 1;
    } else {
      m = h;
    }
  }
  return a;
}

// One S tile per iteration: keys and inclusive payload prefix sums in shared
// memory (structure of arrays), then every R tuple of the tile's run windows
// looks up its equal-key range [lb, ub) in the tile.
template <u32 MODE>
__global__ void __launch_bounds__(NT_JOIN, 2) k_join(Job* jobs, u32 njobs, const Run* runs, const Tuple* xr,
                                                     const Tuple* xs, u32 tile, const u64* totals, const u32* win,
                                                     u64* tile_cnt, const u64* tile_out, Tuple* pairs, u32* err) {
  constexpr u32 IT = TILE_MAX / NT_JOIN;  // 8
  constexpr u32 NW = NT_JOIN / 32;
  extern __shared__ __align__(128) unsigned char sm_raw[];
  u64* keys = reinterpret_cast<u64*>(sm_raw);          // TILE_MAX
  u64* psum = keys + TILE_MAX;                         // TILE_MAX inclusive prefix sums of payloads
  u64* roff = psum + TILE_MAX;                         // RUNS_MAX
  u32* wl = reinterpret_cast<u32*>(roff + RUNS_MAX);   // RUNS_MAX window starts
  u32* wpre = wl + RUNS_MAX;                           // RUNS_MAX + 1 window prefix
  u16* dir = reinterpret_cast<u16*>(wpre + RUNS_MAX + 1);  // TILE_MAX + 1 bucket starts
  __shared__ u64 s_warp[NW + 1];
  __shared__ u32 s_warp32[NW + 1];
  __shared__ u32 s_job;
  const u32 tid = threadIdx.x, lane = lane_id(), wid = warp_id();
  const u64 ntiles = totals[0];
  for (u64 t = blockIdx.x; t < ntiles; t += gridDim.x) {
    if (tid == 0) s_job = find_job(jobs, njobs, t, [](const Job& j) { return j.tile_base; });
    __syncthreads();
    const u32 ji = s_job;
    const Job& J = jobs[ji];
    const u64 lt = t - J.tile_base;
    const u64 s0 = lt * tile;
    const u32 n = (u32)((J.s_kept - s0) < tile ? (J.s_kept - s0) : tile);
    const u32 nruns = J.runs;
    const Tuple* stile = xs + J.s_base + s0;
    Tuple v[IT];
#pragma unroll
    for (u32 i = 0; i < IT; ++i) {
      const u32 k = i * NT_JOIN + tid;
      if (k < n) v[i] = ld_stream(stile + k);
    }
    const u32* w = win + 2 * (J.win_base + lt * nruns);
    for (u32 j = tid; j < nruns; j += NT_JOIN) {
      const u32 a = w[2 * j], b = w[2 * j + 1];
      wl[j] = a;
      wpre[j] = b - a;
      roff[j] = runs[J.run_base + j].off;
    }
#pragma unroll
    for (u32 i = 0; i < IT; ++i) {
      const u32 k = i * NT_JOIN + tid;
      if (k < n) {
        keys[k] = v[i].key;
        psum[k] = v[i].pay;
      }
    }
    __syncthreads();
    // inclusive prefix sums (mod 2^64): warp w scans entries [w*PERW, (w+1)*PERW)
    {
      constexpr u32 PERW = TILE_MAX / NW;
      u64 carry = 0;
#pragma unroll
      for (u32 i = 0; i < PERW / 32; ++i) {
        const u32 k = wid * PERW + i * 32 + lane;
        u64 x = k < n ? psum[k] : 0ull;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const u64 y = __shfl_up_sync(0xffffffffu, x, d);
          if (lane >= (u32)d) x += y;
        }
        x += carry;
        if (k < n) psum[k] = x;
        carry = __shfl_sync(0xffffffffu, x, 31);
      }
      if (lane == 0) s_warp[wid] = carry;
      __syncthreads();
      u64 add = 0;
      for (u32 w2 = 0; w2 < wid; ++w2) add += s_warp[w2];
      if (add) {
#pragma unroll
        for (u32 i = 0; i < PERW / 32; ++i) {
          const u32 k = wid * PERW + i * 32 + lane;
          if (k < n) psum[k] += add;
        }
      }
    }
    // order-preserving bucket directory over the tile's key range: bucket i of
    // (key - kmin) >> dsh starts at dir[i]; dir[nbk] = n
    const u64 kmin = keys[0], kmax = keys[n - 1];
    const u32 rbits = bitlen64(kmax - kmin);
    const u32 dsh = rbits > 12u ? rbits - 12u : 0u;
    const u32 nbk = (u32)((kmax - kmin) >> dsh) + 1u;
#pragma unroll
    for (u32 i = 0; i < IT; ++i) {
      const u32 k = i * NT_JOIN + tid;
      if (k < n) {
        // the tile is sorted, so every key lies in [kmin, kmax]; the clamp keeps the
        // writes inside the nbk + 1 entries even if it were not
        auto bucket = [&](u32 e) {
          const u64 d = (keys[e] - kmin) >> dsh;
          return d < (u64)nbk ? (u32)d : nbk - 1u;
        };
        const u32 b = bucket(k);
        const u32 bp = k ? bucket(k - 1) : 0u;
        for (u32 x = (k ? bp + 1u : 0u); x <= b; ++x) dir[x] = (u16)k;
        if (k == n - 1)
          for (u32 x = b + 1u; x <= nbk; ++x) dir[x] = (u16)n;
      }
    }
    const u32 W = smem_exclusive_scan<u32, NT_JOIN, (RUNS_MAX + NT_JOIN - 1) / NT_JOIN>(wpre, nruns, s_warp32);
    if (tid == 0) wpre[nruns] = W;
    __syncthreads();
    u64 cnt = 0, chk = 0;
    if (MODE != JOIN_WRITE) {
      constexpr u32 U = 4;  // R loads in flight per thread before the tile lookups
      for (u32 q0 = 0; q0 < W; q0 += NT_JOIN * U) {
        Tuple r[U];
#pragma unroll
        for (u32 u = 0; u < U; ++u) {
          const u32 q = q0 + u * NT_JOIN + tid;
          r[u].key = 0;
          r[u].pay = 0;
          if (q < W) {
            u32 lo = 0, hi = nruns;  // run j: last with wpre[j] <= q
            while (hi - lo > 1) {
              const u32 mid = (lo + hi) >> 1;
              if (wpre[mid] <= q) lo = mid; else hi = mid;
            }
            r[u] = ld_stream(xr + roff[lo] + wl[lo] + (q - wpre[lo]));
          }
        }
#pragma unroll
        for (u32 u = 0; u < U; ++u) {
          const u32 q = q0 + u * NT_JOIN + tid;
          if (q >= W) continue;
          const u64 key = r[u].key;
          if (key < kmin || key > kmax) continue;
          const u32 bi = (u32)((key - kmin) >> dsh);
          u32 lb = dir[bi], ub = dir[bi + 1];
          if (ub <= lb) continue;  // an empty bucket (the directory is non-decreasing)
          if (dsh) {  // a bucket spans several keys: narrow [lb, ub) to `key`
            lb += lower_bound_s(keys + lb, ub - lb, key);
            if (lb >= ub || keys[lb] != key) continue;
            ub = equal_run_end(keys, ub, lb, key);
          }
          if (lb >= ub) continue;
          const u64 c = ub - lb;
          cnt += c;
          chk += c * r[u].pay + (psum[ub - 1] - (lb ? psum[lb - 1] : 0ull));
        }
      }
    } else {
      u64 out_pos = J.pair_base + tile_out[t];
      const u32 rounds = (W + NT_JOIN - 1) / NT_JOIN;
      for (u32 rd = 0; rd < rounds; ++rd) {
        const u32 q = rd * NT_JOIN + tid;
        u32 lb = 0, ub = 0;
        Tuple r{0, 0};
        if (q < W) {
          u32 lo = 0, hi = nruns;
          while (hi - lo > 1) {
            const u32 mid = (lo + hi) >> 1;
            if (wpre[mid] <= q) lo = mid; else hi = mid;
          }
          r = ld_stream(xr + roff[lo] + wl[lo] + (q - wpre[lo]));
          if (r.key >= kmin && r.key <= kmax) {
            const u32 bi = (u32)((r.key - kmin) >> dsh);
            lb = dir[bi];
            ub = dir[bi + 1];
            if (ub < lb) ub = lb;
            if (dsh) {
              lb += lower_bound_s(keys + lb, ub - lb, r.key);
              ub = (lb < ub && keys[lb] == r.key) ? equal_run_end(keys, ub, lb, r.key) : lb;
            }
          }
        }
        u32 tot;
        const u32 pre = block_exclusive_scan<u32, NT_JOIN>(ub - lb, &tot, s_warp32);
        Tuple* o = pairs + out_pos + pre;
        for (u32 i = lb; i < ub; ++i) {
          const u64 sp = psum[i] - (i ? psum[i - 1] : 0ull);
          st_tuple(o + (i - lb), Tuple{r.pay, sp});
        }
        out_pos += tot;
      }
    }
    if (MODE != JOIN_WRITE) {
      cnt = warp_sum(cnt);
      chk = warp_sum(chk);
      if (lane == 0) s_warp[wid] = cnt;
      __syncthreads();
      if (tid == 0) {
        u64 c = 0;
        for (u32 i = 0; i < NW; ++i) c += s_warp[i];
        cnt = c;
      }
      __syncthreads();
      if (lane == 0) s_warp[wid] = chk;
      __syncthreads();
      if (tid == 0) {
        u64 k = 0;
        for (u32 i = 0; i < NW; ++i) k += s_warp[i];
        if (MODE == JOIN_COUNT) tile_cnt[t] = cnt;
        atomicAdd(&jobs[ji].count, cnt);
        atomicAdd(&jobs[ji].checksum, k);
      }
    }
    __syncthreads();
  }
}

// exclusive scan of per-tile pair counts over all tiles (pairs mode, job 0)
__global__ void __launch_bounds__(1024) k_pair_offsets(Job* jobs, u32 njobs, const u64* totals, const u64* tile_cnt,
                                                       u64* tile_out, u64* pair_total) {
  __shared__ u64 s_warp[33];
  __shared__ u64 carry;
  const u64 n = totals[0];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (u64 base = 0; base < n; base += 1024) {
    const u64 i = base + threadIdx.x;
    const u64 v = i < n ? tile_cnt[i] : 0;
    u64 tot;
    const u64 p = block_exclusive_scan<u64, 1024>(v, &tot, s_warp);
    if (i < n) tile_out[i] = carry + p;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *pair_total = carry;
    for (u32 j = 0; j < njobs; ++j) jobs[j].pair_base = 0;
  }
}

constexpr size_t SMEM_JOIN = 2 * TILE_MAX * sizeof(u64) + RUNS_MAX * sizeof(u64) + (2 * RUNS_MAX + 1) * sizeof(u32) +
                             (TILE_MAX + 8) * sizeof(u16);

}  // namespace

void init_attrs_join() {
  cudaFuncSetAttribute(k_join<JOIN_AGG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_JOIN);
  cudaFuncSetAttribute(k_join<JOIN_COUNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_JOIN);
  cudaFuncSetAttribute(k_join<JOIN_WRITE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_JOIN);
  cudaFuncSetAttribute(k_join<JOIN_AGG>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  cudaFuncSetAttribute(k_join<JOIN_COUNT>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  cudaFuncSetAttribute(k_join<JOIN_WRITE>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

void launch_tiles(Job* jobs, u32 njobs, u32 tile, u64* totals, const u32* err, cudaStream_t st) {
  k_tiles<<<1, 1024, 0, st>>>(jobs, njobs, tile, totals, err);
}

void launch_search(const Job* jobs, u32 njobs, const Run* runs, const Tuple* xr, const Tuple* xs, u32 tile,
                   const u64* totals, u32* win, const LearnCtx& lc, cudaStream_t st, int nsm) {
  k_search<<<nsm * 8, 256, 0, st>>>(jobs, njobs, runs, xr, xs, tile, totals, win, lc);
}

void launch_join(u32 mode, Job* jobs, u32 njobs, const Run* runs, const Tuple* xr, const Tuple* xs, u32 tile,
                 const u64* totals, const u32* win, u64* tile_cnt, const u64* tile_out, Tuple* pairs, u32* err,
                 cudaStream_t st, int nsm) {
  const int grid = nsm * 2;
  if (mode == JOIN_AGG) {
    k_join<JOIN_AGG><<<grid, NT_JOIN, SMEM_JOIN, st>>>(jobs, njobs, runs, xr, xs, tile, totals, win, tile_cnt,
                                                       tile_out, pairs, err);
  } else if (mode == JOIN_COUNT) {
    k_join<JOIN_COUNT><<<grid, NT_JOIN, SMEM_JOIN, st>>>(jobs, njobs, runs, xr, xs, tile, totals, win, tile_cnt,
                                                         tile_out, pairs, err);
  } else {
    k_join<JOIN_WRITE><<<grid, NT_JOIN, SMEM_JOIN, st>>>(jobs, njobs, runs, xr, xs, tile, totals, win, tile_cnt,
                                                         tile_out, pairs, err);
  }
}

// (a, b) -> (b, a) for n pairs (role reversal: the run side wrote its payload first)
__global__ void k_swap_pairs(Tuple* pairs, u64 n) {
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
    const Tuple t = pairs[i];
    st_tuple(pairs + i, Tuple{t.pay, t.key});
  }
}

void launch_swap_pairs(Tuple* pairs, u64 n, cudaStream_t st, int nsm) {
  if (n) k_swap_pairs<<<nsm * 8, 256, 0, st>>>(pairs, n);
}

// One block waits on a shared-memory barrier that no copy will complete: the bounded
// wait every kernel uses gives up after `limit` polls and the block reports it.
__global__ void k_wait_selftest(u32* flag, u32 limit) {
  __shared__ __align__(8) u64 bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0, limit);
  if (!__syncthreads_and(ok) && threadIdx.x == 0) atomicOr(flag, (u32)DERR_TMA_TIMEOUT);
}

void launch_wait_selftest(u32* flag, u32 limit, cudaStream_t st) { k_wait_selftest<<<1, 32, 0, st>>>(flag, limit); }

void launch_pair_offsets(Job* jobs, u32 njobs, const u64* totals, const u64* tile_cnt, u64* tile_out,
                         u64* pair_total, cudaStream_t st) {
  k_pair_offsets<<<1, 1024, 0, st>>>(jobs, njobs, totals, tile_cnt, tile_out, pair_total);
}

}  // namespace mpsm
