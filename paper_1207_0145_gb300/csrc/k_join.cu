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
#include "mpsm_launch.h"

namespace mpsm {

namespace {

constexpr u32 NT_JOIN = 256;

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

__global__ void __launch_bounds__(1024) k_tiles(Job* jobs, u32 njobs, u32 tile, u64* totals) {
  __shared__ u64 s_warp[33];
  __shared__ u64 carry[2];
  if (threadIdx.x == 0) carry[0] = carry[1] = 0;
  __syncthreads();
  for (u32 base = 0; base < njobs; base += 1024) {
    const u32 i = base + threadIdx.x;
    u64 nt = 0, nw = 0;
    if (i < njobs) {
      nt = (jobs[i].s_kept + tile - 1) / tile;
      nw = nt * jobs[i].runs;
    }
    u64 t0, t1;
    const u64 p0 = block_exclusive_scan<u64, 1024>(nt, &t0, s_warp);
    const u64 p1 = block_exclusive_scan<u64, 1024>(nw, &t1, s_warp);
    if (i < njobs) {
      jobs[i].ntiles = nt;
      jobs[i].tile_base = carry[0] + p0;
      jobs[i].win_base = carry[1] + p1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      carry[0] += t0;
      carry[1] += t1;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    totals[0] = carry[0];
    totals[1] = carry[1];
  }
}

__global__ void k_search(const Job* jobs, u32 njobs, const Run* runs, const Tuple* xr, const Tuple* xs, u32 tile,
                         const u64* totals, u32* win) {
  const u64 nwin = totals[1];
  for (u64 q = (u64)blockIdx.x * blockDim.x + threadIdx.x; q < nwin; q += (u64)gridDim.x * blockDim.x) {
    const u32 ji = find_job(jobs, njobs, q, [](const Job& j) { return j.win_base; });
    const Job& J = jobs[ji];
    const u64 local = q - J.win_base;
    const u64 t = local / J.runs;
    const u32 j = (u32)(local - t * J.runs);
    const u64 s0 = J.s_base + t * tile;
    const u64 s_end = J.s_base + J.s_kept;
    const u64 s1 = (s0 + tile < s_end ? s0 + tile : s_end) - 1;
    const u64 klo = xs[s0].key, khi = xs[s1].key;
    const Run r = runs[J.run_base + j];
    const u64 lb = lower_bound_g(xr + r.off, r.len, klo);
    const u64 ub = lb + upper_bound_g(xr + r.off + lb, r.len - lb, khi);
    win[2 * q] = (u32)lb;
    win[2 * q + 1] = (u32)ub;
  }
}

template <u32 MODE>
__global__ void __launch_bounds__(NT_JOIN) k_join(Job* jobs, u32 njobs, const Run* runs, const Tuple* xr,
                                                  const Tuple* xs, u32 tile, const u64* totals, const u32* win,
                                                  u64* tile_cnt, const u64* tile_out, Tuple* pairs, u32* err) {
  extern __shared__ __align__(128) unsigned char sm_raw[];
  Tuple* tup = reinterpret_cast<Tuple*>(sm_raw);                 // TILE_MAX: key, payload prefix sum
  u64* roff = reinterpret_cast<u64*>(tup + TILE_MAX);            // RUNS_MAX
  u32* wl = reinterpret_cast<u32*>(roff + RUNS_MAX);             // RUNS_MAX window starts
  u32* wpre = wl + RUNS_MAX;                                     // RUNS_MAX + 1 window prefix
  __shared__ __align__(8) u64 mbar;
  __shared__ u64 s_warp[NT_JOIN / 32 + 1];
  __shared__ u32 s_warp32[NT_JOIN / 32 + 1];
  __shared__ u32 s_job;
  const u32 tid = threadIdx.x;
  if (tid == 0) mbar_init(&mbar, 1);
  __syncthreads();
  u32 phase = 0;
  const u64 ntiles = totals[0];
  for (u64 t = blockIdx.x; t < ntiles; t += gridDim.x) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (tid == 0) s_job = find_job(jobs, njobs, t, [](const Job& j) { return j.tile_base; });
    __syncthreads();
    const u32 ji = s_job;
    const Job& J = jobs[ji];
    const u64 lt = t - J.tile_base;
    const u64 s0 = lt * tile;
    const u32 n = (u32)((J.s_kept - s0) < tile ? (J.s_kept - s0) : tile);
    const u32 nruns = J.runs;
    if (tid == 0) tma_load_1d(tup, xs + J.s_base + s0, n * (u32)sizeof(Tuple), &mbar);
    // windows of this tile, one per run
    const u32* w = win + 2 * (J.win_base + lt * nruns);
    for (u32 j = tid; j < nruns; j += NT_JOIN) {
      const u32 a = w[2 * j], b = w[2 * j + 1];
      wl[j] = a;
      wpre[j] = b - a;
      roff[j] = runs[J.run_base + j].off;
    }
    const bool ok = mbar_wait(&mbar, phase, SPIN_LIMIT);
    phase ^= 1u;
    if (!__syncthreads_and(ok)) {
      if (tid == 0) atomicOr(err, (u32)DERR_TMA_TIMEOUT);
      return;
    }
    // payloads -> inclusive prefix sums (mod 2^64): warp w scans tuples
    // [w*512, (w+1)*512) 32 at a time (conflict-free), then warp offsets are added
    {
      constexpr u32 PERW = TILE_MAX / (NT_JOIN / 32);
      const u32 wid = warp_id(), lane = lane_id();
      u64 carry = 0;
#pragma unroll 4
      for (u32 i = 0; i < PERW / 32; ++i) {
        const u32 k = wid * PERW + i * 32 + lane;
        u64 v = k < n ? tup[k].pay : 0ull;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const u64 y = __shfl_up_sync(0xffffffffu, v, d);
          if (lane >= (u32)d) v += y;
        }
        v += carry;
        if (k < n) tup[k].pay = v;
        carry = __shfl_sync(0xffffffffu, v, 31);
      }
      if (lane == 0) s_warp[wid] = carry;
      __syncthreads();
      u64 add = 0;
      for (u32 w2 = 0; w2 < wid; ++w2) add += s_warp[w2];
      if (add) {
        for (u32 i = 0; i < PERW / 32; ++i) {
          const u32 k = wid * PERW + i * 32 + lane;
          if (k < n) tup[k].pay += add;
        }
      }
      __syncthreads();
    }
    const u32 W = smem_exclusive_scan<u32, NT_JOIN, RUNS_MAX / NT_JOIN>(wpre, nruns, s_warp32);
    if (tid == 0) wpre[nruns] = W;
    __syncthreads();
    u64 cnt = 0, chk = 0;
    u64 out_pos = 0;
    if (MODE == JOIN_WRITE) out_pos = J.pair_base + tile_out[t];
    const u32 rounds = (W + NT_JOIN - 1) / NT_JOIN;
    for (u32 rd = 0; rd < rounds; ++rd) {
      const u32 q = rd * NT_JOIN + tid;
      u32 lb = 0, ub = 0;
      Tuple r{0, 0};
      if (q < W) {
        u32 lo = 0, hi = nruns;  // run j: last with wpre[j] <= q
        while (hi - lo > 1) {
          const u32 mid = (lo + hi) >> 1;
          if (wpre[mid] <= q) lo = mid; else hi = mid;
        }
        const u64 pos = roff[lo] + wl[lo] + (q - wpre[lo]);
        r = ld_stream(xr + pos);
        // equal-key range of r.key in the tile
        u32 a = 0, m = n;
        while (m > 0) {
          const u32 h = m >> 1;
          if (tup[a + h].key < r.key) {
            a += h + 1;
            m -= h + 1;
          } else {
            m = h;
          }
        }
        lb = a;
        m = n - a;
        while (m > 0) {
          const u32 h = m >> 1;
          if (tup[a + h].key <= r.key) {
            a += h + 1;
            m -= h + 1;
          } else {
            m = h;
          }
        }
        ub = a;
        const u64 c = ub - lb;
        if (c) {
          const u64 ps_ub = tup[ub - 1].pay;
          const u64 ps_lb = lb ? tup[lb - 1].pay : 0ull;
          cnt += c;
          chk += c * r.pay + (ps_ub - ps_lb);
        }
      }
      if (MODE == JOIN_WRITE) {
        u32 tot;
        const u32 pre = block_exclusive_scan<u32, NT_JOIN>(ub - lb, &tot, s_warp32);
        Tuple* o = pairs + out_pos + pre;
        for (u32 i = lb; i < ub; ++i) {
          const u64 sp = tup[i].pay - (i ? tup[i - 1].pay : 0ull);
          st_tuple(o + (i - lb), Tuple{r.pay, sp});
        }
        out_pos += tot;
      }
    }
    cnt = warp_sum(cnt);
    chk = warp_sum(chk);
    if (lane_id() == 0) {
      s_warp[warp_id()] = cnt;
    }
    __syncthreads();
    if (tid == 0) {
      u64 c = 0;
      for (u32 i = 0; i < NT_JOIN / 32; ++i) c += s_warp[i];
      cnt = c;
    }
    __syncthreads();
    if (lane_id() == 0) s_warp[warp_id()] = chk;
    __syncthreads();
    if (tid == 0) {
      u64 k = 0;
      for (u32 i = 0; i < NT_JOIN / 32; ++i) k += s_warp[i];
      if (MODE == JOIN_COUNT) tile_cnt[t] = cnt;
      if (MODE != JOIN_WRITE) {
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

constexpr size_t SMEM_JOIN = TILE_MAX * sizeof(Tuple) + RUNS_MAX * sizeof(u64) + (2 * RUNS_MAX + 1) * sizeof(u32);

}  // namespace

void init_attrs_join() {
  cudaFuncSetAttribute(k_join<JOIN_AGG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_JOIN);
  cudaFuncSetAttribute(k_join<JOIN_COUNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_JOIN);
  cudaFuncSetAttribute(k_join<JOIN_WRITE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_JOIN);
}

void launch_tiles(Job* jobs, u32 njobs, u32 tile, u64* totals, cudaStream_t st) {
  k_tiles<<<1, 1024, 0, st>>>(jobs, njobs, tile, totals);
}

void launch_search(const Job* jobs, u32 njobs, const Run* runs, const Tuple* xr, const Tuple* xs, u32 tile,
                   const u64* totals, u32* win, cudaStream_t st, int nsm) {
  k_search<<<nsm * 8, 256, 0, st>>>(jobs, njobs, runs, xr, xs, tile, totals, win);
}

void launch_join(u32 mode, Job* jobs, u32 njobs, const Run* runs, const Tuple* xr, const Tuple* xs, u32 tile,
                 const u64* totals, const u32* win, u64* tile_cnt, const u64* tile_out, Tuple* pairs, u32* err,
                 cudaStream_t st, int nsm) {
  const int grid = nsm * 3;
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

void launch_pair_offsets(Job* jobs, u32 njobs, const u64* totals, const u64* tile_cnt, u64* tile_out,
                         u64* pair_total, cudaStream_t st) {
  k_pair_offsets<<<1, 1024, 0, st>>>(jobs, njobs, totals, tile_cnt, tile_out, pair_total);
}

}  // namespace mpsm
