// mpsm_internal.cuh -- device data structures and helpers shared by the MPSM kernels.
//
// Data layout in HBM (all tuples 16-byte {key, payload} records):
//   xr : the R runs after phase 1, back to back (run g of job i at runs[g].off)
//   xs : S after phase 2 (partitions back to back, tuples outside R's key range
//        dropped) and, after phase 3, the same ranges sorted
//   y  : ping-pong buffer of the radix passes (shared by phases 1 and 3)
// A "segment" is a contiguous key-ordered slice still to be sorted; radix
// passes split segments into children until they fit a thread block's shared
// memory, where a final in-SMEM sort finishes them.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mpsm {

typedef unsigned long long u64;
typedef unsigned int u32;
typedef unsigned short u16;

struct __align__(16) Tuple {
  u64 key, pay;
};

// ---------------------------------------------------------------- constants
constexpr u32 NMAX = 8192;        // tuples one block sorts in shared memory (128 KB)
constexpr u32 N_LEAF = 4096;      // target segment size after a radix pass
// tuples per bucket that the radix passes before the fused sort-and-join aim for:
// 7/8 of its N_LEAF-tuple tile, so the spread of uniform keys (about sqrt(3584) =
// 60) stays far below the tile and a segment is joined in one piece
constexpr u64 FILL_FUSED = N_LEAF - N_LEAF / 16;
constexpr u32 F_MIN = 16;         // smallest radix fan-out (guarantees 4 bits/pass progress)
constexpr u32 F_MAX = 2048;       // largest radix fan-out (radix_bits <= 11)
constexpr u32 FINE_MAX = 4096;    // largest fine histogram (fine_bits <= 12)
constexpr u32 P_MAX = 2048;       // largest number of S partitions
constexpr u32 RUNS_MAX = 1024;    // largest T_R per job
constexpr u32 TILE_MAX = 4096;    // largest join tile
constexpr u32 MAX_LEVELS = 16;    // radix passes of 4..11 bits cover any 64-bit key range
constexpr u32 SEARCH_TB = 32;     // consecutive tiles one search thread walks through per run

// where a segment's tuples live
enum Where : u32 { W_RIN = 0, W_SIN = 1, W_XR = 2, W_XS = 3, W_Y = 4 };
// segment flag bits above the 3-bit `where`
constexpr u32 SEG_EXACT = 8u;     // every key of the segment lies in [kmin, kmax] (the extremes, or the
                                  // key range of the bucket that made it)

// bucket functions of a partitioning pass
// MODE_RLEARN: a sort pass over the runs whose bucket function is the run side's
// sample quantiles (RunLearn in learn.cuh) instead of equal-width key ranges
enum PassMode : u32 { MODE_RADIX = 0, MODE_FINE = 1, MODE_SPLIT = 2, MODE_LEARN = 3, MODE_RLEARN = 4 };

// device-side error flags (bit set)
enum DevErr : u32 {
  DERR_SEG_OVERFLOW = 1u,   // a work list ran out of capacity
  DERR_SEG_TOO_BIG = 2u,    // a final segment larger than NMAX reached the SMEM sort
  DERR_TMA_TIMEOUT = 4u,    // a bulk copy did not complete within the spin limit
  DERR_LEVELS = 8u,         // radix levels exhausted with big segments left
  DERR_HIST_OVERFLOW = 16u, // a pass needed more histogram entries than allocated
  DERR_LEARN = 32u,         // learned model invariant (prediction window) violated
  DERR_BOUNDS = 64u         // an index check inside a kernel failed (the access was skipped)
};

struct Job {
  const Tuple* R;
  const Tuple* S;
  u64 nR, nS;
  u64 r_base, s_base;       // offsets of this job's region in xr / xs / y
  u32 runs, run_base;       // T_R and the job's first global run index
  u32 parts_req, part_base; // requested P; first global partition index (job * P_MAX)
  u32 fine_bits, fine_base; // B; first global fine-bucket index (job * FINE_MAX)
  // written on the device
  u64 kmin, kmax;           // R's key range
  u32 has_range;            // R non-empty
  u32 fine_shift, nfine;    // fine bucket = (key - kmin) >> fine_shift, < nfine
  u32 parts;                // P used
  u64 s_kept;               // S tuples inside [kmin, kmax]
  u64 tile_base, ntiles;    // global index of the job's first join tile; its tile count
  u64 win_base;             // first window entry of the job (tiles * runs pairs before it)
  u64 search_base;          // first search work item of the job (runs x tile blocks)
  u64 count, checksum;      // result
  u64 pair_base;            // first output pair of the job (pairs mode)
};

struct Run {
  u64 off;                  // offset in xr (and in the job's R input: off - r_base)
  u64 len;
};

struct Seg {
  u64 off, len;             // global offset in the buffer family of its side
  u64 kmin, kmax;           // bounds on the keys (exact when SEG_EXACT)
  u32 job;
  u32 flags;                // Where | SEG_EXACT
};

// per big segment of one partitioning pass
struct LSeg {
  u64 lo;                   // key origin of the bucket function
  u64 chunk_base;           // first global chunk of the segment
  u64 hist_base;            // first histogram entry (chunks x F, chunk-major)
  u64 bucket_base;          // first bucket-bound entry (F)
  u32 shift, F;             // bucket = min(F-1, (key - lo) >> shift), or with mul set:
  u32 nchunks;
  u32 nominal;              // MODE_RADIX on dense keys: buckets 1..F-2 take the key range their
                            // bucket function gives them instead of their keys' exact extremes
  u64 mul;                  // bucket = min(F-1, mulhi(key - lo, mul)) (MODE_RADIX)
};

// Phases 3 and 4 fused: the final sort of each S segment joins it, still in
// shared memory, against the window of every R run that can hold its keys.
struct FuseCtx {
  const u32* swin;          // per (segment, run): window [lo, hi) in the run; segment-major, stride maxT
  u32 maxT;                 // largest T_R of the call's jobs
  const Run* runs;
  const Tuple* xr;          // the sorted runs
  Job* jobs;                // count and checksum accumulate here
};

// pointer table of the buffers a segment may live in
struct Bufs {
  Tuple* xr;
  Tuple* xs;
  Tuple* y;
};

__device__ __forceinline__ const Tuple* seg_src(const Bufs& b, const Job* jobs, u32 where, u32 job, u64 off) {
  switch (where) {
    case W_RIN: return jobs[job].R + (off - jobs[job].r_base);
    case W_SIN: return jobs[job].S + (off - jobs[job].s_base);
    case W_XR: return b.xr + off;
    case W_XS: return b.xs + off;
    default: return b.y + off;
  }
}

__host__ __device__ __forceinline__ u32 bitlen64(u64 x) {
#if defined(__CUDA_ARCH__)
  return 64u - (u32)__clzll((long long)x);
#else
  return x ? 64u - (u32)__builtin_clzll(x) : 0u;
#endif
}

__device__ __forceinline__ u32 lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ u32 warp_id() { return threadIdx.x >> 5; }

// ---------------------------------------------------------------- block scans
// Exclusive scan of one value per thread; returns the prefix and (via *total) the block sum.
template <typename T, int NT>
__device__ __forceinline__ T block_exclusive_scan(T v, T* total, T* s_warp /* >= NT/32 + 1 */) {
  const u32 lane = lane_id(), wid = warp_id();
  T x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= (u32)d) x += y;
  }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    T w = (lane < (u32)(NT / 32)) ? s_warp[lane] : T(0);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= (u32)d) w += y;
    }
    if (lane < (u32)(NT / 32)) s_warp[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  const T warp_prefix = wid ? s_warp[wid - 1] : T(0);
  const T tot = s_warp[NT / 32 - 1];
  __syncthreads();
  *total = tot;
  return warp_prefix + x - v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v);

// Exclusive scan over the block with one barrier: every warp scans its values, then
// sums the totals of the warps before it (and of all warps) from shared memory on its
// own.  The caller must pass a barrier before s_warp is written again.
template <typename T, int NT>
__device__ __forceinline__ T block_exclusive_scan_1b(T v, T* total, T* s_warp /* >= NT/32 */) {
  static_assert(NT / 32 <= 32, "one warp sums the warp totals");
  const u32 lane = lane_id(), wid = warp_id();
  T x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= (u32)d) x += y;
  }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  T before = 0, all = 0;
  if (lane < (u32)(NT / 32)) {
    all = s_warp[lane];
    before = lane < wid ? all : T(0);
  }
  before = warp_sum(before);
  *total = warp_sum(all);
  return before + x - v;
}

// In-place exclusive scan of n <= NT*ITEMS u32/u64 values in shared memory.
template <typename T, int NT, int ITEMS>
__device__ __forceinline__ T smem_exclusive_scan(T* a, u32 n, T* s_warp) {
  T loc[ITEMS];
  T sum = 0;
  const u32 base = threadIdx.x * ITEMS;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const u32 k = base + i;
    loc[i] = k < n ? a[k] : T(0);
    sum += loc[i];
  }
  T total;
  T pre = block_exclusive_scan_1b<T, NT>(sum, &total, s_warp);
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const u32 k = base + i;
    if (k < n) a[k] = pre;
    pre += loc[i];
  }
  __syncthreads();  // the scanned values are visible, and s_warp may be written again
  return total;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

// ---------------------------------------------------------------- bulk async copy (TMA)
__device__ __forceinline__ u32 smem_u32(const void* p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(u64* bar, u32 count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One elected thread: expect `bytes` and start a bulk global->shared copy.
// dst, src 16-byte aligned; bytes a multiple of 16 and < 2^20.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, u32 bytes, u64* bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Wait for phase `parity` of the barrier; gives up after `limit` polls.
__device__ __forceinline__ bool mbar_wait(u64* bar, u32 parity, u32 limit) {
  const u32 a = smem_u32(bar);
  for (u32 it = 0; it < limit; ++it) {
    u32 done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

constexpr u32 SPIN_LIMIT = 1u << 26;

// streaming 16-byte load (read once; do not keep in L2)
__device__ __forceinline__ Tuple ld_stream(const Tuple* p) {
  longlong2 v = __ldcs(reinterpret_cast<const longlong2*>(p));
  Tuple t;
  t.key = (u64)v.x;
  t.pay = (u64)v.y;
  return t;
}

__device__ __forceinline__ void st_tuple(Tuple* p, const Tuple& t) {
  *reinterpret_cast<longlong2*>(p) = make_longlong2((long long)t.key, (long long)t.pay);
}

// First index of a[0, n) whose key is >= k, by interpolation search (Sec. 3.2.2,
// Fig. 7).  The answer lies in (L, H], with key_at(L) < k <= key_at(H) known; each
// step probes the position the rule of proportion gives between the two known
// keys, L + (H - L) (k - key(L)) / (key(H) - key(L)), and keeps the side that holds
// the answer, so the second step searches between the first key and the first
// probe, as in the paper's example.  After INTERP_STEPS steps a binary search
// ends it, which bounds the worst case (clustered keys) by log2 n probes more.
// (On 10^6 uniform keys the search takes about 7 probes, at most 12.)
constexpr u32 INTERP_STEPS = 16;

template <typename KeyAt>
__device__ __forceinline__ u64 interp_lower_bound(KeyAt key_at, u64 n, u64 k, u32& probes) {
  if (n == 0) return 0;
  ++probes;
  u64 kl = key_at(0);
  if (kl >= k) return 0;
  ++probes;
  u64 kh = key_at(n - 1);
  if (kh < k) return n;
  u64 L = 0, H = n - 1;  // key(L) = kl < k <= kh = key(H)
  for (u32 step = 0; step < INTERP_STEPS && H - L > 1; ++step) {
    // FP32 is enough for a guess (the exact steps follow) and far cheaper than FP64 here
    const float f = __fdividef((float)(k - kl), (float)(kh - kl));  // in (0, 1]
    u64 pos = L + (u64)(f * (float)(H - L));
    pos = pos <= L ? L + 1 : (pos >= H ? H - 1 : pos);
    ++probes;
    const u64 kp = key_at(pos);
    if (kp < k) {
      L = pos;
      kl = kp;
    } else {
      H = pos;
      kh = kp;
    }
  }
  u64 lo = L + 1, hi = H;  // binary search of the rest: answer in [lo, hi]
  while (lo < hi) {
    const u64 mid = lo + ((hi - lo) >> 1);
    ++probes;
    if (key_at(mid) < k) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

}  // namespace mpsm
