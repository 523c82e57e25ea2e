// learn.cuh -- the learned CDF model (a two-stage recursive model index) as
// the kernels see it, and its inference.
//
// The model predicts the CDF value y in [0, 1] of a key.  It plays the role of
// the paper's equi-height CDF of the runs (Sec. 4.1-4.2, Fig. 8): y times a
// run's length predicts where the key's merge starts in that run (Sec. 3.2.2).
// Every prediction is followed by an exact search, so the model changes speed,
// never results.  The learned partitions (Sec. 4.3) and the learned run buckets
// take the sorted sample's own quantiles -- its empirical CDF -- tabulated per
// key cell, below.
//
//   stage 1 (root):  x = (key - kmin) / (kmax - kmin)
//                    h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), yhat = W3 . h2 + b3
//                    (32 and 32 hidden units, FP32 weights, trained on the GPU)
//   stage 2 (leaf):  leaf l = clamp(floor(4096 yhat)); y = a_l (key - base_l) + b_l
//                    (least squares per leaf on the exact integer offset)
//
// Inference tabulates the root: the key range is cut into at most 2^16 equal
// cells, cell = (key - kmin) >> cshift, and tab[cell] holds the leaf the root
// picks at the cell's centre.  A prediction is then one table load, one leaf
// load and one FMA -- no FP64 and no MLP per key.
#pragma once

#include "mpsm_internal.cuh"

namespace mpsm {

constexpr u32 RMI_H = 32;
constexpr u32 RMI_NP = 1153;             // root parameters
constexpr u32 RMI_NPAD = 1156;           // padded; slot RMI_NP carries the loss in gradient partials
constexpr u32 RMI_LEAVES = 4096;
constexpr u32 RMI_CELL_BITS = 16;
constexpr u32 RMI_CELLS = 1u << RMI_CELL_BITS;
constexpr u32 RMI_TRAIN_MAX = 4096;      // training points per model (evenly spaced over its sample)
constexpr u32 RMI_GT = 32;               // points per block of the gradient kernel
constexpr u32 RMI_GMAX = RMI_TRAIN_MAX / RMI_GT;
// parameter vector layout: W1[32], b1[32], W2[32][32] (row = output unit), b2[32], W3[32], b3
constexpr u32 RO_W1 = 0, RO_B1 = 32, RO_W2 = 64, RO_B2 = 1088, RO_W3 = 1120, RO_B3 = 1152;

struct RmiLeaf {
  u64 base;                 // smallest training key routed to the leaf (0 when empty)
  float a, b;               // y = a * (key - base) + b
};

struct RmiModel {
  float theta[RMI_NPAD];
  float m[RMI_NPAD];        // Adam moments
  float v[RMI_NPAD];
  u64 kmin, kmax;           // key normalisation range
  u32 cshift, ncell;        // cell = min((key - kmin) >> cshift, ncell - 1)
  u64 fit_off;              // first fit point of this model in the fit arrays
  u32 fit_n, train_n;       // fit points (all of the model's sample); training points
  float loss0, loss;        // training loss before the first and before the last step
  u32 active, pad;
  u16 tab[RMI_CELLS];       // tabulated root: cell -> leaf
  RmiLeaf leaf[RMI_LEAVES];
};

// Predicted CDF value of `key`, clamped to [0, 1].
__device__ __forceinline__ float rmi_predict(const RmiModel* M, u64 key) {
  const u64 off = key > M->kmin ? key - M->kmin : 0ull;
  const u64 c = off >> M->cshift;
  const u32 cell = c >= (u64)M->ncell ? M->ncell - 1u : (u32)c;
  const u32 l = __ldg(&M->tab[cell]);
  const u64 base = __ldg(&M->leaf[l].base);
  const float a = __ldg(&M->leaf[l].a), b = __ldg(&M->leaf[l].b);
  const float d = key >= base ? (float)(key - base) : -(float)(base - key);
  const float y = fmaf(a, d, b);
  return fminf(fmaxf(y, 0.0f), 1.0f);
}

// lower bound (first index whose key >= k) in a[0, n), searched outward from the
// guess g: exponential steps to bracket, then binary search.  Counts probes.
template <typename KeyAt>
__device__ __forceinline__ u64 gallop_from(KeyAt key_at, u64 n, u64 g, u64 k, u32& probes) {
  if (g > n) g = n;
  u64 lo, hi;  // answer in [lo, hi]
  if (g < n && (++probes, key_at(g) < k)) {
    lo = g + 1;
    hi = n;
    u64 s = 1;
    for (;;) {
      const u64 t = g + s;
      if (t >= n) break;
      ++probes;
      if (key_at(t) >= k) {
        hi = t;
        break;
      }
      lo = t + 1;
      s <<= 1;
    }
  } else {
    hi = g;
    lo = 0;
    u64 s = 1;
    for (;;) {
      if (s > g) break;
      const u64 t = g - s;
      ++probes;
      if (key_at(t) < k) {
        lo = t + 1;
        break;
      }
      hi = t;
      s <<= 1;
    }
  }
  while (lo < hi) {
    const u64 mid = lo + ((hi - lo) >> 1);
    ++probes;
    if (key_at(mid) < k) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// finaliser of a 64-bit mixing hash (public-domain MurmurHash3 fmix64)
__device__ __forceinline__ u64 mix64(u64 z) {
  z ^= z >> 33;
  z *= 0xff51afd7ed558ccdull;
  z ^= z >> 33;
  z *= 0xc4ceb9fe1a85ec53ull;
  z ^= z >> 33;
  return z;
}

// Learned partition of an S tuple.  bnd holds the P - 1 sorted partition
// boundaries, the quantiles p/P of a sorted sample of m keys; rank[2p] and
// rank[2p + 1] count the sample keys < bnd[p] and <= bnd[p].  A key lies in
// partition #(bnd < key) unless it equals boundaries: then its share of the
// sample's CDF, [rank_lt, rank_le) / m, is cut across the partitions it spans, and
// each tuple takes the partition of a point drawn from that share by a hash of its
// row -- a hot key fills its partitions to the mean instead of making one huge.
// The function is computed from the key's fine cell (learned_cell_part).

// Fine-cell table of the learned partitions (one u32 per fine bucket of the job):
// the partition of every key in the cell, or -- with LCELL_SPLIT set -- the
// partitions plo (bits 0-13) to phi (bits 16-29) that the cell reaches when
// boundaries fall inside it.  LCELL_HOT marks a cell whose boundaries all equal one
// key (a hot key cut across partitions plo..phi): a key below it lies in plo, one
// above it in phi, and the key itself takes its hash-drawn share, with no search.
constexpr u32 LCELL_SPLIT = 0x80000000u;
constexpr u32 LCELL_HOT = 0x40000000u;

// The learned partition of `key` (above) from its fine cell's entry e; bnd and rank
// in shared memory.
__device__ __forceinline__ u32 learned_cell_part(u32 e, const u64* bnd, const u32* rank, u32 P, u32 m, u64 key,
                                                 u64 row, u64 seed, u32& probes) {
  if (!(e & LCELL_SPLIT)) return e;
  const u32 plo = e & 0x3FFFu, phi = (e >> 16) & 0x3FFFu;
  if (!(e & LCELL_HOT)) {
    // the boundaries that cut the cell are bnd[plo, phi), every other one lies outside
    // it: #(bnd < key) and, for a key equal to boundaries, #(bnd <= key) by bisection
    // among them
    u32 lb = plo, len = phi - plo;
    while (len > 0) {
      const u32 h = len >> 1;
      ++probes;
      if (bnd[lb + h] < key) {
        lb += h + 1;
        len -= h + 1;
      } else {
        len = h;
      }
    }
    if (lb >= phi || bnd[lb] != key) return lb;
    u32 ub = lb;
    len = phi - lb;
    while (len > 0) {
      const u32 h = len >> 1;
      ++probes;
      if (bnd[ub + h] <= key) {
        ub += h + 1;
        len -= h + 1;
      } else {
        len = h;
      }
    }
    const float lo = (float)rank[2 * lb], hi = (float)rank[2 * lb + 1];
    const float u = (float)(mix64(row ^ seed) >> 40) * (1.0f / 16777216.0f);  // [0, 1)
    const float c = fmaf(u, hi - lo, lo) * ((float)P / (float)m);
    u32 q = c > 0.0f ? (u32)c : 0u;
    q = q < lb ? lb : q;
    return q > ub ? ub : q;
  }
  ++probes;
  const u64 hot = bnd[plo];
  if (key != hot) return key < hot ? plo : phi;
  const float lo = (float)rank[2 * plo], hi = (float)rank[2 * plo + 1];
  const float u = (float)(mix64(row ^ seed) >> 40) * (1.0f / 16777216.0f);  // [0, 1)
  const float c = fmaf(u, hi - lo, lo) * ((float)P / (float)m);
  u32 q = c > 0.0f ? (u32)c : 0u;
  q = q < plo ? plo : q;
  return q > phi ? phi : q;
}

// The bucket function of a learned first sort pass over a job's runs: F buckets cut
// at F - 1 quantiles of a sorted, evenly spaced sample of m run-side keys, found
// through a table of ncell equal cells over the sample's key range: cell =
// min((key - lo) >> shift, ncell - 1), a key below lo taking cell 0.  The bucket of a
// key is run_learn_bucket's.
struct RunLearn {
  u64 lo;
  u32 shift, ncell;
  u32 F, m;
};

// the cell of `key` in a learned run bucket function's table
__device__ __forceinline__ u32 run_learn_cell(const RunLearn& RL, u64 key) {
  const u64 c = (key > RL.lo ? key - RL.lo : 0ull) >> RL.shift;
  return c < (u64)RL.ncell ? (u32)c : RL.ncell - 1u;
}

// The learned bucket of `key` for sorted boundaries bnd: #(bnd < key), plus one when the
// key equals a boundary.  Bucket b then holds the keys strictly between two boundary
// values or one boundary value alone, so a key equal to two or more boundaries (a hot
// key) fills a bucket of its own, a constant child; the function stays monotone.  From
// the key's cell entry e (the cell table's encoding, LCELL_*): the cell's bucket when no
// boundary falls in it, else a bisection over the boundaries plo..phi - 1 that do
// (bnd in shared memory).
__device__ __forceinline__ u32 run_learn_bucket(u32 e, const u64* bnd, u64 key) {
  if (!(e & LCELL_SPLIT)) return e;
  u32 pos = e & 0x3FFFu;
  const u32 phi = (e >> 16) & 0x3FFFu;
  if (e & LCELL_HOT) {  // every boundary here is one key
    const u64 hot = bnd[pos];
    return key < hot ? pos : (key == hot ? pos + 1u : phi);
  }
  u32 len = phi - pos;
  while (len > 0) {
    const u32 h = len >> 1;
    if (bnd[pos + h] < key) {
      pos += h + 1;
      len -= h + 1;
    } else {
      len = h;
    }
  }
  return (pos < phi && bnd[pos] == key) ? pos + 1u : pos;
}

struct LearnCtx {
  const RmiModel* models;   // 2 per job: [2 j] = S-side model, [2 j + 1] = R-side model
  const u64* bnd;           // per job P_MAX learned partition boundaries
  const u32* brank;         // per job 2 P_MAX sample ranks of the boundaries (< and <=)
  const u32* cell;          // per job FINE_MAX fine-cell table (LCELL_SPLIT marks cells a boundary cuts)
  u64 seed;                 // seed of the hot-key spreading hash
  u64* stat;                // [0] partition probes, [1] keys partitioned, [2] search probes,
                            // [3] searches, [4] sum of |prediction - exact| start positions
  u32 interp;               // without models: merge starts by interpolation search, not binary
  const RunLearn* rl;       // per job: the learned run bucket function (MODE_RLEARN) ...
  const u32* rcell;         // ... its cell table (FINE_MAX per job)
  const u64* rbnd;          // ... and boundaries (P_MAX per job)
};

}  // namespace mpsm
