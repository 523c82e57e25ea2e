/*
 * gen_core.h -- seeded, counter-based synthetic workloads for the MPSM join.
 *
 * This module produces INPUTS only.  It holds none of the join's arithmetic
 * (no sorting, partitioning, searching or matching): every value it returns is
 * a pure function of (seed, stream, index), so the same bytes come out on the
 * host (oracle side) and on the device (kernel side), and the bookkeeping a
 * closed-form expected result needs (which R row an S tuple was drawn from) can
 * be regenerated without storing anything.
 *
 * Workload shapes follow the paper's experiments (Sec. 5.1): tuples of a 64-bit
 * join key and a 64-bit payload; R with unique keys; S drawn from R's keys with
 * a multiplicity (foreign keys), optionally Zipf-skewed, or from a sparse,
 * clustered 64-bit domain with a share of keys that match nothing, or with the
 * negatively correlated 80:20 skew of Sec. 5.6 (R's keys crowd the low fifth of
 * the key domain, S's foreign keys the high fifth), or with the location skew of
 * Sec. 5.5 (R stored in small-to-large key order by clusters, each shuffled).
 *
 * Building blocks (all published, restated here):
 *  - splitmix64 finaliser (Steele, Lea, Flood 2014; Vigna's constants) as the
 *    counter-based random source;
 *  - a 6-round balanced Feistel network on 2h bits with cycle walking
 *    (Black & Rogaway 2002) as a seeded bijection of [0, n);
 *  - Lemire's multiply-high map of a 64-bit draw onto [0, n);
 *  - inverse-CDF table sampling for Zipf(theta) and for the sparse clusters'
 *    key spacing (tables are built on the host in FP64 and shared byte-for-byte,
 *    so sampling itself is integer-exact on both sides).
 */
#ifndef MPSM_GEN_CORE_H
#define MPSM_GEN_CORE_H

#include <stdint.h>

#if defined(__CUDACC__)
#define GEN_HD __host__ __device__ __forceinline__
#else
#define GEN_HD static inline
#endif

typedef struct { uint64_t key, payload; } gen_tuple_t;

enum { GEN_KIND_UNIFORM = 0, GEN_KIND_ZIPF = 1, GEN_KIND_SPARSE = 2, GEN_KIND_NEGCORR = 3, GEN_KIND_LOCSKEW = 4 };

/* Streams: each independent draw has its own stream id. */
enum {
  GEN_ST_RPERM = 1, GEN_ST_RPAY = 2, GEN_ST_SROW = 3, GEN_ST_SROW2 = 4,
  GEN_ST_SPAY = 5, GEN_ST_HOT = 6, GEN_ST_FK = 7, GEN_ST_GAP = 8, GEN_ST_GAPKEY = 9
};

#define GEN_NONE (~0ull)

typedef struct {
  uint64_t g0;      /* first global sorted index of the cluster          */
  uint64_t n;       /* number of keys in the cluster                      */
  uint64_t lo;      /* base key of the cluster                            */
  uint64_t spread;  /* last entry of the cluster's offset table           */
} gen_cluster_t;

typedef struct {
  int32_t kind;               /* GEN_KIND_*                                     */
  uint32_t hR, hS;            /* Feistel half widths for [0,nR) and [0,nS)      */
  uint32_t pad0;
  uint64_t nR, nS;
  uint64_t seed;
  /* Zipf: entry e covers ranks [zlo[e], zlo[e+1]); a draw u picks the first e
   * with u < zthr[e] (zthr[nz-1] == 2^64-1). */
  const uint64_t* zthr;
  const uint64_t* zlo;        /* nz + 1 entries                                 */
  uint64_t nz;
  /* Sparse: keys of R in sorted order are f(g), g in [0,nR).  Cluster c owns
   * g in [cl[c].g0, cl[c].g0 + cl[c].n); f(g) = lo + 2j + Q_c(j), j = g - g0,
   * Q_c interpolates the non-decreasing table qtab[c*(nq+1) + 0..nq]. */
  const gen_cluster_t* cl;
  const uint64_t* qtab;
  uint32_t ncl, nq;
  uint64_t n_fk;              /* sparse: how many S tuples are drawn from R     */
} gen_spec_t;

/* splitmix64 output function */
GEN_HD uint64_t gen_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* value i of the splitmix64 sequence seeded by (seed, stream) */
GEN_HD uint64_t gen_rand(uint64_t seed, uint64_t stream, uint64_t i) {
  uint64_t base = gen_mix(seed ^ (stream * 0xD1342543DE82EF95ull) ^ 0x5851F42D4C957F2Dull);
  return gen_mix(base + (i + 1ull) * 0x9E3779B97F4A7C15ull);
}

GEN_HD uint64_t gen_mulhi(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
#endif
}

/* Lemire: a uniform 64-bit draw mapped onto [0, n) */
GEN_HD uint64_t gen_below(uint64_t r, uint64_t n) { return gen_mulhi(r, n); }

/* smallest h >= 1 with 4^h >= n */
GEN_HD uint32_t gen_half_bits(uint64_t n) {
  uint64_t m = n > 1 ? n - 1 : 1;
  uint32_t b = 0;
  while (m) { ++b; m >>= 1; }
  return (b + 1) / 2;
}

GEN_HD uint64_t gen_perm_key(uint64_t seed, uint64_t stream) {
  return gen_mix(seed * 0x2545F4914F6CDD1Dull + stream * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull);
}

/* one 6-round Feistel network on 2h bits (L = high h bits, R = low h bits) */
GEN_HD uint64_t gen_feistel_fwd(uint64_t x, uint32_t h, uint64_t key) {
  const uint64_t mask = (h >= 64) ? ~0ull : ((1ull << h) - 1ull);
  uint64_t L = x >> h, R = x & mask;
  for (uint32_t r = 0; r < 6; ++r) {
    uint64_t f = gen_mix(key + (uint64_t)(r + 1) * 0xA0761D6478BD642Full + R) & mask;
    uint64_t t = L ^ f;
    L = R;
    R = t;
  }
  return (L << h) | R;
}

GEN_HD uint64_t gen_feistel_inv(uint64_t y, uint32_t h, uint64_t key) {
  const uint64_t mask = (h >= 64) ? ~0ull : ((1ull << h) - 1ull);
  uint64_t L = y >> h, R = y & mask;
  for (int r = 5; r >= 0; --r) {
    uint64_t f = gen_mix(key + (uint64_t)(r + 1) * 0xA0761D6478BD642Full + L) & mask;
    uint64_t t = R ^ f;
    R = L;
    L = t;
  }
  return (L << h) | R;
}

/* bijection of [0, n) by cycle walking (4^h >= n, so < 4 steps on average) */
GEN_HD uint64_t gen_perm(uint64_t i, uint64_t n, uint32_t h, uint64_t key) {
  uint64_t y = gen_feistel_fwd(i, h, key);
  while (y >= n) y = gen_feistel_fwd(y, h, key);
  return y;
}

GEN_HD uint64_t gen_perm_inv(uint64_t y, uint64_t n, uint32_t h, uint64_t key) {
  uint64_t x = gen_feistel_inv(y, h, key);
  while (x >= n) x = gen_feistel_inv(x, h, key);
  return x;
}

/* --- sparse clustered domain: g-th smallest R key ------------------------ */
GEN_HD uint64_t gen_sparse_key(const gen_spec_t* s, uint64_t g) {
  uint32_t lo = 0, hi = s->ncl; /* last cluster with g0 <= g */
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (s->cl[mid].g0 <= g) lo = mid; else hi = mid;
  }
  const gen_cluster_t c = s->cl[lo];
  const uint64_t j = g - c.g0;
  const uint64_t t = j * (uint64_t)s->nq;
  const uint64_t i = t / c.n;
  const uint64_t r = t - i * c.n;
  const uint64_t* q = s->qtab + (uint64_t)lo * (s->nq + 1u);
  const uint64_t d0 = q[i];
  const uint64_t d1 = q[i + 1 <= s->nq ? i + 1 : s->nq];
  const uint64_t add = (uint64_t)(((unsigned __int128)(d1 - d0) * (unsigned __int128)r) / (unsigned __int128)c.n);
  return c.lo + 2ull * j + d0 + add;
}

/* --- negatively correlated 80:20 domain --------------------------------- */
/* g-th smallest R key: the first 4/5 of R's keys are 1, 2, ... (dense), the rest
 * follow 16 apart, so 80 % of R's keys sit in the low fifth of [1, max key]. */
GEN_HD uint64_t gen_negcorr_key(uint64_t nR, uint64_t g) {
  const uint64_t lo = nR / 5 * 4 + nR % 5 * 4 / 5;  /* floor(4 nR / 5) */
  return g < lo ? 1ull + g : 1ull + lo + 16ull * (g - lo);
}

/* first g whose key lies in the top fifth of the domain (above 4/5 of the max key) */
GEN_HD uint64_t gen_negcorr_hi(uint64_t nR) {
  if (nR <= 1) return 0;
  const uint64_t lo = nR / 5 * 4 + nR % 5 * 4 / 5;
  const uint64_t top = gen_negcorr_key(nR, nR - 1);
  const uint64_t cut = top / 5 * 4 + top % 5 * 4 / 5;
  /* below lo, key 1 + cut is the first above the cut; from lo on, the smallest g
   * with 1 + lo + 16 (g - lo) > cut, i.e. 16 (g - lo) >= cut - lo */
  const uint64_t g = cut < lo ? cut : lo + (cut - lo) / 16 + ((cut - lo) % 16 ? 1u : 0u);
  return g < nR ? g : nR - 1;
}

/* --- location skew: R in GEN_LOC_CLUSTERS clusters of rows ----------------- */
/* Cluster c holds rows [b_c, b_{c+1}), b_c = floor(nR c / C), and exactly the keys
 * 1 + b_c .. b_{c+1} in a random order of its own: small to large key order across
 * clusters, no order inside one. */
#define GEN_LOC_CLUSTERS 64ull

GEN_HD uint64_t gen_loc_bound(uint64_t nR, uint64_t c) {
  return (uint64_t)(((unsigned __int128)nR * c) / GEN_LOC_CLUSTERS);
}

GEN_HD uint64_t gen_loc_key(const gen_spec_t* s, uint64_t row) {
  uint64_t c = (uint64_t)(((unsigned __int128)row * GEN_LOC_CLUSTERS) / s->nR);
  while (c + 1 < GEN_LOC_CLUSTERS && gen_loc_bound(s->nR, c + 1) <= row) ++c;
  while (c > 0 && gen_loc_bound(s->nR, c) > row) --c;
  const uint64_t b0 = gen_loc_bound(s->nR, c), nc = gen_loc_bound(s->nR, c + 1) - b0;
  const uint64_t key = gen_perm_key(s->seed ^ ((c + 1ull) * 0xC2B2AE3D27D4EB4Full), GEN_ST_RPERM);
  return 1ull + b0 + gen_perm(row - b0, nc, gen_half_bits(nc), key);
}

/* --- R ------------------------------------------------------------------- */
GEN_HD uint64_t gen_r_key(const gen_spec_t* s, uint64_t row) {
  if (s->kind == GEN_KIND_LOCSKEW) return gen_loc_key(s, row);
  uint64_t p = gen_perm(row, s->nR, s->hR, gen_perm_key(s->seed, GEN_ST_RPERM));
  if (s->kind == GEN_KIND_SPARSE) return gen_sparse_key(s, p);
  if (s->kind == GEN_KIND_NEGCORR) return gen_negcorr_key(s->nR, p);
  return 1ull + p;
}

GEN_HD uint64_t gen_r_payload(const gen_spec_t* s, uint64_t row) {
  return gen_rand(s->seed, GEN_ST_RPAY, row);
}

/* --- S ------------------------------------------------------------------- */
GEN_HD uint64_t gen_zipf_rank(const gen_spec_t* s, uint64_t j) {
  const uint64_t u = gen_rand(s->seed, GEN_ST_SROW, j);
  uint64_t lo = 0, hi = s->nz - 1; /* first e with u < zthr[e] */
  while (lo < hi) {
    uint64_t mid = (lo + hi) >> 1;
    if (u < s->zthr[mid]) hi = mid; else lo = mid + 1;
  }
  const uint64_t a = s->zlo[lo], b = s->zlo[lo + 1];
  return a + gen_below(gen_rand(s->seed, GEN_ST_SROW2, j), b - a);
}

/* R row that S tuple j was drawn from, or GEN_NONE for a key that matches nothing */
GEN_HD uint64_t gen_s_row(const gen_spec_t* s, uint64_t j) {
  if (s->kind == GEN_KIND_ZIPF) {
    uint64_t rank = gen_zipf_rank(s, j);
    return gen_perm(rank, s->nR, s->hR, gen_perm_key(s->seed, GEN_ST_HOT));
  }
  if (s->kind == GEN_KIND_SPARSE) {
    uint64_t q = gen_perm(j, s->nS, s->hS, gen_perm_key(s->seed, GEN_ST_FK));
    if (q >= s->n_fk) return GEN_NONE;
  }
  if (s->kind == GEN_KIND_NEGCORR) {
    /* 4 in 5 tuples take one of R's keys in the top fifth of the domain, the rest
     * one of the keys below it; g is the key's rank among R's keys */
    const uint64_t gh = gen_negcorr_hi(s->nR);
    const uint64_t v = gen_rand(s->seed, GEN_ST_SROW2, j);
    const uint64_t g = (gen_below(gen_rand(s->seed, GEN_ST_SROW, j), 5) != 0 || gh == 0)
                           ? gh + gen_below(v, s->nR - gh)
                           : gen_below(v, gh);
    return gen_perm_inv(g, s->nR, s->hR, gen_perm_key(s->seed, GEN_ST_RPERM));
  }
  return gen_below(gen_rand(s->seed, GEN_ST_SROW, j), s->nR);
}

GEN_HD uint64_t gen_s_key(const gen_spec_t* s, uint64_t j) {
  const uint64_t row = gen_s_row(s, j);
  if (row != GEN_NONE) return gen_r_key(s, row);
  /* a key strictly inside the gap between the (g-1)-th and g-th smallest R keys */
  const uint64_t g = gen_below(gen_rand(s->seed, GEN_ST_GAP, j), s->nR + 1ull);
  const uint64_t a = (g == 0) ? 0ull : gen_sparse_key(s, g - 1);
  const uint64_t b = (g == s->nR) ? ~0ull : gen_sparse_key(s, g);
  return a + 1ull + gen_below(gen_rand(s->seed, GEN_ST_GAPKEY, j), b - a - 1ull);
}

GEN_HD uint64_t gen_s_payload(const gen_spec_t* s, uint64_t j) {
  return gen_rand(s->seed, GEN_ST_SPAY, j);
}

#endif /* MPSM_GEN_CORE_H */
