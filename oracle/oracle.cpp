/*
 * oracle.cpp -- plain, slow, obviously correct CPU reference for the MPSM join.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * benchmark's CPU-baseline leg may load this library.  The join library never
 * links, includes or calls it, and it shares no code with the CUDA path; the
 * only module both sides use is the input generator (gen/), which holds no join
 * arithmetic.
 *
 * What the method computes (Sec. 5.1, the benchmark query; Sec. 2: an exact
 * join of independently sorted runs, without a final merge): the equi-join of R
 * and S on the 64-bit key.  From the multiset of matching pairs {(r, s) : r.key == s.key} we report
 *   count    = number of pairs,
 *   checksum = sum over pairs of (r.payload + s.payload), modulo 2^64,
 *   pairs    = optionally the pairs themselves as (r.payload, s.payload).
 * The paper's query aggregates max(R.payload + S.payload); the wrapping sum is
 * the aggregate this library reports (it feeds every payload through the join
 * just like the max does, and is order-independent).
 *
 * oracle_join follows that definition directly: sort both inputs by key
 * (std::sort, a library primitive) and walk equal-key groups.  A group with c_R
 * tuples in R and c_S in S contributes c_R*c_S pairs and, since Z/2^64 is a
 * ring, c_S*sum_R + c_R*sum_S to the checksum.  oracle_brute is the O(|R||S|)
 * nested loop.  The step oracles below restate the intermediate results the
 * paper defines for each phase, in the paper's order and notation.
 *
 * Parity pins (tests/test_oracle.py): brute force on tiny inputs, closed forms
 * of the generator's foreign-key workloads, the worked examples of Fig. 6 and
 * Fig. 10, exhaustive DP for the splitter objective, and textbook lower/upper
 * bounds.
 */
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <thread>
#include <vector>

#include "../gen/gen_core.h"

#define OEXPORT extern "C" __attribute__((visibility("default")))

typedef struct { uint64_t key, payload; } otuple;
typedef struct { uint64_t r_payload, s_payload; } opair;

static bool by_key(const otuple& a, const otuple& b) { return a.key < b.key; }

/* ------------------------------------------------------------ the join */

/* Equi-join R and S (Sec. 5.1).  If pairs != NULL, writes up to cap pairs in
 * lexicographic (r_payload, s_payload) order; *count is always the full count. */
OEXPORT int oracle_join(const otuple* R, uint64_t nR, const otuple* S, uint64_t nS,
                        uint64_t* count, uint64_t* checksum, opair* pairs, uint64_t cap) {
  std::vector<otuple> r(R, R + nR), s(S, S + nS);
  std::sort(r.begin(), r.end(), by_key);
  std::sort(s.begin(), s.end(), by_key);
  uint64_t cnt = 0, chk = 0;
  std::vector<opair> out;
  uint64_t i = 0, j = 0;
  while (i < nR && j < nS) {
    if (r[i].key < s[j].key) { ++i; continue; }
    if (s[j].key < r[i].key) { ++j; continue; }
    const uint64_t k = r[i].key;
    uint64_t i1 = i, j1 = j, sum_r = 0, sum_s = 0;
    while (i1 < nR && r[i1].key == k) sum_r += r[i1++].payload;
    while (j1 < nS && s[j1].key == k) sum_s += s[j1++].payload;
    const uint64_t c_r = i1 - i, c_s = j1 - j;
    cnt += c_r * c_s;
    chk += c_s * sum_r + c_r * sum_s;
    if (pairs)
      for (uint64_t a = i; a < i1; ++a)
        for (uint64_t b = j; b < j1; ++b) out.push_back({r[a].payload, s[b].payload});
    i = i1;
    j = j1;
  }
  *count = cnt;
  *checksum = chk;
  if (pairs) {
    std::sort(out.begin(), out.end(), [](const opair& a, const opair& b) {
      return a.r_payload != b.r_payload ? a.r_payload < b.r_payload : a.s_payload < b.s_payload;
    });
    const uint64_t w = std::min<uint64_t>(cap, out.size());
    if (w) memcpy(pairs, out.data(), w * sizeof(opair));
  }
  return 0;
}

/* Nested loop over all |R| x |S| combinations. */
OEXPORT int oracle_brute(const otuple* R, uint64_t nR, const otuple* S, uint64_t nS,
                         uint64_t* count, uint64_t* checksum) {
  uint64_t cnt = 0, chk = 0;
  for (uint64_t i = 0; i < nR; ++i)
    for (uint64_t j = 0; j < nS; ++j)
      if (R[i].key == S[j].key) {
        ++cnt;
        chk += R[i].payload + S[j].payload;
      }
  *count = cnt;
  *checksum = chk;
  return 0;
}

/* Closed form for the generator's workloads: R keys are unique, so an S tuple
 * drawn from R row `row` matches exactly that row and nothing else, and a gap
 * key matches nothing.  count = #drawn tuples, checksum = sum of
 * (s.payload + R.payload[row]).  O(|S|), regenerating the draws (no sort). */
OEXPORT int oracle_closed_form(const gen_spec_t* spec, int nthreads, uint64_t* count,
                               uint64_t* checksum) {
  const gen_spec_t s = *spec;
  if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());
  if (s.nS < (1u << 16)) nthreads = 1;
  std::vector<uint64_t> pc(nthreads, 0), pk(nthreads, 0);
  std::vector<std::thread> pool;
  const uint64_t per = (s.nS + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    pool.emplace_back([&, t] {
      const uint64_t a = (uint64_t)t * per, b = std::min<uint64_t>(s.nS, a + per);
      uint64_t c = 0, k = 0;
      for (uint64_t j = a; j < b; ++j) {
        const uint64_t row = gen_s_row(&s, j);
        if (row == GEN_NONE) continue;
        ++c;
        k += gen_s_payload(&s, j) + gen_r_payload(&s, row);
      }
      pc[t] = c;
      pk[t] = k;
    });
  }
  for (auto& th : pool) th.join();
  uint64_t c = 0, k = 0;
  for (int t = 0; t < nthreads; ++t) { c += pc[t]; k += pk[t]; }
  *count = c;
  *checksum = k;
  return 0;
}

/* ------------------------------------------------------------ phase 1: runs */

/* Chunk j of n over T workers is [floor(j n / T), floor((j+1) n / T)) (Sec. 2.1:
 * "the input data is chunked into equally sized chunks among the workers"). */
OEXPORT uint64_t oracle_chunk_start(uint64_t n, uint64_t T, uint64_t j) {
  return (uint64_t)(((unsigned __int128)n * j) / T);
}

/* Phase 1 (Sec. 2.1, Fig. 3/5): cut R into T chunks and sort each into a run.
 * Runs are written back to back in `out`; run_off receives T+1 boundaries.
 * std::stable_sort by key: within equal keys the input order is kept. */
OEXPORT int oracle_sort_runs(const otuple* R, uint64_t nR, uint32_t T, otuple* out,
                             uint64_t* run_off) {
  if (T == 0) return 1;
  memcpy(out, R, nR * sizeof(otuple));
  for (uint32_t j = 0; j < T; ++j) {
    const uint64_t a = oracle_chunk_start(nR, T, j), b = oracle_chunk_start(nR, T, j + 1);
    run_off[j] = a;
    std::stable_sort(out + a, out + b, by_key);
  }
  run_off[T] = nR;
  return 0;
}

/* ------------------------------------------------ phase 2: histograms & splitters */

static uint32_t bitlen64(uint64_t x) {
  uint32_t b = 0;
  while (x) { ++b; x >>= 1; }
  return b;
}

/* Radix clustering on the highest B bits after shifting keys into R's range
 * (Sec. 3.2.1; the key preprocessing of the last paragraph of Sec. 3.2.1):
 * bucket(k) = (k - kmin) >> shift for kmin <= k <= kmax, with
 * shift = max(0, bitlen(kmax - kmin) - B).  Keys outside [kmin, kmax] cannot
 * match any R tuple and are not partitioned.  Returns the number of buckets. */
OEXPORT uint32_t oracle_fine_geometry(uint64_t kmin, uint64_t kmax, uint32_t B, uint32_t* shift) {
  const uint32_t bits = bitlen64(kmax - kmin);
  *shift = bits > B ? bits - B : 0;
  return (uint32_t)((kmax - kmin) >> *shift) + 1u;
}

/* Per-worker histograms h_i over the fine buckets (Sec. 3.2.1, Fig. 6; Sec. 4.2).
 * Worker i owns chunk [chunk_off[i], chunk_off[i+1]) of S; h is W x nb. */
OEXPORT int oracle_worker_histograms(const otuple* S, const uint64_t* chunk_off, uint32_t W,
                                     uint64_t kmin, uint64_t kmax, uint32_t shift, uint32_t nb,
                                     uint64_t* h) {
  memset(h, 0, sizeof(uint64_t) * (uint64_t)W * nb);
  for (uint32_t i = 0; i < W; ++i)
    for (uint64_t t = chunk_off[i]; t < chunk_off[i + 1]; ++t) {
      const uint64_t k = S[t].key;
      if (k < kmin || k > kmax) continue;
      h[(uint64_t)i * nb + ((k - kmin) >> shift)] += 1;
    }
  return 0;
}

/* Number of R tuples per fine bucket, counted in the sorted runs: the run side's
 * share of each key range, which the splitter cost charges as "relevant data"
 * (Sec. 4.3; Sec. 4.1's CDF evaluated at the radix boundaries). */
OEXPORT int oracle_run_counts(const otuple* Rs, const uint64_t* run_off, uint32_t T,
                              uint64_t kmin, uint64_t kmax, uint32_t shift, uint32_t nb,
                              uint64_t* g) {
  memset(g, 0, sizeof(uint64_t) * nb);
  for (uint32_t j = 0; j < T; ++j)
    for (uint64_t t = run_off[j]; t < run_off[j + 1]; ++t) {
      const uint64_t k = Rs[t].key;
      if (k < kmin || k > kmax) continue;
      g[(k - kmin) >> shift] += 1;
    }
  return 0;
}

/* The binary logarithm of the splitter cost, in Q16: L(n) = floor(2^16 log2 n)
 * for n >= 2, and 0 for n <= 1.  Sec. 4.3 charges a partition of n tuples
 * n log n for its sort; the library and this oracle evaluate that term as
 * n * L(n) in integers, so both choose the same splitters bit for bit.
 *
 * Definition: 2^L(n) <= n^65536 < 2^(L(n)+1), i.e. L(n) = bitlen(n^65536) - 1.
 * oracle_log2_q16_big computes exactly that with plain big-integer products. */
typedef std::vector<uint32_t> bignum; /* little-endian base-2^32 digits */

static bignum big_mul(const bignum& a, const bignum& b) {
  bignum r(a.size() + b.size(), 0);
  for (size_t i = 0; i < a.size(); ++i) {
    uint64_t carry = 0;
    for (size_t j = 0; j < b.size(); ++j) {
      const uint64_t t = (uint64_t)a[i] * b[j] + r[i + j] + carry;
      r[i + j] = (uint32_t)t;
      carry = t >> 32;
    }
    r[i + b.size()] = (uint32_t)carry;
  }
  while (r.size() > 1 && r.back() == 0) r.pop_back();
  return r;
}

OEXPORT uint64_t oracle_log2_q16_big(uint64_t n) {
  if (n <= 1) return 0;
  bignum x;
  x.push_back((uint32_t)n);
  if (n >> 32) x.push_back((uint32_t)(n >> 32));
  for (int i = 0; i < 16; ++i) x = big_mul(x, x); /* n^(2^16) */
  return 32ull * (x.size() - 1) + bitlen64(x.back()) - 1;
}

static bignum big_from(uint64_t v) {
  bignum x(1, (uint32_t)v);
  if (v >> 32) x.push_back((uint32_t)(v >> 32));
  return x;
}

static bignum big_shl(const bignum& a, unsigned s) {
  bignum r(s / 32, 0);
  uint32_t carry = 0;
  const unsigned b = s % 32;
  for (uint32_t d : a) {
    r.push_back(b ? (d << b) | carry : d);
    carry = b ? d >> (32 - b) : 0;
  }
  if (carry) r.push_back(carry);
  while (r.size() > 1 && r.back() == 0) r.pop_back();
  return r;
}

/* floor(a / 2^s); *lost is set when a nonzero bit was shifted out */
static bignum big_shr(const bignum& a, unsigned s, bool* lost) {
  const size_t q = s / 32;
  const unsigned b = s % 32;
  *lost = false;
  for (size_t i = 0; i < q && i < a.size(); ++i) *lost = *lost || a[i] != 0;
  if (q < a.size() && b) *lost = *lost || (a[q] & ((1u << b) - 1)) != 0;
  bignum r;
  for (size_t i = q; i < a.size(); ++i) {
    const uint64_t hi = i + 1 < a.size() ? a[i + 1] : 0;
    r.push_back((uint32_t)((((uint64_t)hi << 32) | a[i]) >> b));
  }
  if (r.empty()) r.push_back(0);
  while (r.size() > 1 && r.back() == 0) r.pop_back();
  return r;
}

static bignum big_inc(bignum a) {
  for (size_t i = 0; i < a.size(); ++i)
    if (++a[i] != 0) return a;
  a.push_back(1);
  return a;
}

static int big_cmp(const bignum& a, const bignum& b) {
  if (a.size() != b.size()) return a.size() < b.size() ? -1 : 1;
  for (size_t i = a.size(); i-- > 0;)
    if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
  return 0;
}

/* The same value by the bit-by-bit method: with n = 2^k x, x in [1, 2),
 * log2 n = k + log2 x, and squaring x doubles log2 x, so each squaring yields
 * the next fractional bit (1 when the square reaches 2, which is then halved).
 * x is carried as an interval [lo, hi] of numbers with F fractional bits that
 * holds the true value at every step (squares rounded down for lo, up for hi),
 * so every bit it takes is certain.  Returns -1 if some square's interval
 * straddles 2, i.e. F bits cannot decide that bit. */
static int64_t log2_q16_interval(uint64_t n, unsigned F) {
  const uint32_t k = bitlen64(n) - 1;
  bignum lo = big_shl(big_from(n), F - k), hi = lo; /* F >= 64: exact */
  const bignum two = big_shl(big_from(2), F);
  int64_t r = (int64_t)k << 16;
  bool lost;
  for (int i = 15; i >= 0; --i) {
    const bignum sl = big_shr(big_mul(lo, lo), F, &lost);
    bignum sh = big_shr(big_mul(hi, hi), F, &lost);
    if (lost) sh = big_inc(sh);
    if (big_cmp(sl, two) >= 0) {
      r |= (int64_t)1 << i;
      lo = big_shr(sl, 1, &lost);
      hi = big_shr(sh, 1, &lost);
      if (lost) hi = big_inc(hi);
    } else if (big_cmp(sh, two) < 0) {
      lo = sl;
      hi = sh;
    } else {
      return -1;
    }
  }
  return r;
}

/* L(n): first the interval method in 62 fractional bits with 128-bit products
 * (cheap), then in 128, 256, ... bits on big integers, then the definition. */
OEXPORT uint64_t oracle_log2_q16(uint64_t n) {
  if (n <= 1) return 0;
  typedef unsigned __int128 u128;
  const uint32_t k = bitlen64(n) - 1;
  const uint64_t two = 1ull << 63; /* 2.0 in Q62 */
  uint64_t lo, hi;
  if (k <= 62) {
    lo = hi = n << (62 - k); /* exact */
  } else {
    lo = n >> 1;
    hi = lo + (n & 1);
  }
  uint64_t r = (uint64_t)k << 16;
  for (int i = 15; i >= 0; --i) {
    const u128 sl = ((u128)lo * lo) >> 62;
    const u128 sh = ((u128)hi * hi + ((((u128)1) << 62) - 1)) >> 62;
    if (sl >= two) {
      r |= 1ull << i;
      lo = (uint64_t)(sl >> 1);
      hi = (uint64_t)((sh + 1) >> 1);
    } else if (sh < two) {
      lo = (uint64_t)sl;
      hi = (uint64_t)sh;
    } else {
      for (unsigned F = 128; F <= 8192; F *= 2) {
        const int64_t v = log2_q16_interval(n, F);
        if (v >= 0) return (uint64_t)v;
      }
      return oracle_log2_q16_big(n);
    }
  }
  return r;
}

/* The interval method at a given precision alone (tests). */
OEXPORT int64_t oracle_log2_q16_prec(uint64_t n, uint32_t F) {
  if (n <= 1) return 0;
  return log2_q16_interval(n, F < 64 ? 64 : F);
}

/* split-relevant cost of a partition (Sec. 4.3), in units of 2^-16 tuples:
 *   |S_i| log2|S_i|   (sort the partitioned side's partition)
 * + T |S_i|           (process it once per run of the other side)
 * + |R in range|      (relevant data of the run side, the CDF difference)
 * with S the partitioned side and R the run side. */
static uint64_t split_cost(uint64_t n, uint64_t r, uint32_t T, uint32_t kind) {
  if (kind == 1) return n << 16;  /* equi-height: the partition's share of the partitioned side only */
  return n * oracle_log2_q16(n) + (((uint64_t)T * n + r) << 16);
}

/* Greedy from the left: each partition takes buckets while its cost stays <= C.
 * Returns the number of partitions (UINT32_MAX if one bucket alone exceeds C);
 * fills sp[bucket] = partition when sp != NULL. */
static uint32_t greedy(const uint64_t* H, const uint64_t* G, uint32_t nb, uint32_t T, uint32_t kind, uint64_t C,
                       uint32_t* sp) {
  uint32_t parts = 0, a = 0;
  while (a < nb) {
    uint64_t n = H[a], r = G[a];
    if (split_cost(n, r, T, kind) > C) return UINT32_MAX;
    uint32_t b = a + 1;
    while (b < nb && split_cost(n + H[b], r + G[b], T, kind) <= C) {
      n += H[b];
      r += G[b];
      ++b;
    }
    if (sp)
      for (uint32_t f = a; f < b; ++f) sp[f] = parts;
    ++parts;
    a = b;
  }
  return parts;
}

/* Splitter computation (Sec. 4.3): group the nb fine buckets into at most P
 * contiguous partitions minimising the largest split-relevant cost.  The paper
 * leaves the solver open (it cites Ross & Cieslewicz); this one finds the exact
 * optimum C* by bisection over integer costs (greedy feasibility is exact for
 * costs that grow with the range) and returns the leftmost greedy grouping at
 * C*.  sp[f] = partition of bucket f; returns the number of partitions used. */
OEXPORT uint32_t oracle_splitters_kind(const uint64_t* H, const uint64_t* G, uint32_t nb, uint32_t P,
                                       uint32_t T, uint32_t kind, uint32_t* sp, uint64_t* best) {
  uint64_t n = 0, r = 0, lo = 0;
  for (uint32_t f = 0; f < nb; ++f) {
    n += H[f];
    r += G[f];
    lo = std::max(lo, split_cost(H[f], G[f], T, kind));
  }
  uint64_t hi = split_cost(n, r, T, kind);
  /* smallest C in [lo, hi] with greedy(C) <= P; greedy(hi) == 1 <= P */
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if (greedy(H, G, nb, T, kind, mid, nullptr) <= P) hi = mid; else lo = mid + 1;
  }
  *best = lo;
  return greedy(H, G, nb, T, kind, lo, sp);
}

/* kind 0: the split-relevant cost above; kind 1: equi-height partitions, i.e. the
 * same contiguous grouping minimising the largest partition of the partitioned
 * side alone (the baseline of Sec. 5.6, Fig. 16b). */
OEXPORT uint32_t oracle_splitters(const uint64_t* H, const uint64_t* G, uint32_t nb, uint32_t P,
                                  uint32_t T, uint32_t* sp, uint64_t* best) {
  return oracle_splitters_kind(H, G, nb, P, T, 0, sp, best);
}

/* Exhaustive check of the same objective for small nb (DP over prefixes):
 * the smallest achievable largest cost with at most P contiguous groups. */
OEXPORT uint64_t oracle_splitters_dp_kind(const uint64_t* H, const uint64_t* G, uint32_t nb, uint32_t P,
                                          uint32_t T, uint32_t kind) {
  const uint64_t INF = ~0ull;
  std::vector<uint64_t> prev(nb + 1, INF), cur(nb + 1, INF);
  prev[0] = 0;
  uint64_t bestv = INF;
  for (uint32_t p = 1; p <= P; ++p) {
    std::fill(cur.begin(), cur.end(), INF);
    for (uint32_t b = 1; b <= nb; ++b) {
      uint64_t n = 0, r = 0;
      for (uint32_t a = b; a-- > 0;) {
        n += H[a];
        r += G[a];
        if (prev[a] == INF) continue;
        const uint64_t v = std::max(prev[a], split_cost(n, r, T, kind));
        cur[b] = std::min(cur[b], v);
      }
    }
    bestv = std::min(bestv, cur[nb]);
    prev.swap(cur);
  }
  return bestv;
}

OEXPORT uint64_t oracle_splitters_dp(const uint64_t* H, const uint64_t* G, uint32_t nb, uint32_t P,
                                     uint32_t T) {
  return oracle_splitters_dp_kind(H, G, nb, P, T, 0);
}

/* Prefix sums (Sec. 3.2.1, the ps equation under Fig. 6): ps_i[j] = sum of
 * h_k[j] over workers k < i, offset by the start of partition j in the output
 * (partitions stored back to back).  h is W x P; ps is W x P; part_off is P+1. */
OEXPORT int oracle_prefix_sums(const uint64_t* h, uint32_t W, uint32_t P, uint64_t* ps,
                               uint64_t* part_off) {
  uint64_t base = 0;
  for (uint32_t j = 0; j < P; ++j) {
    part_off[j] = base;
    uint64_t run = 0;
    for (uint32_t i = 0; i < W; ++i) {
      ps[(uint64_t)i * P + j] = base + run;
      run += h[(uint64_t)i * P + j];
    }
    base += run;
  }
  part_off[P] = base;
  return 0;
}

/* Synchronisation-free scatter (Sec. 4.3): worker i writes its next tuple t to
 * ps_i[sp[bucket(t.key)]]++.  Dropped keys (outside R's range) are skipped. */
OEXPORT int oracle_scatter(const otuple* S, const uint64_t* chunk_off, uint32_t W, uint64_t kmin,
                           uint64_t kmax, uint32_t shift, const uint32_t* sp, uint32_t P,
                           const uint64_t* ps, otuple* out) {
  std::vector<uint64_t> cur(ps, ps + (uint64_t)W * P);
  for (uint32_t i = 0; i < W; ++i)
    for (uint64_t t = chunk_off[i]; t < chunk_off[i + 1]; ++t) {
      const uint64_t k = S[t].key;
      if (k < kmin || k > kmax) continue;
      const uint32_t p = sp[(k - kmin) >> shift];
      out[cur[(uint64_t)i * P + p]++] = S[t];
    }
  return 0;
}

/* ------------------------------------------------ phase 4: search windows */

/* For every S tile [tile_off[t], tile_off[t+1]) of the sorted partitioned side
 * and every run j, the part of run j that can join with the tile (Sec. 3.2.2):
 * [first position with key >= tile's first key, first position with key > tile's
 * last key), relative to the run start.  win is ntiles x T x 2. */
OEXPORT int oracle_windows(const otuple* Ss, const uint64_t* tile_off, uint64_t ntiles,
                           const otuple* Rs, const uint64_t* run_off, uint32_t T, uint64_t* win) {
  for (uint64_t t = 0; t < ntiles; ++t) {
    const uint64_t lo_key = Ss[tile_off[t]].key, hi_key = Ss[tile_off[t + 1] - 1].key;
    for (uint32_t j = 0; j < T; ++j) {
      const otuple* a = Rs + run_off[j];
      const otuple* b = Rs + run_off[j + 1];
      const otuple* lb = std::lower_bound(a, b, lo_key, [](const otuple& x, uint64_t k) { return x.key < k; });
      const otuple* ub = std::upper_bound(a, b, hi_key, [](uint64_t k, const otuple& x) { return k < x.key; });
      win[(t * T + j) * 2 + 0] = (uint64_t)(lb - a);
      win[(t * T + j) * 2 + 1] = (uint64_t)(ub - a);
    }
  }
  return 0;
}
