// pmpsm.cpp -- P-MPSM, the paper's own multi-core sort-merge join (Sec. 3.2 and 4),
// on the host's cores: a CPU baseline to set beside the GPU library.  It shares
// no code with the GPU path or with the oracle.
//
// Roles as in the GPU library: R is cut into T chunks that are sorted into runs
// (the paper's public input); S is range-partitioned into T partitions, one per
// worker, and each partition is sorted and merge-joined against every run (the
// paper's private input).  Phases, each run by T worker threads:
//   1    sort the R chunks into runs;
//   2.1  the run side's CDF at the fine bucket bounds (exact counts by binary
//        search in every run, Sec. 4.1);
//   2.2  per worker, a 2^B-bucket radix histogram of its S chunk over R's key
//        range (Sec. 4.2);
//   2.3  splitters: the fine buckets grouped into T contiguous partitions that
//        minimise the largest split-relevant cost |S_i| log|S_i| + T |S_i| +
//        |R in range| (Sec. 4.3); per-worker prefix sums; every worker scatters
//        its chunk to its slots of the partitions (Sec. 3.2.1);
//   3    every worker sorts its partition;
//   4    every worker merge-joins its partition with each run from the start
//        found by interpolation search (Sec. 3.2.2).
// The result is the match count and the wrapping u64 sum of r.payload +
// s.payload over all matches, as the GPU library reports them.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

struct Tup {
  uint64_t key, pay;
};

using u64 = uint64_t;
using u32 = uint32_t;

template <class F>
void parallel(u32 T, F f) {
  std::vector<std::thread> th;
  th.reserve(T);
  for (u32 i = 0; i < T; ++i) th.emplace_back(f, i);
  for (auto& t : th) t.join();
}

u64 chunk(u64 n, u32 T, u32 i) { return (u64)(((unsigned __int128)n * i) / T); }

u32 bit_length(u64 x) {
  u32 b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

// LSD radix sort of tuples by key, 8 bits per pass over the key bits that vary
void sort_tuples(Tup* a, Tup* tmp, u64 n, u64 kmin, u64 kmax) {
  if (n < 64) {
    std::sort(a, a + n, [](const Tup& x, const Tup& y) { return x.key < y.key; });
    return;
  }
  const u32 bits = bit_length(kmax - kmin);
  Tup* src = a;
  Tup* dst = tmp;
  for (u32 sh = 0; sh < bits; sh += 8) {
    u64 cnt[257] = {0};
    for (u64 i = 0; i < n; ++i) ++cnt[(((src[i].key - kmin) >> sh) & 255u) + 1];
    for (u32 d = 0; d < 256; ++d) cnt[d + 1] += cnt[d];
    for (u64 i = 0; i < n; ++i) dst[cnt[((src[i].key - kmin) >> sh) & 255u]++] = src[i];
    std::swap(src, dst);
  }
  if (src != a) std::memcpy(a, src, n * sizeof(Tup));
}

void sort_range(Tup* a, Tup* tmp, u64 n) {
  if (!n) return;
  u64 mn = ~0ull, mx = 0;
  for (u64 i = 0; i < n; ++i) {
    mn = std::min(mn, a[i].key);
    mx = std::max(mx, a[i].key);
  }
  sort_tuples(a, tmp, n, mn, mx);
}

// first index of a[0, n) with key >= k: interpolation search between the known
// end keys (Sec. 3.2.2, Fig. 7), finished by bisection after 16 steps
u64 interpolation_search(const Tup* a, u64 n, u64 k) {
  if (n == 0 || a[0].key >= k) return 0;
  if (a[n - 1].key < k) return n;
  u64 L = 0, H = n - 1;  // a[L] < k <= a[H]
  for (int step = 0; step < 16 && H - L > 1; ++step) {
    const double f = (double)(k - a[L].key) / (double)(a[H].key - a[L].key);
    u64 pos = L + (u64)(f * (double)(H - L));
    pos = pos <= L ? L + 1 : (pos >= H ? H - 1 : pos);
    if (a[pos].key < k) L = pos;
    else H = pos;
  }
  u64 lo = L + 1, hi = H;
  while (lo < hi) {
    const u64 mid = lo + (hi - lo) / 2;
    if (a[mid].key < k) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

u64 lower_bound(const Tup* a, u64 n, u64 k) {
  u64 lo = 0;
  while (n) {
    const u64 h = n / 2;
    if (a[lo + h].key < k) {
      lo += h + 1;
      n -= h + 1;
    } else {
      n = h;
    }
  }
  return lo;
}

// split-relevant cost of a partition with n S tuples and r R tuples in range, in 1/65536
u64 split_cost(u64 n, u64 r, u32 T) {
  const double c = (n > 1 ? (double)n * std::log2((double)n) : 0.0) + (double)T * (double)n + (double)r;
  return (u64)std::llround(c * 65536.0);
}

// greedy grouping under the bound C: the number of groups, or UINT32_MAX if a bucket alone exceeds C
u32 group(const std::vector<u64>& H, const std::vector<u64>& G, u32 T, u64 C, std::vector<u32>* sp) {
  const u32 nb = (u32)H.size();
  u32 g = 0, a = 0;
  while (a < nb) {
    u64 n = H[a], r = G[a];
    if (split_cost(n, r, T) > C) return UINT32_MAX;
    u32 b = a + 1;
    while (b < nb && split_cost(n + H[b], r + G[b], T) <= C) {
      n += H[b];
      r += G[b];
      ++b;
    }
    if (sp)
      for (u32 f = a; f < b; ++f) (*sp)[f] = g;
    ++g;
    a = b;
  }
  return g;
}

}  // namespace

extern "C" __attribute__((visibility("default"))) int pmpsm_join(const void* R_, u64 nR, const void* S_, u64 nS,
                                                                  u32 threads, u32 fine_bits, u64* out_count,
                                                                  u64* out_checksum, double* phase_ms) {
  using clk = std::chrono::steady_clock;
  const Tup* R = static_cast<const Tup*>(R_);
  const Tup* S = static_cast<const Tup*>(S_);
  u32 T = threads ? threads : std::max(1u, std::thread::hardware_concurrency());
  if (fine_bits == 0) fine_bits = 10;
  if (fine_bits > 16 || !out_count || !out_checksum) return 1;
  *out_count = 0;
  *out_checksum = 0;
  double ms[5] = {0, 0, 0, 0, 0};
  auto t0 = clk::now();
  auto lap = [&](int i) {
    const auto t = clk::now();
    ms[i] = std::chrono::duration<double, std::milli>(t - t0).count();
    t0 = t;
  };
  if (nR == 0 || nS == 0) {
    if (phase_ms) std::memset(phase_ms, 0, sizeof(ms));
    return 0;
  }
  if (T > nR) T = (u32)nR;

  // phase 1: sorted runs of R
  std::vector<Tup> runs(R, R + nR), tmp(std::max(nR, nS));
  parallel(T, [&](u32 i) {
    const u64 a = chunk(nR, T, i), b = chunk(nR, T, i + 1);
    sort_range(runs.data() + a, tmp.data() + a, b - a);
  });
  u64 kmin = ~0ull, kmax = 0;
  for (u32 i = 0; i < T; ++i) {
    const u64 a = chunk(nR, T, i), b = chunk(nR, T, i + 1);
    if (a < b) {
      kmin = std::min(kmin, runs[a].key);
      kmax = std::max(kmax, runs[b - 1].key);
    }
  }
  lap(0);

  // phase 2.1: R tuples below each fine bucket bound, summed over the runs
  const u32 rbits = bit_length(kmax - kmin);
  const u32 shift = rbits > fine_bits ? rbits - fine_bits : 0;
  const u32 nb = (u32)((kmax - kmin) >> shift) + 1;
  std::vector<u64> below(nb + 1, 0);
  parallel(T, [&](u32 i) {
    for (u32 f = 1 + i; f < nb; f += T) {
      const u64 bound = kmin + ((u64)f << shift);
      u64 c = 0;
      for (u32 j = 0; j < T; ++j) {
        const u64 a = chunk(nR, T, j), b = chunk(nR, T, j + 1);
        c += lower_bound(runs.data() + a, b - a, bound);
      }
      below[f] = c;
    }
  });
  below[nb] = nR;
  std::vector<u64> G(nb);
  for (u32 f = 0; f < nb; ++f) G[f] = below[f + 1] - below[f];

  // phase 2.2: per-worker radix histograms of S over R's key range
  std::vector<std::vector<u64>> h(T, std::vector<u64>(nb, 0));
  parallel(T, [&](u32 i) {
    const u64 a = chunk(nS, T, i), b = chunk(nS, T, i + 1);
    std::vector<u64>& hi = h[i];
    for (u64 t = a; t < b; ++t) {
      const u64 k = S[t].key;
      if (k >= kmin && k <= kmax) ++hi[(k - kmin) >> shift];
    }
  });
  std::vector<u64> H(nb, 0);
  for (u32 i = 0; i < T; ++i)
    for (u32 f = 0; f < nb; ++f) H[f] += h[i][f];

  // phase 2.3: splitters (bisection on the largest cost, greedy feasibility), prefix sums, scatter
  u64 lo = 0, tn = 0, tr = 0;
  for (u32 f = 0; f < nb; ++f) {
    lo = std::max(lo, split_cost(H[f], G[f], T));
    tn += H[f];
    tr += G[f];
  }
  u64 hi = std::max(lo, split_cost(tn, tr, T));
  while (lo < hi) {
    const u64 mid = lo + (hi - lo) / 2;
    if (group(H, G, T, mid, nullptr) <= T) hi = mid;
    else lo = mid + 1;
  }
  std::vector<u32> sp(nb);
  const u32 P = group(H, G, T, lo, &sp);
  // ps[i][p]: where worker i writes its first tuple of partition p
  std::vector<u64> part_off(P + 1, 0);
  std::vector<std::vector<u64>> ps(T, std::vector<u64>(P, 0));
  for (u32 f = 0; f < nb; ++f) part_off[sp[f] + 1] += H[f];
  for (u32 p = 0; p < P; ++p) part_off[p + 1] += part_off[p];
  {
    std::vector<u64> run(part_off.begin(), part_off.end() - 1);
    for (u32 i = 0; i < T; ++i) {
      std::vector<u64> cnt(P, 0);
      for (u32 f = 0; f < nb; ++f) cnt[sp[f]] += h[i][f];
      for (u32 p = 0; p < P; ++p) {
        ps[i][p] = run[p];
        run[p] += cnt[p];
      }
    }
  }
  const u64 kept = part_off[P];
  std::vector<Tup> parts(kept);
  parallel(T, [&](u32 i) {
    const u64 a = chunk(nS, T, i), b = chunk(nS, T, i + 1);
    std::vector<u64> w = ps[i];
    for (u64 t = a; t < b; ++t) {
      const u64 k = S[t].key;
      if (k < kmin || k > kmax) continue;
      parts[w[sp[(k - kmin) >> shift]]++] = S[t];
    }
  });
  lap(1);

  // phase 3: every worker sorts its partition
  parallel(T, [&](u32 i) {
    for (u32 p = i; p < P; p += T) sort_range(parts.data() + part_off[p], tmp.data() + part_off[p], part_off[p + 1] - part_off[p]);
  });
  lap(2);

  // phase 4: merge join of every partition with every run
  std::vector<u64> cnt(T, 0), chk(T, 0);
  parallel(T, [&](u32 i) {
    u64 c = 0, k = 0;
    for (u32 p = i; p < P; p += T) {
      const Tup* s = parts.data() + part_off[p];
      const u64 ns = part_off[p + 1] - part_off[p];
      if (!ns) continue;
      const u64 last = s[ns - 1].key;
      for (u32 j = 0; j < T; ++j) {
        const u64 a = chunk(nR, T, j), b = chunk(nR, T, j + 1);
        const Tup* r = runs.data() + a;
        const u64 nr = b - a;
        u64 x = interpolation_search(r, nr, s[0].key), y = 0;
        while (x < nr && y < ns && r[x].key <= last) {
          if (r[x].key < s[y].key) {
            ++x;
          } else if (s[y].key < r[x].key) {
            ++y;
          } else {
            const u64 key = r[x].key;
            u64 cr = 0, sr = 0, cs = 0, ss = 0;
            for (; x < nr && r[x].key == key; ++x) {
              ++cr;
              sr += r[x].pay;
            }
            for (; y < ns && s[y].key == key; ++y) {
              ++cs;
              ss += s[y].pay;
            }
            c += cr * cs;
            k += cs * sr + cr * ss;
          }
        }
      }
    }
    cnt[i] = c;
    chk[i] = k;
  });
  for (u32 i = 0; i < T; ++i) {
    *out_count += cnt[i];
    *out_checksum += chk[i];
  }
  lap(3);
  if (phase_ms) {
    ms[4] = ms[0] + ms[1] + ms[2] + ms[3];
    std::memcpy(phase_ms, ms, sizeof(ms));
  }
  return 0;
}
