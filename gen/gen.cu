/*
 * gen.cu -- host and device fills of the synthetic workloads in gen_core.h.
 *
 * Input generation only: tests, the benchmark and the oracle's closed forms call
 * it; the join library never does.  Host fills split the index range over
 * std::threads; device fills are one grid-stride kernel.  Both evaluate the same
 * gen_core.h functions, so for the same spec they write identical bytes.
 */
#include <cuda_runtime.h>
#include <stdint.h>
#include <thread>
#include <vector>
#include <algorithm>

#include "gen_core.h"

#define GEN_EXPORT extern "C" __attribute__((visibility("default")))

namespace {

enum { FILL_R = 0, FILL_S = 1, FILL_SROW = 2 };

__global__ void k_fill(gen_spec_t spec, int what, gen_tuple_t* out, uint64_t* rows,
                       uint64_t begin, uint64_t count) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += stride) {
    const uint64_t i = begin + t;
    if (what == FILL_R) {
      gen_tuple_t v;
      v.key = gen_r_key(&spec, i);
      v.payload = gen_r_payload(&spec, i);
      out[t] = v;
    } else if (what == FILL_S) {
      gen_tuple_t v;
      v.key = gen_s_key(&spec, i);
      v.payload = gen_s_payload(&spec, i);
      out[t] = v;
    } else {
      rows[t] = gen_s_row(&spec, i);
    }
  }
}

template <class F>
void host_parallel(uint64_t count, int nthreads, F&& body) {
  if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());
  if (count < (1u << 16)) nthreads = 1;
  std::vector<std::thread> pool;
  const uint64_t per = (count + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    const uint64_t a = (uint64_t)t * per, b = std::min<uint64_t>(count, a + per);
    if (a >= b) break;
    pool.emplace_back([=, &body] { body(a, b); });
  }
  for (auto& th : pool) th.join();
}

int fill(const gen_spec_t* spec, int what, gen_tuple_t* out, uint64_t* rows, uint64_t begin,
         uint64_t count, int device, void* stream, int nthreads) {
  if (!spec) return 1;
  if (count == 0) return 0;
  if (device) {
    const int threads = 256;
    const uint64_t want = (count + threads - 1) / threads;
    const int blocks = (int)std::min<uint64_t>(want, 152ull * 16ull);
    k_fill<<<blocks, threads, 0, (cudaStream_t)stream>>>(*spec, what, out, rows, begin, count);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
  }
  const gen_spec_t s = *spec;
  host_parallel(count, nthreads, [&](uint64_t a, uint64_t b) {
    for (uint64_t t = a; t < b; ++t) {
      const uint64_t i = begin + t;
      if (what == FILL_R) {
        out[t].key = gen_r_key(&s, i);
        out[t].payload = gen_r_payload(&s, i);
      } else if (what == FILL_S) {
        out[t].key = gen_s_key(&s, i);
        out[t].payload = gen_s_payload(&s, i);
      } else {
        rows[t] = gen_s_row(&s, i);
      }
    }
  });
  return 0;
}

}  // namespace

/* R rows [begin, begin+count) into out (host or device memory per `device`). */
GEN_EXPORT int gen_fill_r(const gen_spec_t* spec, gen_tuple_t* out, uint64_t begin, uint64_t count,
                          int device, void* stream, int nthreads) {
  return fill(spec, FILL_R, out, nullptr, begin, count, device, stream, nthreads);
}

/* S tuples [begin, begin+count). */
GEN_EXPORT int gen_fill_s(const gen_spec_t* spec, gen_tuple_t* out, uint64_t begin, uint64_t count,
                          int device, void* stream, int nthreads) {
  return fill(spec, FILL_S, out, nullptr, begin, count, device, stream, nthreads);
}

/* Generator bookkeeping: the R row each S tuple was drawn from (GEN_NONE = no match). */
GEN_EXPORT int gen_s_rows(const gen_spec_t* spec, uint64_t* rows, uint64_t begin, uint64_t count,
                          int device, void* stream, int nthreads) {
  return fill(spec, FILL_SROW, nullptr, rows, begin, count, device, stream, nthreads);
}

GEN_EXPORT uint32_t gen_half_width(uint64_t n) { return gen_half_bits(n); }

GEN_EXPORT uint64_t gen_sorted_key(const gen_spec_t* spec, uint64_t g) {
  return gen_sparse_key(spec, g);
}

GEN_EXPORT uint64_t gen_permute(uint64_t i, uint64_t n, uint64_t seed, uint64_t stream) {
  return gen_perm(i, n, gen_half_bits(n), gen_perm_key(seed, stream));
}

GEN_EXPORT uint64_t gen_permute_inv(uint64_t y, uint64_t n, uint64_t seed, uint64_t stream) {
  return gen_perm_inv(y, n, gen_half_bits(n), gen_perm_key(seed, stream));
}

GEN_EXPORT uint64_t gen_draw(uint64_t seed, uint64_t stream, uint64_t i) {
  return gen_rand(seed, stream, i);
}
