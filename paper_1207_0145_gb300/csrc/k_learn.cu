// k_learn.cu -- training and tabulation of the learned CDF model on the GPU.
//
// Per model (two per job: one over a sorted sample of S, one over positions of
// the sorted R runs, whose ranks are exact), on the plan's stream:
//   k_rmi_setup     normalisation range, cell geometry, initial weights
//   k_fit_data      the model's sample as (key, CDF value) pairs
//   k_train_data    up to 16384 of them, evenly spaced, as (x, y) in FP32
//   k_rmi_grad      forward and backward pass of the root MLP, one partial
//                   gradient per block (128 points)            } x steps
//   k_rmi_adam      sum of the partials in a fixed order, Adam  }
//   k_rmi_tabulate  root evaluated at every cell centre -> leaf index
//   k_leaf_pass<0..2>, k_leaf_solve   least-squares line per leaf
// The forward/backward pass restates the chain rule of the root
// h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), yhat = W3 . h2 + b3 under the
// mean squared error; Adam follows Kingma & Ba (2015) with bias correction.
#include "learn.cuh"
#include "mpsm_launch.h"

namespace mpsm {

namespace {

struct LeafAcc {
  u64 base;
  u32 cnt, pad;
  double sd, sy, sdd, sdy;
};

__device__ __forceinline__ float norm_key(u64 key, u64 kmin, u64 kmax) {
  if (kmax <= kmin) return 0.0f;
  const u64 off = key > kmin ? key - kmin : 0ull;
  const double x = (double)off / (double)(kmax - kmin);
  return (float)(x < 1.0 ? x : 1.0);
}

__device__ __forceinline__ u32 key_cell(const RmiModel& M, u64 key) {
  const u64 off = key > M.kmin ? key - M.kmin : 0ull;
  const u64 c = off >> M.cshift;
  return c >= (u64)M.ncell ? M.ncell - 1u : (u32)c;
}

__device__ __forceinline__ u32 leaf_index(float yhat) {
  const float f = yhat * (float)RMI_LEAVES;
  if (f >= (float)(RMI_LEAVES - 1)) return RMI_LEAVES - 1;
  return f > 0.0f ? (u32)f : 0u;  // NaN lands in leaf 0
}

// root output at x with the weights in shared (or global) memory
__device__ __forceinline__ float root_forward(const float* th, float x) {
  float h1[RMI_H];
#pragma unroll
  for (u32 k = 0; k < RMI_H; ++k) h1[k] = fmaxf(fmaf(th[RO_W1 + k], x, th[RO_B1 + k]), 0.0f);
  float y = th[RO_B3];
#pragma unroll 4
  for (u32 j = 0; j < RMI_H; ++j) {
    float a = th[RO_B2 + j];
#pragma unroll
    for (u32 k = 0; k < RMI_H; ++k) a = fmaf(th[RO_W2 + j * RMI_H + k], h1[k], a);
    y = fmaf(th[RO_W3 + j], fmaxf(a, 0.0f), y);
  }
  return y;
}

__global__ void k_rmi_setup(RmiModel* models, const RmiTask* tasks, const Job* jobs, u32 init) {
  RmiModel& M = models[blockIdx.x];
  const RmiTask T = tasks[blockIdx.x];
  if (threadIdx.x == 0) {
    u64 lo = T.kmin, hi = T.kmax;
    if (T.kind != RMI_KIND_GIVEN) {
      const Job& J = jobs[T.job];
      lo = J.has_range ? J.kmin : 0ull;
      hi = J.has_range ? J.kmax : 0ull;
    }
    M.kmin = lo;
    M.kmax = hi;
    const u32 bits = bitlen64(hi - lo);
    M.cshift = bits > RMI_CELL_BITS ? bits - RMI_CELL_BITS : 0u;
    M.ncell = (u32)((hi - lo) >> M.cshift) + 1u;
    M.fit_off = T.fit_off;
    M.fit_n = 0;
    M.train_n = 0;
    M.loss0 = M.loss = 0.0f;
    M.active = T.active;
  }
  if (init) {
    for (u32 p = threadIdx.x; p < RMI_NPAD; p += blockDim.x) {
      float w = 0.0f;  // start at yhat = x: hinges relu(x - k/32), identity middle layer, read out by unit 0
      if (p < RO_B1) w = 1.0f;
      else if (p < RO_W2) w = -(float)(p - RO_B1) / (float)RMI_H;
      else if (p < RO_B2) w = ((p - RO_W2) / RMI_H == (p - RO_W2) % RMI_H) ? 1.0f : 0.0f;
      else if (p == RO_W3) w = 1.0f;
      M.theta[p] = w;
    }
  }
  for (u32 p = threadIdx.x; p < RMI_NPAD; p += blockDim.x) {
    M.m[p] = 0.0f;
    M.v[p] = 0.0f;
  }
}

template <typename KeyAt>
__device__ __forceinline__ u64 lower_bound_at(KeyAt at, u64 n, u64 key) {
  u64 a = 0, m = n;
  while (m > 0) {
    const u64 h = m >> 1;
    if (at(a + h) < key) {
      a += h + 1;
      m -= h + 1;
    } else {
      m = h;
    }
  }
  return a;
}

__global__ void k_fit_data(RmiModel* models, const RmiTask* tasks, const Job* jobs, const Run* runs, const Tuple* xr,
                           const Tuple* samp, u64* fitk, float* fity) {
  RmiModel& M = models[blockIdx.y];
  const RmiTask T = tasks[blockIdx.y];
  if (!T.active) return;
  if (T.kind == RMI_KIND_GIVEN) {
    if (blockIdx.x == 0 && threadIdx.x == 0) M.fit_n = T.cap;
    return;
  }
  const Job& J = jobs[T.job];
  u64* fk = fitk + T.fit_off;
  float* fy = fity + T.fit_off;
  if (T.kind == RMI_KIND_SAMPLE) {
    // the in-range slice [a, b) of the sorted sample of S
    const Tuple* s = samp + T.src_off;
    auto at = [&](u64 i) { return s[i].key; };
    u64 a = 0, b = 0;
    if (J.has_range) {
      a = lower_bound_at(at, T.cap, J.kmin);
      b = J.kmax == ~0ull ? T.cap : lower_bound_at(at, T.cap, J.kmax + 1ull);
    }
    const u64 n = b - a;
    if (blockIdx.x == 0 && threadIdx.x == 0) M.fit_n = (u32)n;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
      fk[i] = s[a + i].key;
      fy[i] = (float)(((double)i + 0.5) / (double)n);
    }
  } else {
    // evenly spaced positions of the job's runs (back to back in xr); a run's rank is exact
    const u64 m = J.nR ? T.cap : 0ull;
    if (blockIdx.x == 0 && threadIdx.x == 0) M.fit_n = (u32)m;
    const Run* rj = runs + J.run_base;
    for (u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (u64)gridDim.x * blockDim.x) {
      const u64 g = ((2 * t + 1) * J.nR) / (2 * m);
      // run holding position g: last run whose start is <= g
      u32 lo = 0, hi = J.runs - 1;
      while (lo < hi) {
        const u32 mid = (lo + hi + 1) >> 1;
        if (rj[mid].off - J.r_base <= g) lo = mid;
        else hi = mid - 1;
      }
      const Run r = rj[lo];
      const u64 q = g - (r.off - J.r_base);
      fk[t] = xr[J.r_base + g].key;
      fy[t] = (float)(((double)q + 0.5) / (double)r.len);
    }
  }
}

__global__ void k_train_data(RmiModel* models, const u64* fitk, const float* fity, float* X, float* Y) {
  RmiModel& M = models[blockIdx.y];
  if (!M.active) return;
  const u64 n = M.fit_n;
  const u32 tn = (u32)(n < RMI_TRAIN_MAX ? n : RMI_TRAIN_MAX);
  if (blockIdx.x == 0 && threadIdx.x == 0) M.train_n = tn;
  float* x = X + (u64)blockIdx.y * RMI_TRAIN_MAX;
  float* y = Y + (u64)blockIdx.y * RMI_TRAIN_MAX;
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < tn; i += gridDim.x * blockDim.x) {
    const u64 idx = ((2ull * i + 1ull) * n) / (2ull * tn);
    x[i] = norm_key(fitk[M.fit_off + idx], M.kmin, M.kmax);
    y[i] = fity[M.fit_off + idx];
  }
}

// Partial gradient (and loss) of model mdl over its training points [blk RMI_GT,
// (blk + 1) RMI_GT) into out[RMI_NPAD], the weights already in gsm[0, RMI_NPAD).
// RMI_TPP threads share a point: thread sub = tid % RMI_TPP of point tid / RMI_TPP
// owns hidden units sub and sub + RMI_TPP of each layer, so every thread's chains
// are short and a block keeps 16 warps busy.  Shared memory: th[RMI_NPAD] | W2 with
// rows padded to GP floats (the owners of a point read different banks) | h1, h2,
// da2, da1 [RMI_GT][GP] | x, g, l [RMI_GT].  Sums over points run in point order;
// yhat adds its owners' shares.  Every thread of the block calls it; a block without
// points writes zeros.
constexpr u32 GP = 33;
constexpr u32 RMI_TPP = 16;
constexpr u32 RMI_NTH = RMI_GT * RMI_TPP;
static_assert(RMI_H == 2 * RMI_TPP, "two units per owner");
constexpr size_t SMEM_GRAD = (RMI_NPAD + RMI_H * GP + 4 * RMI_GT * GP + 3 * RMI_GT) * sizeof(float);

__device__ __forceinline__ void grad_block(const RmiModel& M, u32 mdl, u32 blk, const float* X, const float* Y,
                                           float* out, float* gsm) {
  float* th = gsm;
  float* w2 = th + RMI_NPAD;
  float* sh1 = w2 + RMI_H * GP;
  float* sh2 = sh1 + RMI_GT * GP;
  float* sda2 = sh2 + RMI_GT * GP;
  float* sda1 = sda2 + RMI_GT * GP;
  float* sx = sda1 + RMI_GT * GP;
  float* sg = sx + RMI_GT;
  float* sl = sg + RMI_GT;
  const u32 tid = threadIdx.x;
  const u32 n = M.active ? M.train_n : 0u;
  if (blk * RMI_GT >= n) {  // no points in this block: a zero partial
    for (u32 p = tid; p < RMI_NPAD; p += RMI_NTH) out[p] = 0.0f;
    return;
  }
  for (u32 e = tid; e < RMI_H * RMI_H; e += RMI_NTH) w2[(e >> 5) * GP + (e & 31u)] = th[RO_W2 + e];
  __syncthreads();
  const u32 pt = tid / RMI_TPP, sub = tid % RMI_TPP;
  const u32 q = blk * RMI_GT + pt;
  const bool valid = q < n;
  const float x = valid ? X[(u64)mdl * RMI_TRAIN_MAX + q] : 0.0f;
  const float yv = valid ? Y[(u64)mdl * RMI_TRAIN_MAX + q] : 0.0f;
  float a1[RMI_H];
#pragma unroll
  for (u32 k = 0; k < RMI_H; ++k) a1[k] = fmaf(th[RO_W1 + k], x, th[RO_B1 + k]);
  float a2[2];
  float part = 0.0f;
#pragma unroll
  for (u32 jj = 0; jj < 2; ++jj) {
    const u32 j = sub + jj * RMI_TPP;
    float a = th[RO_B2 + j];
#pragma unroll
    for (u32 k = 0; k < RMI_H; ++k) a = fmaf(w2[j * GP + k], fmaxf(a1[k], 0.0f), a);
    a2[jj] = a;
    part = fmaf(th[RO_W3 + j], fmaxf(a, 0.0f), part);
  }
#pragma unroll
  for (u32 d = 1; d < RMI_TPP; d <<= 1) part += __shfl_xor_sync(0xffffffffu, part, d);
  const float yh = th[RO_B3] + part;
  const float r = yh - yv;
  const float g = valid ? 2.0f * r / (float)n : 0.0f;
  if (sub == 0) {
    sx[pt] = x;
    sg[pt] = g;
    sl[pt] = valid ? r * r / (float)n : 0.0f;
  }
  // dL/da2 = g W3 [a2 > 0]; h2 = relu(a2)
#pragma unroll
  for (u32 jj = 0; jj < 2; ++jj) {
    const u32 j = sub + jj * RMI_TPP;
    const bool on = a2[jj] > 0.0f;
    sda2[pt * GP + j] = on ? g * th[RO_W3 + j] : 0.0f;
    sh2[pt * GP + j] = on ? a2[jj] : 0.0f;
  }
  __syncwarp();  // a point's owners share a warp
  // dL/da1 = [a1 > 0] W2^T da2, for k = sub, sub + RMI_TPP
#pragma unroll
  for (u32 kk = 0; kk < 2; ++kk) {
    const u32 k = sub + kk * RMI_TPP;
    float t = 0.0f;
#pragma unroll 8
    for (u32 j = 0; j < RMI_H; ++j) t = fmaf(w2[j * GP + k], sda2[pt * GP + j], t);
    const float ak = fmaf(th[RO_W1 + k], x, th[RO_B1 + k]);  // a1[k], recomputed: k depends on the thread
    sda1[pt * GP + k] = (ak > 0.0f && valid) ? t : 0.0f;
    sh1[pt * GP + k] = valid ? fmaxf(ak, 0.0f) : 0.0f;
  }
  __syncthreads();
  // dW2[j][k] = sum_i da2[i][j] h1[i][k]: entries tid + r RMI_NTH (warp: fixed j, k = lane)
  {
    constexpr u32 R = (RMI_H * RMI_H) / RMI_NTH;
    const u32 k = tid & 31u, j0 = tid >> 5;
    float acc[R];
#pragma unroll
    for (u32 rr = 0; rr < R; ++rr) acc[rr] = 0.0f;
#pragma unroll 8
    for (u32 i = 0; i < RMI_GT; ++i) {
      const float h = sh1[i * GP + k];
#pragma unroll
      for (u32 rr = 0; rr < R; ++rr) acc[rr] = fmaf(sda2[i * GP + j0 + rr * (RMI_NTH / 32)], h, acc[rr]);
    }
#pragma unroll
    for (u32 rr = 0; rr < R; ++rr) out[RO_W2 + tid + rr * RMI_NTH] = acc[rr];
  }
  // the other parameters: one sum over the points per thread
  if (tid < 32) {
    float w = 0.0f;
    for (u32 i = 0; i < RMI_GT; ++i) w = fmaf(sda1[i * GP + tid], sx[i], w);
    out[RO_W1 + tid] = w;
  } else if (tid < 64) {
    float bsum = 0.0f;
    for (u32 i = 0; i < RMI_GT; ++i) bsum += sda1[i * GP + tid - 32];
    out[RO_B1 + tid - 32] = bsum;
  } else if (tid < 96) {
    float bsum = 0.0f;
    for (u32 i = 0; i < RMI_GT; ++i) bsum += sda2[i * GP + tid - 64];
    out[RO_B2 + tid - 64] = bsum;
  } else if (tid < 128) {
    float w = 0.0f;
    for (u32 i = 0; i < RMI_GT; ++i) w = fmaf(sg[i], sh2[i * GP + tid - 96], w);
    out[RO_W3 + tid - 96] = w;
  } else if (tid == 128) {
    float bsum = 0.0f;
    for (u32 i = 0; i < RMI_GT; ++i) bsum += sg[i];
    out[RO_B3] = bsum;
  } else if (tid == 129) {
    float l = 0.0f;
    for (u32 i = 0; i < RMI_GT; ++i) l += sl[i];
    out[RMI_NP] = l;
  } else if (tid < 130 + (RMI_NPAD - RMI_NP - 1)) {
    out[RMI_NP + 1 + (tid - 130)] = 0.0f;  // padding slots
  }
  __syncthreads();  // the shared arrays may be written again
}

__global__ void __launch_bounds__(RMI_NTH) k_rmi_grad(const RmiModel* models, const float* X, const float* Y,
                                                      float* partial) {
  extern __shared__ __align__(16) float gsm[];
  const RmiModel& M = models[blockIdx.y];
  const u32 n = M.active ? M.train_n : 0u;
  if (blockIdx.x * RMI_GT < n) {
    for (u32 p = threadIdx.x; p < RMI_NPAD; p += RMI_NTH) gsm[p] = M.theta[p];
    __syncthreads();
  }
  grad_block(M, blockIdx.y, blockIdx.x, X, Y, partial + ((u64)blockIdx.y * RMI_GMAX + blockIdx.x) * RMI_NPAD, gsm);
}

// sum of the block partials of one model, in block order (deterministic)
__device__ __forceinline__ float sum_partial(const float* partial, u32 mdl, u32 p) {
  const float* base = partial + (u64)mdl * RMI_GMAX * RMI_NPAD + p;
  float s = 0.0f;
  for (u32 b = 0; b < RMI_GMAX; ++b) s += base[(u64)b * RMI_NPAD];
  return s;
}

__global__ void __launch_bounds__(1024) k_rmi_adam(RmiModel* models, const float* partial, u32 step, float lr) {
  RmiModel& M = models[blockIdx.x];
  if (!M.active || M.train_n == 0) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.0f - powf(b1, (float)step);
  const float c2 = 1.0f - powf(b2, (float)step);
  for (u32 p = threadIdx.x; p < RMI_NP; p += blockDim.x) {
    const float g = sum_partial(partial, blockIdx.x, p);
    const float m = b1 * M.m[p] + (1.0f - b1) * g;
    const float v = b2 * M.v[p] + (1.0f - b2) * g * g;
    M.m[p] = m;
    M.v[p] = v;
    M.theta[p] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
  }
  if (threadIdx.x == 0) {
    const float l = sum_partial(partial, blockIdx.x, RMI_NP);
    M.loss = l;
    if (step == 1) M.loss0 = l;
  }
}

__global__ void __launch_bounds__(1024) k_rmi_reduce(const float* partial, float* grad, float* loss) {
  for (u32 p = threadIdx.x; p < RMI_NP; p += blockDim.x) grad[p] = sum_partial(partial, 0, p);
  if (threadIdx.x == 0) *loss = sum_partial(partial, 0, RMI_NP);
}

// Barrier of the RMI_GMAX blocks of one model, which a cooperative launch keeps
// resident together: each block adds one to the model's arrival count, which only
// grows, and waits until it reaches RMI_GMAX times the number of barriers passed so
// far; it polls at most `limit` times and then gives up (false).
__device__ __forceinline__ bool model_barrier(u32* cnt, u32& phase, u32 limit) {
  __shared__ u32 s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    u32 ok = 1;
    const u32 target = (phase + 1u) * RMI_GMAX;
    __threadfence();  // this block's partials and parameters before its arrival
    atomicAdd(cnt, 1u);
    u32 it = 0;
    while (*reinterpret_cast<volatile u32*>(cnt) < target) {
      if (++it >= limit) {
        ok = 0;
        break;
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  ++phase;
  return s_ok != 0;
}

constexpr u32 ADAM_SLICE = (RMI_NP + 1 + RMI_GMAX - 1) / RMI_GMAX;  // parameters (and the loss) per block

// Every Adam step of the active models in one launch: grid (RMI_GMAX, models).
// Per step each block writes its partial gradient; after a barrier, block b sums
// the partials of parameters [b ADAM_SLICE, (b + 1) ADAM_SLICE) -- each in a fixed
// order, one warp per parameter -- and applies the same update as k_rmi_adam to
// them; after a second barrier every block reads the new weights.  bar holds two
// zeroed words per model; a barrier that gives up sets DERR_TMA_TIMEOUT in err.
// losses (optional, one model): the loss before each step.
__global__ void __launch_bounds__(RMI_NTH, 2) k_rmi_train(RmiModel* models, const float* X, const float* Y,
                                                      float* partial, u32* bar, u32 steps, float lr, u32 limit,
                                                      float* losses, u32* err) {
  extern __shared__ __align__(16) float gsm[];
  RmiModel& M = models[blockIdx.y];
  if (!M.active || M.train_n == 0) return;  // the same for every block of the model
  const u32 tid = threadIdx.x, lane = lane_id(), wid = warp_id();
  const u32 blk = blockIdx.x, mdl = blockIdx.y;
  u32* cnt = bar + 2 * mdl;
  u32 phase = 0;
  float* out = partial + ((u64)mdl * RMI_GMAX + blk) * RMI_NPAD;
  const float* all = partial + (u64)mdl * RMI_GMAX * RMI_NPAD;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (u32 step = 1; step <= steps; ++step) {
    for (u32 p = tid; p < RMI_NPAD; p += RMI_NTH) gsm[p] = __ldcg(&M.theta[p]);  // other blocks wrote them
    __syncthreads();
    grad_block(M, mdl, blk, X, Y, out, gsm);
    if (!model_barrier(cnt, phase, limit)) {
      if (tid == 0) atomicOr(err, (u32)DERR_TMA_TIMEOUT);
      return;
    }
    const float c1 = 1.0f - powf(b1, (float)step);
    const float c2 = 1.0f - powf(b2, (float)step);
    for (u32 k = wid; k < ADAM_SLICE; k += RMI_NTH / 32) {
      const u32 p = blk * ADAM_SLICE + k;
      if (p > RMI_NP) break;  // the same for the whole warp
      float g = 0.0f;
      for (u32 b = lane; b < RMI_GMAX; b += 32) g += __ldcg(&all[(u64)b * RMI_NPAD + p]);
      g = warp_sum(g);
      if (lane == 0) {
        if (p == RMI_NP) {  // the loss slot
          M.loss = g;
          if (step == 1) M.loss0 = g;
          if (losses) losses[step - 1] = g;
        } else {
          const float m = b1 * M.m[p] + (1.0f - b1) * g;
          const float v = b2 * M.v[p] + (1.0f - b2) * g * g;
          M.m[p] = m;
          M.v[p] = v;
          M.theta[p] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
        }
      }
    }
    if (!model_barrier(cnt, phase, limit)) {
      if (tid == 0) atomicOr(err, (u32)DERR_TMA_TIMEOUT);
      return;
    }
  }
}

__global__ void k_rmi_tabulate(RmiModel* models) {
  __shared__ float th[RMI_NPAD];
  RmiModel& M = models[blockIdx.y];
  if (!M.active) return;
  for (u32 p = threadIdx.x; p < RMI_NPAD; p += blockDim.x) th[p] = M.theta[p];
  __syncthreads();
  const u64 range = M.kmax - M.kmin;
  for (u32 c = blockIdx.x * blockDim.x + threadIdx.x; c < M.ncell; c += gridDim.x * blockDim.x) {
    // centre of cell c, clamped to the range
    const u64 lo = (u64)c << M.cshift;
    u64 mid = lo + ((1ull << M.cshift) >> 1);
    if (mid > range) mid = range;
    const float x = range ? (float)((double)mid / (double)range) : 0.0f;
    M.tab[c] = (u16)leaf_index(root_forward(th, x));
  }
}

__global__ void k_leaf_init(RmiModel* models, LeafAcc* acc) {
  if (!models[blockIdx.y].active) return;
  LeafAcc* A = acc + (u64)blockIdx.y * RMI_LEAVES;
  for (u32 l = blockIdx.x * blockDim.x + threadIdx.x; l < RMI_LEAVES; l += gridDim.x * blockDim.x) {
    A[l].base = ~0ull;
    A[l].cnt = 0;
    A[l].sd = A[l].sy = A[l].sdd = A[l].sdy = 0.0;
  }
}

// Pass 0: smallest key and count per leaf; pass 1: sums of d = key - base and y;
// pass 2: centred sums of d^2 and d*y.  Each thread walks LEAF_CH consecutive fit
// points (consecutive points mostly share a leaf) and flushes its running sums
// with one set of atomics per leaf change.
constexpr u32 LEAF_CH = 16;

template <u32 PASS>
__global__ void k_leaf_pass(const RmiModel* models, LeafAcc* acc, const u64* fitk, const float* fity) {
  const RmiModel& M = models[blockIdx.y];
  if (!M.active) return;
  LeafAcc* A = acc + (u64)blockIdx.y * RMI_LEAVES;
  const u64 n = M.fit_n;
  const u64* fk = fitk + M.fit_off;
  const float* fy = fity + M.fit_off;
  for (u64 i0 = ((u64)blockIdx.x * blockDim.x + threadIdx.x) * LEAF_CH; i0 < n;
       i0 += (u64)gridDim.x * blockDim.x * LEAF_CH) {
    const u64 i1 = i0 + LEAF_CH < n ? i0 + LEAF_CH : n;
    u32 cur = 0xFFFFFFFFu;
    u64 mn = ~0ull;
    u32 cnt = 0;
    double s0 = 0.0, s1 = 0.0;
    u64 base = 0;
    double dm = 0.0, ym = 0.0;
    auto flush = [&]() {
      if (cur == 0xFFFFFFFFu) return;
      if (PASS == 0) {
        atomicMin(&A[cur].base, mn);
        atomicAdd(&A[cur].cnt, cnt);
      } else if (PASS == 1) {
        atomicAdd(&A[cur].sd, s0);
        atomicAdd(&A[cur].sy, s1);
      } else {
        atomicAdd(&A[cur].sdd, s0);
        atomicAdd(&A[cur].sdy, s1);
      }
    };
    for (u64 i = i0; i < i1; ++i) {
      const u64 key = fk[i];
      const u32 l = M.tab[key_cell(M, key)];
      if (l != cur) {
        flush();
        cur = l;
        mn = ~0ull;
        cnt = 0;
        s0 = s1 = 0.0;
        if (PASS > 0) {
          base = A[l].base;
          if (PASS == 2) {
            dm = A[l].sd / (double)A[l].cnt;
            ym = A[l].sy / (double)A[l].cnt;
          }
        }
      }
      if (PASS == 0) {
        mn = key < mn ? key : mn;
        ++cnt;
      } else {
        const double d = (double)(key - base);
        if (PASS == 1) {
          s0 += d;
          s1 += (double)fy[i];
        } else {
          const double dd = d - dm;
          s0 += dd * dd;
          s1 += dd * ((double)fy[i] - ym);
        }
      }
    }
    flush();
  }
}

__global__ void k_leaf_solve(RmiModel* models, const LeafAcc* acc) {
  RmiModel& M = models[blockIdx.y];
  if (!M.active) return;
  const LeafAcc* A = acc + (u64)blockIdx.y * RMI_LEAVES;
  for (u32 l = blockIdx.x * blockDim.x + threadIdx.x; l < RMI_LEAVES; l += gridDim.x * blockDim.x) {
    RmiLeaf L;
    if (A[l].cnt == 0) {
      L.base = 0;
      L.a = 0.0f;
      L.b = ((float)l + 0.5f) / (float)RMI_LEAVES;
    } else {
      const double n = (double)A[l].cnt, dm = A[l].sd / n, ym = A[l].sy / n;
      const double a = A[l].sdd > 0.0 ? A[l].sdy / A[l].sdd : 0.0;
      L.base = A[l].base;
      L.a = (float)a;
      L.b = (float)(ym - a * dm);
    }
    M.leaf[l] = L;
  }
}

// Learned partition boundaries: the P - 1 quantiles p/P of the model's sorted
// in-range sample of S (the empirical inverse CDF the model was trained on),
// with the sample ranks (#keys < and <= the boundary) of each.
__global__ void k_learn_bounds(Job* jobs, const RmiModel* models, const u64* fitk, u64* bnd, u32* brank) {
  Job& J = jobs[blockIdx.x];
  const RmiModel& M = models[2 * blockIdx.x];
  const u64 n = M.fit_n;
  u32 P = J.parts_req ? J.parts_req : 1u;
  if (P > P_MAX) P = P_MAX;
  if ((u64)P > n) P = n ? (u32)n : 1u;
  const u64* fk = fitk + M.fit_off;
  u64* b = bnd + (u64)blockIdx.x * P_MAX;
  u32* r = brank + (u64)blockIdx.x * 2 * P_MAX;
  auto at = [&](u64 i) { return fk[i]; };
  for (u32 p = threadIdx.x + 1; p < P; p += blockDim.x) {
    const u64 key = fk[((u64)p * n) / P];
    b[p - 1] = key;
    r[2 * (p - 1)] = (u32)lower_bound_at(at, n, key);
    r[2 * (p - 1) + 1] = key == ~0ull ? (u32)n : (u32)lower_bound_at(at, n, key + 1ull);
  }
  if (threadIdx.x == 0) J.parts = P;
}

// Fine-cell table: for each fine bucket [lo, hi] of the job's key range, the
// partition its keys fall in when no boundary lies in [lo, hi], else the first and
// last partitions it reaches, marked LCELL_SPLIT (and LCELL_HOT when every boundary
// inside is the same key).
__global__ void k_learn_cells(const Job* jobs, const u64* bnd, u32* cell) {
  const Job& J = jobs[blockIdx.x];
  const u32 nb = J.parts ? J.parts - 1u : 0u;
  const u64* b = bnd + (u64)blockIdx.x * P_MAX;
  auto at = [&](u64 i) { return b[i]; };
  for (u32 f = threadIdx.x; f < J.nfine; f += blockDim.x) {
    const u64 lo = J.kmin + ((u64)f << J.fine_shift);
    const u64 w = (J.fine_shift >= 64) ? ~0ull : ((1ull << J.fine_shift) - 1ull);
    const u64 hi = (J.kmax - lo < w) ? J.kmax : lo + w;
    const u32 plo = (u32)lower_bound_at(at, nb, lo);                                    // #bnd < lo
    const u32 phi = hi == ~0ull ? nb : (u32)lower_bound_at(at, nb, hi + 1ull);          // #bnd <= hi
    const u32 hot = (plo < phi && b[plo] == b[phi - 1]) ? LCELL_HOT : 0u;  // one key is every boundary here
    cell[J.fine_base + f] = plo == phi ? plo : (plo | (phi << 16) | LCELL_SPLIT | hot);
  }
}

// Evenly spaced rows of each job's S, gathered for the sample sort (payload 0).
__global__ void k_sample_s(const Job* jobs, const u64* samp_off, const u32* samp_n, Tuple* samp) {
  const Job& J = jobs[blockIdx.y];
  const u64 m = samp_n[blockIdx.y];
  Tuple* out = samp + samp_off[blockIdx.y];
  for (u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (u64)gridDim.x * blockDim.x) {
    const u64 row = ((2 * t + 1) * J.nS) / (2 * m);
    Tuple v;
    v.key = J.S[row].key;
    v.pay = 0;
    out[t] = v;
  }
}

// Evenly spaced rows of each job's run-side input R, gathered for the sample sort
// that the learned run bucket function is cut from (payload 0).
__global__ void k_sample_r(const Job* jobs, const u64* samp_off, const u32* samp_n, Tuple* samp) {
  const Job& J = jobs[blockIdx.y];
  const u64 m = samp_n[blockIdx.y];
  Tuple* out = samp + samp_off[blockIdx.y];
  for (u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (u64)gridDim.x * blockDim.x) {
    const u64 row = ((2 * t + 1) * J.nR) / (2 * m);
    Tuple v;
    v.key = J.R[row].key;
    v.pay = 0;
    out[t] = v;
  }
}

// One block per job: the learned run bucket function (RunLearn) from the job's sorted
// sample of m run-side keys (sorted[samp_off[j] ...]).  F buckets aim at N_LEAF tuples of
// one run each (the runs of a job have equal lengths), at most P_MAX and at most one per 8
// sample keys; boundary q is the sample key of rank (q + 1) m / F, and the cell table
// marks where boundaries fall, as for the learned partitions (k_learn_cells).
__global__ void k_rlearn_tables(const Job* jobs, const Tuple* sorted, const u64* samp_off, const u32* samp_n,
                                RunLearn* rl, u32* rcell, u64* rbnd) {
  const u32 j = blockIdx.x;
  const Job& J = jobs[j];
  const u64 m = samp_n[j];
  const Tuple* sk = sorted + samp_off[j];
  const u64 run_len = J.runs ? (J.nR + J.runs - 1) / J.runs : 0;
  u64 F = (run_len + N_LEAF - 1) / N_LEAF;
  F = F > P_MAX ? P_MAX : F;
  F = F > m / 8 ? m / 8 : F;
  F = F < 1 ? 1 : F;
  const u32 nb = (u32)F - 1u;
  u64* b = rbnd + (u64)j * P_MAX;
  for (u32 q = threadIdx.x; q < nb; q += blockDim.x) b[q] = sk[((u64)(q + 1) * m) / F].key;
  const u64 lo = m ? sk[0].key : 0ull, hi = m ? sk[m - 1].key : 0ull;
  const u32 bits = bitlen64(hi - lo);
  const u32 shift = bits > 12u ? bits - 12u : 0u;  // at most 4096 = FINE_MAX cells
  const u32 ncell = (u32)((hi - lo) >> shift) + 1u;
  if (threadIdx.x == 0) rl[j] = RunLearn{lo, shift, ncell, (u32)F, (u32)m};
  __syncthreads();  // the boundaries, before the cells search them
  auto at = [&](u64 i) { return b[i]; };
  const u64 w = (1ull << shift) - 1ull;
  for (u32 f = threadIdx.x; f < ncell; f += blockDim.x) {
    const u64 clo = lo + ((u64)f << shift);
    const u64 chi = (hi - clo < w) ? hi : clo + w;
    // the last cell also takes every key above hi, the first every key below lo: no
    // boundary lies there, so the entries below still give their buckets
    const u64 top = f + 1u == ncell ? ~0ull : chi;
    const u32 plo = (u32)lower_bound_at(at, nb, clo);                                 // #bnd < clo
    const u32 phi = top == ~0ull ? nb : (u32)lower_bound_at(at, nb, top + 1ull);      // #bnd <= top
    const u32 hot = (plo < phi && b[plo] == b[phi - 1]) ? LCELL_HOT : 0u;
    rcell[(u64)j * FINE_MAX + f] = plo == phi ? plo : (plo | (phi << 16) | LCELL_SPLIT | hot);
  }
}

__global__ void k_rmi_predict(const RmiModel* M, const u64* keys, u64 n, float* yhat, u32* leaf) {
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
    const u64 k = keys[i];
    yhat[i] = rmi_predict(M, k);
    if (leaf) leaf[i] = M->tab[key_cell(*M, k)];
  }
}

}  // namespace

void launch_sample_s(const Job* jobs, u32 njobs, const u64* samp_off, const u32* samp_n, Tuple* samp,
                     cudaStream_t st, int nsm) {
  k_sample_s<<<dim3(nsm, njobs), 256, 0, st>>>(jobs, samp_off, samp_n, samp);
}

void launch_sample_r(const Job* jobs, u32 njobs, const u64* samp_off, const u32* samp_n, Tuple* samp,
                     cudaStream_t st, int nsm) {
  k_sample_r<<<dim3(nsm, njobs), 256, 0, st>>>(jobs, samp_off, samp_n, samp);
}

void launch_rlearn_tables(const Job* jobs, u32 njobs, const Tuple* sorted, const u64* samp_off, const u32* samp_n,
                          RunLearn* rl, u32* rcell, u64* rbnd, cudaStream_t st) {
  k_rlearn_tables<<<njobs, 1024, 0, st>>>(jobs, sorted, samp_off, samp_n, rl, rcell, rbnd);
}

void launch_learn_cells(const Job* jobs, u32 njobs, const u64* bnd, u32* cell, cudaStream_t st) {
  k_learn_cells<<<njobs, 1024, 0, st>>>(jobs, bnd, cell);
}

void launch_rmi_predict(const RmiModel* M, const u64* keys, u64 n, float* yhat, u32* leaf, cudaStream_t st, int nsm) {
  if (n) k_rmi_predict<<<nsm * 4, 256, 0, st>>>(M, keys, n, yhat, leaf);
}

void init_attrs_learn() {
  cudaFuncSetAttribute(k_rmi_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_GRAD);
  cudaFuncSetAttribute(k_rmi_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_GRAD);
}

// blocks of k_rmi_train that can be resident at once on this device
u32 rmi_train_capacity(int dev) {
  int per_sm = 0, nsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rmi_train, RMI_NTH, SMEM_GRAD) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (u32)(per_sm > 0 ? per_sm : 0) * (u32)(nsm > 0 ? nsm : 0);
}

// All steps in one cooperative launch (bar: 2 u32 per model, zeroed here first).
cudaError_t launch_rmi_train(RmiModel* models, u32 nmodels, const float* X, const float* Y, float* partial, u32* bar,
                             u32 steps, float lr, float* losses, u32* err, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(bar, 0, 2ull * nmodels * sizeof(u32), st);
  if (e != cudaSuccess) return e;
  u32 limit = 1u << 22;  // polls of a barrier (at least 64 ns each) before it gives up
  void* args[] = {&models, &X, &Y, &partial, &bar, &steps, &lr, &limit, &losses, &err};
  return cudaLaunchCooperativeKernel((const void*)k_rmi_train, dim3(RMI_GMAX, nmodels), dim3(RMI_NTH), args,
                                     SMEM_GRAD, st);
}

size_t leaf_acc_bytes() { return sizeof(LeafAcc) * RMI_LEAVES; }

void launch_rmi_setup(RmiModel* models, const RmiTask* tasks, u32 nmodels, const Job* jobs, bool init,
                      cudaStream_t st) {
  k_rmi_setup<<<nmodels, 256, 0, st>>>(models, tasks, jobs, init ? 1u : 0u);
}

void launch_fit_data(RmiModel* models, const RmiTask* tasks, u32 nmodels, const Job* jobs, const Run* runs,
                     const Tuple* xr, const Tuple* samp, u64* fitk, float* fity, cudaStream_t st, int nsm) {
  k_fit_data<<<dim3(nsm, nmodels), 256, 0, st>>>(models, tasks, jobs, runs, xr, samp, fitk, fity);
}

void launch_train_data(RmiModel* models, u32 nmodels, const u64* fitk, const float* fity, float* X, float* Y,
                       cudaStream_t st) {
  k_train_data<<<dim3(16, nmodels), 256, 0, st>>>(models, fitk, fity, X, Y);
}

void launch_rmi_grad(const RmiModel* models, u32 nmodels, const float* X, const float* Y, float* partial,
                     cudaStream_t st) {
  k_rmi_grad<<<dim3(RMI_GMAX, nmodels), RMI_NTH, SMEM_GRAD, st>>>(models, X, Y, partial);
}

void launch_rmi_adam(RmiModel* models, u32 nmodels, const float* partial, u32 step, float lr, cudaStream_t st) {
  k_rmi_adam<<<nmodels, 1024, 0, st>>>(models, partial, step, lr);
}

void launch_rmi_reduce(const float* partial, float* grad, float* loss, cudaStream_t st) {
  k_rmi_reduce<<<1, 1024, 0, st>>>(partial, grad, loss);
}

void launch_rmi_tabulate(RmiModel* models, u32 nmodels, cudaStream_t st) {
  k_rmi_tabulate<<<dim3(RMI_CELLS / 256, nmodels), 256, 0, st>>>(models);
}

void launch_leaf_fit(RmiModel* models, u32 nmodels, void* acc, const u64* fitk, const float* fity, cudaStream_t st,
                     int nsm) {
  LeafAcc* A = reinterpret_cast<LeafAcc*>(acc);
  k_leaf_init<<<dim3(16, nmodels), 256, 0, st>>>(models, A);
  k_leaf_pass<0><<<dim3(nsm, nmodels), 256, 0, st>>>(models, A, fitk, fity);
  k_leaf_pass<1><<<dim3(nsm, nmodels), 256, 0, st>>>(models, A, fitk, fity);
  k_leaf_pass<2><<<dim3(nsm, nmodels), 256, 0, st>>>(models, A, fitk, fity);
  k_leaf_solve<<<dim3(16, nmodels), 256, 0, st>>>(models, A);
}

void launch_learn_bounds(Job* jobs, u32 njobs, const RmiModel* models, const u64* fitk, u64* bnd, u32* brank,
                         cudaStream_t st) {
  k_learn_bounds<<<njobs, 256, 0, st>>>(jobs, models, fitk, bnd, brank);
}

}  // namespace mpsm
