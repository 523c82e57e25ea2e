// api.cu -- libmpsm: plan management, phase orchestration and the C ABI (include/mpsm.h).
//
// Every phase is a fixed sequence of kernel launches on the plan's stream; work
// lists (segments, chunks, tiles) live on the device, so the host never needs
// the data-dependent sizes.  The host only reads back the number of segments
// still too big after a radix pass (one 4-byte copy per pass) to stop early;
// the batched path replaces that check by a fixed number of passes so that the
// whole sequence can be captured into a CUDA graph.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cstddef>
#include <chrono>
#include <new>
#include <vector>

#include "mpsm.h"
#include "mpsm_internal.cuh"
#include "mpsm_launch.h"

using namespace mpsm;

#define MPSM_API extern "C" __attribute__((visibility("default")))

namespace {

constexpr u64 CH_RADIX = 131072;  // tuples per chunk in the sort passes
// counters in d_cnt
enum { C_BIG0 = 0, C_BIG1 = 1, C_FIN = 2, C_WORK = 3, C_WORK2 = 4, C_ERR = 5, C_SPLIT = 6, C_NUM = 8 };
// totals in d_tot
enum { T_LEVEL = 0, T_FINE = 3, T_SPLIT = 6, T_TILES = 9, T_PAIRS = 13, T_NUM = 16 };
enum Stage { ST_NONE = 0, ST_RUNS, ST_SPLIT, ST_SCATTER, ST_SORTED, ST_SEARCH, ST_DONE };
enum { EV_START = 0, EV_RUNS, EV_LEARN, EV_SPLIT, EV_SCATTER, EV_SORTS, EV_SEARCH, EV_JOIN, EV_NUM };

struct Jobh {
  const Tuple* R;
  const Tuple* S;
  u64 nR, nS;
};

// kernel families for launch counting and per-kernel timing
enum Kid {
  K_SAMPLE, K_PLAN, K_INIT, K_HIST_RADIX, K_SCAN_RADIX, K_SCATTER_RADIX, K_SEG_SORT, K_RUN_BOUNDS, K_HIST_FINE,
  K_RUN_CDF, K_SPLITTERS, K_FOLD, K_SCAN_SPLIT, K_SCATTER_SPLIT, K_TILES, K_SEARCH, K_JOIN, K_PAIR_OFFSETS, K_CHECK,
  K_SAMPLE_S, K_RMI_DATA, K_RMI_GRAD, K_RMI_ADAM, K_RMI_TAB, K_RMI_LEAF, K_LEARN_BOUNDS, K_HIST_LEARN, K_SCAN_LEARN,
  K_SCATTER_LEARN, K_FENCES, K_SEG_SEARCH, K_SORT_JOIN, K_RMI_TRAIN, K_SAMPLE_R, K_RLEARN_TAB, K_HIST_RLEARN,
  K_SCATTER_RLEARN, K_NUM
};
const char* const KNAME[K_NUM] = {"sample_bounds", "level_plan", "init_buckets", "hist_radix", "scan_radix",
                                  "scatter_radix", "seg_sort", "run_bounds", "hist_fine", "run_cdf", "splitters",
                                  "fold", "scan_split", "scatter_split", "tiles", "search", "join", "pair_offsets",
                                  "check_empty", "sample_s", "rmi_data", "rmi_grad", "rmi_adam", "rmi_tabulate",
                                  "rmi_leaves", "learn_bounds", "hist_learn", "scan_learn", "scatter_learn",
                                  "fences", "seg_search", "sort_join", "rmi_train", "sample_r", "rlearn_tables",
                                  "hist_rlearn", "scatter_rlearn"};
// learned model: sample and training sizes
constexpr u32 RMI_SAMPLE_MAX = 1u << 21;  // largest sample per model
constexpr u32 RMI_STEPS = 200;            // full-batch Adam steps
constexpr float RMI_LR = 3e-3f;
u32 rmi_sample_size(u64 n) {
  if (n == 0) return 0;
  u64 m = std::max<u64>(std::min<u64>(n, 1024), n / 64);
  return (u32)std::min<u64>(m, RMI_SAMPLE_MAX);
}
constexpr u32 KT_POOL = 1024;

}  // namespace

struct mpsm_plan {
  int device = 0, nsm = 0;
  cudaStream_t st = nullptr;
  mpsm_options_t opt{};
  u64 max_nR = 0, max_nS = 0;
  u32 max_jobs = 1;
  // data buffers
  Tuple *xr = nullptr, *xs = nullptr, *y = nullptr;
  Tuple *stage_r = nullptr, *stage_s = nullptr;
  // mpsm_join_host: the partitioned side's copy runs on its own stream, so the run
  // side's sort overlaps it; the join waits for it before it first reads that side
  cudaStream_t st_copy = nullptr;
  cudaEvent_t ev_run_copied = nullptr, ev_part_copied = nullptr;
  bool part_copy_pending = false;
  bool runs_reused = false;         // a later piece of a host join: the runs' fences and per-bucket
                                    // counts from the first piece still hold
  // piecewise host join: one event per piece of the partitioned side that has landed
  static constexpr u32 MAX_PIECES = 64;
  cudaEvent_t ev_piece[MAX_PIECES] = {};
  u32 device_errors = 0;            // MPSM_DEVERR_* bits read back by the last call
  // job / run tables
  Job *d_jobs = nullptr, *h_jobs = nullptr;
  Run *d_runs = nullptr, *h_runs = nullptr;
  u32 runs_cap = 0;
  // work lists
  Seg *d_split = nullptr, *h_segs = nullptr;
  Seg *d_big[2] = {nullptr, nullptr}, *d_fin = nullptr;
  u32 big_cap = 0, fin_cap = 0, hseg_cap = 0;
  u32 *d_cnt = nullptr, *h_cnt = nullptr;
  // per-pass arrays
  LSeg *d_ls = nullptr, *d_ls2 = nullptr;
  u64* d_tot = nullptr;
  u32 *d_hist_a = nullptr, *d_hist_b = nullptr;
  u64 hist_a_cap = 0, hist_b_cap = 0;
  u64 *d_bmin = nullptr, *d_bmax = nullptr;
  u64 bucket_cap = 0;
  // splitters
  u64 *d_fine_s = nullptr, *d_fine_min = nullptr, *d_fine_max = nullptr, *d_fine_r = nullptr, *d_rc = nullptr;
  u32 *d_sp = nullptr, *d_fstart = nullptr;
  u64* d_part_off = nullptr;
  // join
  u32* d_win = nullptr;
  u64 win_cap = 0;
  u64 *d_tile_cnt = nullptr, *d_tile_out = nullptr;
  u64 tile_cap = 0;
  u64* d_chunk_off = nullptr;
  u64 chunk_off_cap = 0;
  u64* h_scalar = nullptr;  // pinned scratch for small reads
  // state of the current call
  int stage = ST_NONE;
  u32 njobs = 0;
  u64 ch_s = 0;
  u32 tile = 4096;
  u32 levels_r = 0, levels_s = 0;
  u64 segs_r = 0, segs_s = 0;
  bool graph_mode = false;
  bool own_stream = false;
  cudaEvent_t ev[EV_NUM] = {};
  bool timing = false;
  // launch counting / per-kernel timing
  u32 launches = 0;
  cudaEvent_t* kt_ev = nullptr;
  u32 kt_id[KT_POOL];
  u32 kt_n = 0;
  // batched graph
  cudaGraphExec_t gexec = nullptr;
  std::vector<u64> gsig;
  u32 graph_launches = 0;           // kernels in the captured graph
  // fused phases 3 + 4
  bool fused = false;               // the current call joins S segments inside their final sort
  u32 maxT = 1;                     // largest T_R of the current call's jobs
  u64* d_fence = nullptr;           // every 64th key of the sorted runs
  u32* d_swin = nullptr;            // per (final S segment, run) windows
  u64 swin_cap = 0;
  // learned CDF model (allocated on first use)
  bool learn = false;               // the current call uses a learned mode
  RmiModel* d_models = nullptr;     // 2 per job
  RmiTask *d_tasks = nullptr, *h_tasks = nullptr;
  void* d_leafacc = nullptr;
  float *d_tx = nullptr, *d_ty = nullptr, *d_partial = nullptr;
  u32* d_trainbar = nullptr;        // barrier words of the one-launch trainer, 2 per model
  u32 train_cap = 0;                // its blocks that fit on the device at once
  u64* d_fitk = nullptr;
  float* d_fity = nullptr;
  u64 fit_cap = 0;
  Tuple* d_samp = nullptr;          // unsorted S samples (the sub-plan's R input)
  u64 samp_cap = 0;
  u64 *d_samp_off = nullptr, *h_samp_off = nullptr;
  u32 *d_samp_n = nullptr, *h_samp_n = nullptr;
  u64* d_bnd = nullptr;             // learned partition boundaries, P_MAX per job
  u32* d_brank = nullptr;           // their sample ranks, 2 P_MAX per job
  u64* d_lstat = nullptr;           // learned-path counters (LearnCtx::stat)
  mpsm_plan* sub = nullptr;         // sorts the S samples (one run per job)
  // learned run bucket function (MPSM_RUNS_LEARNED)
  RunLearn* d_rl = nullptr;         // per job
  u32* d_rcell = nullptr;           // cell tables, FINE_MAX per job
  u64* d_rbnd = nullptr;            // boundaries, P_MAX per job
  Tuple* d_rsamp = nullptr;         // unsorted run-side samples (the run sub-plan's R input)
  u64 rsamp_cap = 0;
  u64 *d_rsamp_off = nullptr, *h_rsamp_off = nullptr;
  u32 *d_rsamp_n = nullptr, *h_rsamp_n = nullptr;
  mpsm_plan* rsub = nullptr;        // sorts the run-side samples (one run per job)
};

namespace {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? MPSM_OK : MPSM_ERR_CUDA; }

#define CK(x)                                          \
  do {                                                 \
    cudaError_t e_ = (x);                              \
    if (e_ != cudaSuccess) {                           \
      return e_ == cudaErrorMemoryAllocation ? MPSM_ERR_OOM : MPSM_ERR_CUDA; \
    }                                                  \
  } while (0)

template <typename T>
int dalloc(T** p, u64 n) {
  *p = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return MPSM_ERR_OOM;
  }
  return MPSM_OK;
}

template <typename T>
int halloc(T** p, u64 n) {
  *p = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMallocHost((void**)p, n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return MPSM_ERR_OOM;
  }
  return MPSM_OK;
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

template <typename T>
void hfree(T*& p) {
  if (p) cudaFreeHost(p);
  p = nullptr;
}

u64 chunk_start(u64 n, u64 T, u64 j) { return (u64)(((unsigned __int128)n * j) / T); }

u32 auto_runs(u64 nR) {
  // runs of at most ~2048 sort buckets x 6K tuples finish in one radix pass + the SMEM sort;
  // small inputs keep the paper's T = 32 while each run still spans a few SMEM tiles
  const u64 per = 2048ull * 6144ull;
  u64 t = (nR + per - 1) / per;
  const u64 small = std::min<u64>(32, (nR + NMAX - 1) / NMAX);
  t = std::max<u64>(t, small);
  return (u32)std::min<u64>(std::max<u64>(t, 1), RUNS_MAX);
}

u32 auto_parts(u64 nS) {
  // phase 2's scatter fans out to P partitions and phase 3's first pass to about
  // nS / (P * N_LEAF) buckets; P near sqrt(nS / N_LEAF) keeps both fan-outs moderate
  u64 p = 32;
  while (p < P_MAX && (p * 2) * (p * 2) * N_LEAF <= nS * 2) p <<= 1;
  return (u32)p;
}

u32 runs_for(const mpsm_plan* p, u64 nR) {
  u32 t = p->opt.runs_r ? p->opt.runs_r
                        : (p->opt.run_len ? (u32)std::min<u64>((nR + p->opt.run_len - 1) / p->opt.run_len, RUNS_MAX)
                                          : auto_runs(nR));
  if (nR && t > nR) t = (u32)nR;
  return std::max<u32>(1, std::min<u32>(t, RUNS_MAX));
}

Bufs bufs(const mpsm_plan* p) { return Bufs{p->xr, p->xs, p->y}; }

bool split_learned(const mpsm_plan* p) { return p->opt.splitter_mode == MPSM_SPLIT_LEARNED; }
bool runs_learned(const mpsm_plan* p) { return p->opt.run_buckets == MPSM_RUNS_LEARNED; }
bool search_learned(const mpsm_plan* p) { return p->opt.search_mode == MPSM_SEARCH_LEARNED; }

LearnCtx lctx(const mpsm_plan* p, bool models) {
  LearnCtx c{};
  c.models = models ? p->d_models : nullptr;
  c.bnd = p->d_bnd;
  c.brank = p->d_brank;
  c.cell = p->d_sp;  // the fine bucket -> partition array doubles as the learned cell table
  c.seed = p->opt.seed;
  c.stat = p->d_lstat;
  c.interp = p->opt.search_mode == MPSM_SEARCH_INTERP;
  c.rl = p->d_rl;
  c.rcell = p->d_rcell;
  c.rbnd = p->d_rbnd;
  return c;
}

void record(mpsm_plan* p, int i) {
  if (p->timing) cudaEventRecord(p->ev[i], p->st);
}

bool kernel_timing(const mpsm_plan* p) { return (p->opt.flags & MPSM_FLAG_KERNEL_TIMING) && p->kt_ev && !p->graph_mode; }

void kt_begin(mpsm_plan* p, u32 id) {
  p->launches += (id == K_SEG_SORT) ? 2u : 1u;  // the unfused final sort is two kernels (size classes)
  if (kernel_timing(p) && p->kt_n < KT_POOL) {
    p->kt_id[p->kt_n] = id;
    cudaEventRecord(p->kt_ev[2 * p->kt_n], p->st);
  }
}

void kt_end(mpsm_plan* p) {
  if (kernel_timing(p) && p->kt_n < KT_POOL) {
    cudaEventRecord(p->kt_ev[2 * p->kt_n + 1], p->st);
    ++p->kt_n;
  }
}

// MPSM_DEBUG=1 in the environment: synchronise after every launch and name the
// kernel family that failed on stderr (diagnostics only; off by default)
bool debug_sync() {
  static const int on = [] {
    const char* e = getenv("MPSM_DEBUG");
    return e && e[0] == '1';
  }();
  return on;
}

int debug_check(mpsm_plan* p, u32 id) {
  if (!debug_sync() || p->graph_mode) return MPSM_OK;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
  if (e != cudaSuccess) {
    fprintf(stderr, "mpsm debug: kernel family %s failed: %s\n", KNAME[id], cudaGetErrorString(e));
    return MPSM_ERR_CUDA;
  }
  u32 err = 0;
  cudaMemcpy(&err, &p->d_cnt[C_ERR], sizeof(u32), cudaMemcpyDeviceToHost);
  if (err) fprintf(stderr, "mpsm debug: device error flags 0x%x after %s\n", err, KNAME[id]);
  return MPSM_OK;
}

#define LAUNCH(id, call)                  \
  do {                                    \
    kt_begin(p, id);                      \
    call;                                 \
    kt_end(p);                            \
    if (debug_check(p, id)) return MPSM_ERR_CUDA; \
  } while (0)

int setup_jobs(mpsm_plan* p, const Jobh* jobs, u32 njobs);

// ---------------------------------------------------------------- learned model state
int alloc_learn(mpsm_plan* p) {
  if (p->d_models) return MPSM_OK;
  const u64 nm = 2ull * p->max_jobs;
  p->samp_cap = p->max_nS / 64 + 1024ull * p->max_jobs + 16;
  p->fit_cap = p->samp_cap + p->max_nR / 64 + 1024ull * p->max_jobs + 16;
  if (dalloc(&p->d_models, nm) || dalloc(&p->d_tasks, nm) || halloc(&p->h_tasks, nm)) return MPSM_ERR_OOM;
  if (cudaMalloc(&p->d_leafacc, leaf_acc_bytes() * nm) != cudaSuccess) {
    cudaGetLastError();
    p->d_leafacc = nullptr;
    return MPSM_ERR_OOM;
  }
  if (dalloc(&p->d_tx, nm * RMI_TRAIN_MAX) || dalloc(&p->d_ty, nm * RMI_TRAIN_MAX) ||
      dalloc(&p->d_partial, nm * RMI_GMAX * RMI_NPAD) || dalloc(&p->d_fitk, p->fit_cap) ||
      dalloc(&p->d_fity, p->fit_cap) || dalloc(&p->d_samp, p->samp_cap) || dalloc(&p->d_samp_off, p->max_jobs) ||
      halloc(&p->h_samp_off, p->max_jobs) || dalloc(&p->d_samp_n, p->max_jobs) || halloc(&p->h_samp_n, p->max_jobs) ||
      dalloc(&p->d_bnd, (u64)p->max_jobs * P_MAX) || dalloc(&p->d_brank, 2ull * p->max_jobs * P_MAX) ||
      dalloc(&p->d_trainbar, 2 * nm))
    return MPSM_ERR_OOM;
  p->train_cap = rmi_train_capacity(p->device);
  CK(cudaMemsetAsync(p->d_models, 0, nm * sizeof(RmiModel), p->st));
  mpsm_options_t so;
  mpsm_options_default(&so);
  so.runs_r = 1;  // each job's sample is one run
  mpsm_plan_t* sub = nullptr;
  const int rc = mpsm_plan_create(&sub, p->samp_cap, 16, p->max_jobs, &so, p->st);
  if (rc) return rc;
  p->sub = sub;
  return MPSM_OK;
}

// learned run bucket function: tables, the run-side samples and the plan that sorts them
int alloc_rlearn(mpsm_plan* p) {
  if (p->d_rl) return MPSM_OK;
  p->rsamp_cap = p->max_nR / 64 + 1024ull * p->max_jobs + 16;
  if (dalloc(&p->d_rl, p->max_jobs) || dalloc(&p->d_rcell, (u64)p->max_jobs * FINE_MAX) ||
      dalloc(&p->d_rbnd, (u64)p->max_jobs * P_MAX) ||
      dalloc(&p->d_rsamp, p->rsamp_cap) || dalloc(&p->d_rsamp_off, p->max_jobs) ||
      halloc(&p->h_rsamp_off, p->max_jobs) || dalloc(&p->d_rsamp_n, p->max_jobs) || halloc(&p->h_rsamp_n, p->max_jobs))
    return MPSM_ERR_OOM;
  mpsm_options_t so;
  mpsm_options_default(&so);
  so.runs_r = 1;  // each job's sample is one run
  mpsm_plan_t* rsub = nullptr;
  const int rc = mpsm_plan_create(&rsub, p->rsamp_cap, 16, p->max_jobs, &so, p->st);
  if (rc) return rc;
  p->rsub = rsub;
  return MPSM_OK;
}

// sample sizes and the sample sort's jobs of a call with learned run buckets
int setup_rlearn(mpsm_plan* p, const Jobh* jobs, u32 njobs) {
  int rc = alloc_rlearn(p);
  if (rc) return rc;
  std::vector<Jobh> rj(njobs);
  u64 so = 0;
  for (u32 i = 0; i < njobs; ++i) {
    const u32 m = rmi_sample_size(p->h_jobs[i].nR);
    p->h_rsamp_off[i] = so;
    p->h_rsamp_n[i] = m;
    rj[i] = Jobh{p->d_rsamp + so, nullptr, m, 0};
    so += m;
  }
  if (so > p->rsamp_cap) return MPSM_ERR_INVALID_ARG;
  CK(cudaMemcpyAsync(p->d_rsamp_off, p->h_rsamp_off, njobs * sizeof(u64), cudaMemcpyHostToDevice, p->st));
  CK(cudaMemcpyAsync(p->d_rsamp_n, p->h_rsamp_n, njobs * sizeof(u32), cudaMemcpyHostToDevice, p->st));
  CK(cudaStreamSynchronize(p->st));
  return setup_jobs(p->rsub, rj.data(), njobs);
}

// sample sizes, model tasks and the sample sort's jobs of a learned call
int setup_learn(mpsm_plan* p, const Jobh* jobs, u32 njobs) {
  int rc = alloc_learn(p);
  if (rc) return rc;
  const bool sl = split_learned(p), rl = search_learned(p);
  std::vector<Jobh> sj(njobs);
  u64 so = 0, fo = 0;
  for (u32 i = 0; i < njobs; ++i) {
    const u32 ms = sl ? rmi_sample_size(jobs[i].nS) : 0u;
    const u32 mr = rl ? rmi_sample_size(jobs[i].nR) : 0u;
    p->h_samp_off[i] = so;
    p->h_samp_n[i] = ms;
    sj[i] = Jobh{p->d_samp + so, nullptr, ms, 0};
    p->h_tasks[2 * i] = RmiTask{fo, so, 0, 0, i, RMI_KIND_SAMPLE, ms, (u32)(ms > 0)};
    fo += ms;
    so += ms;
    p->h_tasks[2 * i + 1] = RmiTask{fo, 0, 0, 0, i, RMI_KIND_RUNS, mr, (u32)(mr > 0)};
    fo += mr;
  }
  if (so > p->samp_cap || fo > p->fit_cap) return MPSM_ERR_INVALID_ARG;
  CK(cudaMemcpyAsync(p->d_tasks, p->h_tasks, 2ull * njobs * sizeof(RmiTask), cudaMemcpyHostToDevice, p->st));
  CK(cudaMemcpyAsync(p->d_samp_off, p->h_samp_off, njobs * sizeof(u64), cudaMemcpyHostToDevice, p->st));
  CK(cudaMemcpyAsync(p->d_samp_n, p->h_samp_n, njobs * sizeof(u32), cudaMemcpyHostToDevice, p->st));
  CK(cudaStreamSynchronize(p->st));
  if (sl) return setup_jobs(p->sub, sj.data(), njobs);
  return MPSM_OK;
}

// Adam steps of the first nm models: every step in one cooperative launch when all
// its blocks fit on the device together and no graph is being captured, else a
// gradient and an update launch per step.  losses (device, optional): the loss
// before each step of model 0.
int train_models(mpsm_plan* p, u32 nm, u32 steps, float lr, float* losses) {
  if (!steps) return MPSM_OK;
  if (!p->graph_mode && p->d_trainbar && (u64)RMI_GMAX * nm <= p->train_cap) {
    LAUNCH(K_RMI_TRAIN, CK(launch_rmi_train(p->d_models, nm, p->d_tx, p->d_ty, p->d_partial, p->d_trainbar, steps, lr,
                                            losses, &p->d_cnt[C_ERR], p->st)));
    return MPSM_OK;
  }
  for (u32 t = 1; t <= steps; ++t) {
    LAUNCH(K_RMI_GRAD, launch_rmi_grad(p->d_models, nm, p->d_tx, p->d_ty, p->d_partial, p->st));
    LAUNCH(K_RMI_ADAM, launch_rmi_adam(p->d_models, nm, p->d_partial, t, lr, p->st));
    if (losses)
      CK(cudaMemcpyAsync(losses + (t - 1), &p->d_models[0].loss, sizeof(float), cudaMemcpyDeviceToDevice, p->st));
  }
  CK(cudaGetLastError());
  return MPSM_OK;
}

// ---------------------------------------------------------------- per-call setup
int setup_jobs(mpsm_plan* p, const Jobh* jobs, u32 njobs) {
  if (njobs == 0 || njobs > p->max_jobs) return MPSM_ERR_INVALID_ARG;
  u64 totR = 0, totS = 0, totRuns = 0, win_need = 0, tiles_need = 0;
  std::vector<u32> T(njobs);
  for (u32 i = 0; i < njobs; ++i) {
    totR += jobs[i].nR;
    totS += jobs[i].nS;
    T[i] = runs_for(p, jobs[i].nR);
    totRuns += T[i];
    const u64 nt = (jobs[i].nS + p->tile - 1) / p->tile;
    tiles_need += nt;
    win_need += nt * T[i];
  }
  if (totR > p->max_nR || totS > p->max_nS) return MPSM_ERR_INVALID_ARG;
  if (totRuns > p->runs_cap) return MPSM_ERR_INVALID_ARG;
  p->maxT = 1;
  for (u32 i = 0; i < njobs; ++i) p->maxT = std::max(p->maxT, T[i]);
  if (p->fused && (u64)p->fin_cap * p->maxT * 2 > p->swin_cap) {
    dfree(p->d_swin);
    p->swin_cap = (u64)p->fin_cap * p->maxT * 2;
    if (dalloc(&p->d_swin, p->swin_cap)) {
      p->swin_cap = 0;
      return MPSM_ERR_OOM;
    }
  }
  // grow the window / tile arrays if this call needs more
  if (win_need * 2 > p->win_cap) {
    dfree(p->d_win);
    p->win_cap = std::max<u64>(win_need * 2, 1024);
    if (dalloc(&p->d_win, p->win_cap)) return MPSM_ERR_OOM;
  }
  if (tiles_need + njobs > p->tile_cap) {
    dfree(p->d_tile_cnt);
    dfree(p->d_tile_out);
    p->tile_cap = tiles_need + njobs + 1024;
    if (dalloc(&p->d_tile_cnt, p->tile_cap) || dalloc(&p->d_tile_out, p->tile_cap)) return MPSM_ERR_OOM;
  }
  // S chunk (worker) size: about 4 chunks per SM in total
  u64 ch = (totS + 4ull * p->nsm - 1) / (4ull * p->nsm);
  ch = std::max<u64>(ch, 65536);
  ch = (ch + 4095) / 4096 * 4096;
  p->ch_s = ch;
  // host tables
  u64 rb = 0, sb = 0;
  u32 rbase = 0;
  u32 nbig = 0, nfin = 0;
  std::vector<Seg> big, fin, split;
  for (u32 i = 0; i < njobs; ++i) {
    Job J{};
    J.R = jobs[i].R;
    J.S = jobs[i].S;
    J.nR = jobs[i].nR;
    J.nS = jobs[i].nS;
    J.r_base = rb;
    J.s_base = sb;
    J.runs = T[i];
    J.run_base = rbase;
    J.parts_req = p->opt.partitions_s ? std::min<u32>(p->opt.partitions_s, P_MAX) : auto_parts(jobs[i].nS);
    J.part_base = i * (P_MAX + 1);
    J.fine_bits = p->opt.fine_bits ? p->opt.fine_bits : 12u;
    J.fine_base = i * FINE_MAX;
    p->h_jobs[i] = J;
    for (u32 j = 0; j < T[i]; ++j) {
      const u64 a = chunk_start(J.nR, T[i], j), b = chunk_start(J.nR, T[i], j + 1);
      p->h_runs[rbase + j] = Run{rb + a, b - a};
      if (b - a > NMAX) big.push_back(Seg{rb + a, b - a, 0, ~0ull, i, W_RIN});
      else if (b > a) fin.push_back(Seg{rb + a, b - a, 0, ~0ull, i, W_RIN});
    }
    split.push_back(Seg{sb, J.nS, 0, 0, i, W_SIN});
    rb += J.nR;
    sb += J.nS;
    rbase += T[i];
  }
  nbig = (u32)big.size();
  nfin = (u32)fin.size();
  if (nbig > p->big_cap || nfin > p->fin_cap) return MPSM_ERR_INVALID_ARG;
  const u64 need = (u64)nbig + nfin + njobs;
  if (need > p->hseg_cap) {
    hfree(p->h_segs);
    p->hseg_cap = (u32)(need + 1024);
    if (halloc(&p->h_segs, p->hseg_cap)) return MPSM_ERR_OOM;
  }
  std::copy(big.begin(), big.end(), p->h_segs);
  std::copy(fin.begin(), fin.end(), p->h_segs + nbig);
  std::copy(split.begin(), split.end(), p->h_segs + nbig + nfin);
  p->njobs = njobs;
  for (int i = 0; i < C_NUM; ++i) p->h_cnt[i] = 0;
  p->h_cnt[C_BIG0] = nbig;
  p->h_cnt[C_FIN] = nfin;
  p->h_cnt[C_SPLIT] = njobs;
  CK(cudaMemcpyAsync(p->d_jobs, p->h_jobs, njobs * sizeof(Job), cudaMemcpyHostToDevice, p->st));
  CK(cudaMemcpyAsync(p->d_runs, p->h_runs, rbase * sizeof(Run), cudaMemcpyHostToDevice, p->st));
  if (nbig) CK(cudaMemcpyAsync(p->d_big[0], p->h_segs, nbig * sizeof(Seg), cudaMemcpyHostToDevice, p->st));
  if (nfin) CK(cudaMemcpyAsync(p->d_fin, p->h_segs + nbig, nfin * sizeof(Seg), cudaMemcpyHostToDevice, p->st));
  CK(cudaMemcpyAsync(p->d_split, p->h_segs + nbig + nfin, njobs * sizeof(Seg), cudaMemcpyHostToDevice, p->st));
  CK(cudaMemcpyAsync(p->d_cnt, p->h_cnt, C_NUM * sizeof(u32), cudaMemcpyHostToDevice, p->st));
  // the host copies above read pinned memory asynchronously; keep it stable until they ran
  CK(cudaStreamSynchronize(p->st));
  p->levels_r = p->levels_s = 0;
  p->launches = 0;
  p->device_errors = 0;
  p->kt_n = 0;
  p->learn = split_learned(p) || search_learned(p);
  CK(cudaMemsetAsync(p->d_lstat, 0, 8 * sizeof(u64), p->st));
  if (runs_learned(p)) {
    const int rc = setup_rlearn(p, jobs, njobs);
    if (rc) return rc;
  }
  if (p->learn) return setup_learn(p, jobs, njobs);
  return MPSM_OK;
}

// radix passes over the big-segment list until every segment is final
// keep_const: constant-key children stay where they are (the fused join reads them
// in place) and the buckets aim at the fused kernel's tile
// first_mode: the bucket function of the first pass -- MODE_RADIX or MODE_RLEARN (each
// job's learned run buckets); later passes are MODE_RADIX
int run_levels(mpsm_plan* p, u32 first_src, u32 final_where, u32* levels, bool keep_const = false,
               u32 first_mode = MODE_RADIX) {
  u32 cur = 0, src = first_src;
  u32 done = 0;
  for (u32 lvl = 0; lvl < MAX_LEVELS; ++lvl) {
    const u32 mode = lvl == 0 ? first_mode : (u32)MODE_RADIX;
    const LearnCtx lcm = lctx(p, false);
    if (!p->graph_mode) {
      CK(cudaMemcpyAsync(&p->h_cnt[C_BIG0 + cur], &p->d_cnt[C_BIG0 + cur], sizeof(u32), cudaMemcpyDeviceToHost, p->st));
      CK(cudaStreamSynchronize(p->st));
      if (p->h_cnt[C_BIG0 + cur] == 0) break;
    }
    const u32 dst = (src == W_Y) ? final_where : (u32)W_Y;
    CK(cudaMemsetAsync(&p->d_cnt[C_BIG0 + (cur ^ 1)], 0, sizeof(u32), p->st));
    u64* tot = p->d_tot + T_LEVEL;
    const u32 rb = p->opt.radix_bits ? p->opt.radix_bits : 11u;
    LAUNCH(K_PLAN, launch_level_plan(p->d_big[cur], &p->d_cnt[C_BIG0 + cur], p->big_cap, p->d_ls, tot, mode, CH_RADIX, rb,
                      p->d_jobs, p->hist_a_cap, p->bucket_cap, &p->d_cnt[C_ERR], p->st,
                      keep_const ? FILL_FUSED : 0, &lcm));
    LAUNCH(K_INIT, launch_init_buckets(p->d_bmin, p->d_bmax, nullptr, tot, p->st, p->nsm));
    const Kid kh = mode == MODE_RLEARN ? K_HIST_RLEARN : K_HIST_RADIX;
    const Kid ks = mode == MODE_RLEARN ? K_SCATTER_RLEARN : K_SCATTER_RADIX;
    LAUNCH(kh, launch_hist(mode, p->d_big[cur], &p->d_cnt[C_BIG0 + cur], p->d_ls, tot, CH_RADIX, bufs(p), p->d_jobs, src,
                p->d_hist_a, p->d_bmin, p->d_bmax, nullptr, lcm, p->st, p->nsm));
    LAUNCH(K_SCAN_RADIX, launch_scan(MODE_RADIX, p->d_big[cur], &p->d_cnt[C_BIG0 + cur], p->d_ls, p->d_hist_a, p->d_bmin, p->d_bmax,
                nullptr, p->d_big[cur ^ 1], &p->d_cnt[C_BIG0 + (cur ^ 1)], p->big_cap, p->d_fin, &p->d_cnt[C_FIN],
                p->fin_cap, dst, p->d_jobs, nullptr, &p->d_cnt[C_ERR], p->st, p->nsm, keep_const));
    LAUNCH(ks, launch_scatter(mode, p->d_big[cur], &p->d_cnt[C_BIG0 + cur], p->d_ls, tot, CH_RADIX, bufs(p), p->d_jobs,
                   src, dst, p->d_hist_a, nullptr, &p->d_cnt[C_ERR], lcm, p->st, p->nsm, lvl == 0));
    CK(cudaGetLastError());
    src = dst;
    cur ^= 1;
    ++done;
  }
  if (p->graph_mode) {
    LAUNCH(K_CHECK, launch_check_empty(&p->d_cnt[C_BIG0 + cur], &p->d_cnt[C_ERR], DERR_LEVELS, p->st));
  } else if (done == MAX_LEVELS) {
    CK(cudaMemcpyAsync(&p->h_cnt[C_BIG0 + cur], &p->d_cnt[C_BIG0 + cur], sizeof(u32), cudaMemcpyDeviceToHost, p->st));
    CK(cudaStreamSynchronize(p->st));
    if (p->h_cnt[C_BIG0 + cur]) return MPSM_ERR_DEVICE;
  }
  // the finished list must be list 0 for the next user
  if (cur != 0) {
    CK(cudaMemcpyAsync(&p->d_cnt[C_BIG0], &p->d_cnt[C_BIG0 + cur], sizeof(u32), cudaMemcpyDeviceToDevice, p->st));
  }
  *levels = done;
  return MPSM_OK;
}

int final_sort(mpsm_plan* p, u32 dst_where) {
  CK(cudaMemsetAsync(&p->d_cnt[C_WORK], 0, 2 * sizeof(u32), p->st));  // one work counter per size class
  LAUNCH(K_SEG_SORT, launch_seg_sort(p->d_fin, &p->d_cnt[C_FIN], p->fin_cap, &p->d_cnt[C_WORK], bufs(p), p->d_jobs, dst_where,
                  &p->d_cnt[C_ERR], p->st, p->nsm));
  CK(cudaGetLastError());
  return MPSM_OK;
}

// ---------------------------------------------------------------- phases
int phase_runs(mpsm_plan* p) {
  record(p, EV_START);
  CK(cudaMemsetAsync(&p->d_cnt[C_ERR], 0, sizeof(u32), p->st));
  const bool rl = runs_learned(p) && p->rsub;
  if (rl) {
    // the learned run bucket function: a run-side sample, sorted by the sub-plan, cut
    // into quantiles
    LAUNCH(K_SAMPLE_R, launch_sample_r(p->d_jobs, p->njobs, p->d_rsamp_off, p->d_rsamp_n, p->d_rsamp, p->st, p->nsm));
    p->rsub->graph_mode = p->graph_mode;
    p->rsub->opt.flags = p->opt.flags & MPSM_FLAG_KERNEL_TIMING;
    const int src = phase_runs(p->rsub);
    p->launches += p->rsub->launches;
    if (src) return src;
    LAUNCH(K_RLEARN_TAB, launch_rlearn_tables(p->d_jobs, p->njobs, p->rsub->xr, p->d_rsamp_off, p->d_rsamp_n, p->d_rl,
                                              p->d_rcell, p->d_rbnd, p->st));
  }
  LAUNCH(K_SAMPLE, launch_sample_bounds(p->d_big[0], &p->d_cnt[C_BIG0], p->h_cnt[C_BIG0] ? p->big_cap : 0, bufs(p), p->d_jobs, p->st));
  int rc = run_levels(p, W_RIN, W_XR, &p->levels_r, false, rl ? (u32)MODE_RLEARN : (u32)MODE_RADIX);
  if (rc) return rc;
  rc = final_sort(p, W_XR);
  if (rc) return rc;
  LAUNCH(K_RUN_BOUNDS, launch_run_bounds(p->d_jobs, p->njobs, p->d_runs, p->xr, p->st));
  CK(cudaGetLastError());
  record(p, EV_RUNS);
  p->stage = ST_RUNS;
  return MPSM_OK;
}

// Learned model of each job: S sample sorted by the sub-plan (the same sort
// kernels as phase 1), fit data, training, tabulation and leaves.
// the partitioned side's host copy must land before its first reader (the learned
// sample, else the fine histogram)
int wait_part_copy(mpsm_plan* p) {
  if (p->part_copy_pending) {
    CK(cudaStreamWaitEvent(p->st, p->ev_part_copied, 0));
    p->part_copy_pending = false;
  }
  return MPSM_OK;
}

int phase_learn(mpsm_plan* p) {
  if (int rc = wait_part_copy(p)) return rc;
  if (!p->learn) {
    record(p, EV_LEARN);
    return MPSM_OK;
  }
  const u32 nm = 2 * p->njobs;
  if (split_learned(p)) {
    LAUNCH(K_SAMPLE_S, launch_sample_s(p->d_jobs, p->njobs, p->d_samp_off, p->d_samp_n, p->d_samp, p->st, p->nsm));
    p->sub->graph_mode = p->graph_mode;
    p->sub->opt.flags = p->opt.flags & MPSM_FLAG_KERNEL_TIMING;
    const int rc = phase_runs(p->sub);
    p->launches += p->sub->launches;
    if (rc) return rc;
  }
  LAUNCH(K_RMI_DATA, launch_rmi_setup(p->d_models, p->d_tasks, nm, p->d_jobs, true, p->st));
  LAUNCH(K_RMI_DATA, launch_fit_data(p->d_models, p->d_tasks, nm, p->d_jobs, p->d_runs, p->xr,
                                     p->sub ? p->sub->xr : nullptr, p->d_fitk, p->d_fity, p->st, p->nsm));
  // The learned splitters take the sorted sample's quantiles (k_learn_bounds) and its
  // cell table, not the network's predictions; only the learned search predicts with the
  // trained models, so only it trains them.
  if (search_learned(p)) {
    LAUNCH(K_RMI_DATA, launch_train_data(p->d_models, nm, p->d_fitk, p->d_fity, p->d_tx, p->d_ty, p->st));
    const u32 steps = p->opt.learn_steps ? p->opt.learn_steps : RMI_STEPS;
    if (int rc = train_models(p, nm, steps, RMI_LR, nullptr)) return rc;
    LAUNCH(K_RMI_TAB, launch_rmi_tabulate(p->d_models, nm, p->st));
    LAUNCH(K_RMI_LEAF, launch_leaf_fit(p->d_models, nm, p->d_leafacc, p->d_fitk, p->d_fity, p->st, p->nsm));
  }
  CK(cudaGetLastError());
  record(p, EV_LEARN);
  return MPSM_OK;
}

// Learned splitters: partition boundaries at the quantiles of the sorted S
// sample, then one counting pass in which the model predicts each S tuple's
// partition and an exact search over the boundaries corrects it.
int phase_splitters_learned(mpsm_plan* p) {
  u64* ts = p->d_tot + T_SPLIT;
  LAUNCH(K_LEARN_BOUNDS, launch_learn_bounds(p->d_jobs, p->njobs, p->d_models, p->d_fitk, p->d_bnd, p->d_brank, p->st));
  LAUNCH(K_LEARN_BOUNDS, launch_learn_cells(p->d_jobs, p->njobs, p->d_bnd, p->d_sp, p->st));
  LAUNCH(K_PLAN, launch_level_plan(p->d_split, &p->d_cnt[C_SPLIT], p->max_jobs, p->d_ls2, ts, MODE_LEARN, p->ch_s, 11,
                                   p->d_jobs, p->hist_a_cap, p->bucket_cap, &p->d_cnt[C_ERR], p->st));
  LAUNCH(K_INIT, launch_init_buckets(p->d_bmin, p->d_bmax, nullptr, ts, p->st, p->nsm));
  LAUNCH(K_HIST_LEARN, launch_hist(MODE_LEARN, p->d_split, &p->d_cnt[C_SPLIT], p->d_ls2, ts, p->ch_s, bufs(p), p->d_jobs,
                                   W_SIN, p->d_hist_a, p->d_bmin, p->d_bmax, nullptr, lctx(p, true), p->st, p->nsm));
  CK(cudaMemsetAsync(&p->d_cnt[C_BIG0], 0, sizeof(u32), p->st));
  CK(cudaMemsetAsync(&p->d_cnt[C_FIN], 0, sizeof(u32), p->st));
  LAUNCH(K_SCAN_LEARN, launch_scan(MODE_LEARN, p->d_split, &p->d_cnt[C_SPLIT], p->d_ls2, p->d_hist_a, p->d_bmin,
                                   p->d_bmax, nullptr, p->d_big[0], &p->d_cnt[C_BIG0], p->big_cap, p->d_fin,
                                   &p->d_cnt[C_FIN], p->fin_cap, W_XS, p->d_jobs, p->d_part_off, &p->d_cnt[C_ERR],
                                   p->st, p->nsm, p->fused, p->d_bnd));
  CK(cudaGetLastError());
  record(p, EV_SPLIT);
  p->stage = ST_SPLIT;
  return MPSM_OK;
}

int phase_splitters(mpsm_plan* p) {
  if (int rc = wait_part_copy(p)) return rc;
  if (split_learned(p)) return phase_splitters_learned(p);
  const u32 nj = p->njobs;
  if (!p->runs_reused) CK(cudaMemsetAsync(p->d_rc, 0, (u64)nj * (FINE_MAX + 1) * sizeof(u64), p->st));
  CK(cudaMemsetAsync(p->d_fine_s, 0, (u64)nj * FINE_MAX * sizeof(u64), p->st));
  CK(cudaMemsetAsync(p->d_fine_min, 0xFF, (u64)nj * FINE_MAX * sizeof(u64), p->st));
  CK(cudaMemsetAsync(p->d_fine_max, 0, (u64)nj * FINE_MAX * sizeof(u64), p->st));
  u64* tf = p->d_tot + T_FINE;
  u64* ts = p->d_tot + T_SPLIT;
  LAUNCH(K_PLAN, launch_level_plan(p->d_split, &p->d_cnt[C_SPLIT], p->max_jobs, p->d_ls, tf, MODE_FINE, p->ch_s, 11, p->d_jobs,
                    p->hist_b_cap, ~0ull, &p->d_cnt[C_ERR], p->st));
  LAUNCH(K_HIST_FINE, launch_hist(MODE_FINE, p->d_split, &p->d_cnt[C_SPLIT], p->d_ls, tf, p->ch_s, bufs(p), p->d_jobs, W_SIN,
              p->d_hist_b, p->d_fine_min, p->d_fine_max, p->d_fine_s, lctx(p, false), p->st, p->nsm));
  if (!p->runs_reused) LAUNCH(K_RUN_CDF, launch_run_cdf(p->d_jobs, nj, p->d_runs, p->xr, p->d_rc, p->st));
  LAUNCH(K_SPLITTERS, launch_splitters(p->d_jobs, nj, p->d_fine_s, p->d_rc, p->d_fine_r, p->d_sp, p->d_fstart, &p->d_cnt[C_ERR], p->st,
                                       p->opt.splitter_mode == MPSM_SPLIT_EQUI_HEIGHT));
  LAUNCH(K_PLAN, launch_level_plan(p->d_split, &p->d_cnt[C_SPLIT], p->max_jobs, p->d_ls2, ts, MODE_SPLIT, p->ch_s, 11, p->d_jobs,
                    p->hist_a_cap, ~0ull, &p->d_cnt[C_ERR], p->st));
  LAUNCH(K_FOLD, launch_fold(p->d_split, &p->d_cnt[C_SPLIT], p->d_ls, p->d_ls2, tf, p->d_jobs, p->d_hist_b, p->d_fstart,
              p->d_hist_a, p->st, p->nsm));
  CK(cudaMemsetAsync(&p->d_cnt[C_BIG0], 0, sizeof(u32), p->st));
  CK(cudaMemsetAsync(&p->d_cnt[C_FIN], 0, sizeof(u32), p->st));
  LAUNCH(K_SCAN_SPLIT, launch_scan(MODE_SPLIT, p->d_split, &p->d_cnt[C_SPLIT], p->d_ls2, p->d_hist_a, p->d_fine_min, p->d_fine_max,
              p->d_fstart, p->d_big[0], &p->d_cnt[C_BIG0], p->big_cap, p->d_fin, &p->d_cnt[C_FIN], p->fin_cap, W_XS,
              p->d_jobs, p->d_part_off, &p->d_cnt[C_ERR], p->st, p->nsm, p->fused));
  CK(cudaGetLastError());
  record(p, EV_SPLIT);
  p->stage = ST_SPLIT;
  return MPSM_OK;
}

int phase_scatter(mpsm_plan* p) {
  const bool sl = split_learned(p);
  // learned partitioning with at most 512 partitions per job takes the larger tiles
  bool small_p = true;
  for (u32 i = 0; i < p->njobs; ++i) small_p = small_p && p->h_jobs[i].parts_req <= 512u;
  LAUNCH(sl ? K_SCATTER_LEARN : K_SCATTER_SPLIT,
         launch_scatter(sl ? MODE_LEARN : MODE_SPLIT, p->d_split, &p->d_cnt[C_SPLIT], p->d_ls2, p->d_tot + T_SPLIT,
                        p->ch_s, bufs(p), p->d_jobs, W_SIN, W_XS, p->d_hist_a, p->d_sp, &p->d_cnt[C_ERR],
                        lctx(p, sl), p->st, p->nsm, sl && small_p));
  CK(cudaGetLastError());
  record(p, EV_SCATTER);
  p->stage = ST_SCATTER;
  return MPSM_OK;
}

// MPSM_FLAG_BOUNDS_TEST: one final S segment's recorded bounds made inexact
int narrow_bounds_test(mpsm_plan* p) {
  if (p->opt.flags & MPSM_FLAG_BOUNDS_TEST) launch_narrow_bounds_test(p->d_fin, &p->d_cnt[C_FIN], p->fin_cap, p->st);
  CK(cudaGetLastError());
  return MPSM_OK;
}

int phase_sort_parts(mpsm_plan* p) {
  int rc = run_levels(p, W_XS, W_XS, &p->levels_s);
  if (rc) return rc;
  if ((rc = narrow_bounds_test(p))) return rc;
  rc = final_sort(p, W_XS);
  if (rc) return rc;
  record(p, EV_SORTS);
  p->stage = ST_SORTED;
  return MPSM_OK;
}

int read_err(mpsm_plan* p);

// Phases 3 and 4 fused: radix passes over the S partitions as in phase 3, then
// per final segment the windows of every R run (fence search), then one kernel
// that sorts each segment in shared memory and joins it there.  Sorted S is
// never written back or read again.
int phase_sort_join(mpsm_plan* p) {
  int rc = run_levels(p, W_XS, W_XS, &p->levels_s, true);
  if (rc) return rc;
  if ((rc = narrow_bounds_test(p))) return rc;
  record(p, EV_SORTS);
  u64 totR = 0;
  for (u32 i = 0; i < p->njobs; ++i) totR += p->h_jobs[i].nR;
  if (!p->runs_reused) LAUNCH(K_FENCES, launch_fences(p->xr, totR, p->d_fence, p->st, p->nsm));
  LAUNCH(K_SEG_SEARCH, launch_seg_search(p->d_fin, &p->d_cnt[C_FIN], p->fin_cap, p->d_jobs, p->d_runs, p->xr, p->d_fence,
                                         p->d_swin, p->maxT, lctx(p, search_learned(p)), p->st, p->nsm));
  record(p, EV_SEARCH);
  FuseCtx fc{p->d_swin, p->maxT, p->d_runs, p->xr, p->d_jobs};
  CK(cudaMemsetAsync(&p->d_cnt[C_WORK], 0, 2 * sizeof(u32), p->st));
  LAUNCH(K_SORT_JOIN, launch_seg_sort_join(p->d_fin, &p->d_cnt[C_FIN], p->fin_cap, &p->d_cnt[C_WORK], bufs(p), p->d_jobs,
                                           &p->d_cnt[C_ERR], fc, p->st, p->nsm));
  CK(cudaGetLastError());
  record(p, EV_JOIN);
  p->stage = ST_DONE;
  return MPSM_OK;
}

// results of a fused call (job 0 to the caller)
int fused_results(mpsm_plan* p, uint64_t* out_count, uint64_t* out_checksum) {
  CK(cudaMemcpyAsync(p->h_jobs, p->d_jobs, p->njobs * sizeof(Job), cudaMemcpyDeviceToHost, p->st));
  const int rc = read_err(p);
  if (rc) return rc;
  if (out_count) *out_count = p->h_jobs[0].count;
  if (out_checksum) *out_checksum = p->h_jobs[0].checksum;
  return MPSM_OK;
}

int phase_search(mpsm_plan* p) {
  LAUNCH(K_TILES, launch_tiles(p->d_jobs, p->njobs, p->tile, p->d_tot + T_TILES, &p->d_cnt[C_ERR], p->st));
  LAUNCH(K_SEARCH, launch_search(p->d_jobs, p->njobs, p->d_runs, p->xr, p->xs, p->tile, p->d_tot + T_TILES, p->d_win,
                                 lctx(p, search_learned(p)), p->st, p->nsm));
  CK(cudaGetLastError());
  record(p, EV_SEARCH);
  p->stage = ST_SEARCH;
  return MPSM_OK;
}

int read_err(mpsm_plan* p) {
  CK(cudaMemcpyAsync(&p->h_cnt[C_ERR], &p->d_cnt[C_ERR], sizeof(u32), cudaMemcpyDeviceToHost, p->st));
  const bool sub = p->learn && split_learned(p) && p->sub;
  const bool rsub = runs_learned(p) && p->rsub;
  if (sub)
    CK(cudaMemcpyAsync(&p->sub->h_cnt[C_ERR], &p->sub->d_cnt[C_ERR], sizeof(u32), cudaMemcpyDeviceToHost, p->st));
  if (rsub)
    CK(cudaMemcpyAsync(&p->rsub->h_cnt[C_ERR], &p->rsub->d_cnt[C_ERR], sizeof(u32), cudaMemcpyDeviceToHost, p->st));
  CK(cudaStreamSynchronize(p->st));
  p->device_errors = p->h_cnt[C_ERR] | (sub ? p->sub->h_cnt[C_ERR] : 0u) | (rsub ? p->rsub->h_cnt[C_ERR] : 0u);
  return p->device_errors ? MPSM_ERR_DEVICE : MPSM_OK;
}

int phase_join(mpsm_plan* p, uint64_t* out_count, uint64_t* out_checksum, mpsm_pairs_t* pairs) {
  const u64* tot = p->d_tot + T_TILES;
  if (pairs) {
    LAUNCH(K_JOIN, launch_join(JOIN_COUNT, p->d_jobs, p->njobs, p->d_runs, p->xr, p->xs, p->tile, tot, p->d_win, p->d_tile_cnt,
                nullptr, nullptr, &p->d_cnt[C_ERR], p->st, p->nsm));
    LAUNCH(K_PAIR_OFFSETS, launch_pair_offsets(p->d_jobs, p->njobs, tot, p->d_tile_cnt, p->d_tile_out, p->d_tot + T_PAIRS, p->st));
    CK(cudaMemcpyAsync(p->h_scalar, p->d_tot + T_PAIRS, sizeof(u64), cudaMemcpyDeviceToHost, p->st));
    CK(cudaStreamSynchronize(p->st));
    const u64 need = p->h_scalar[0];
    if (need <= pairs->capacity && need > 0) {
      if (!pairs->data) return MPSM_ERR_INVALID_ARG;
      LAUNCH(K_JOIN, launch_join(JOIN_WRITE, p->d_jobs, p->njobs, p->d_runs, p->xr, p->xs, p->tile, tot, p->d_win, p->d_tile_cnt,
                  p->d_tile_out, reinterpret_cast<Tuple*>(pairs->data), &p->d_cnt[C_ERR], p->st, p->nsm));
    }
  } else {
    LAUNCH(K_JOIN, launch_join(JOIN_AGG, p->d_jobs, p->njobs, p->d_runs, p->xr, p->xs, p->tile, tot, p->d_win, nullptr, nullptr,
                nullptr, &p->d_cnt[C_ERR], p->st, p->nsm));
  }
  CK(cudaGetLastError());
  record(p, EV_JOIN);
  CK(cudaMemcpyAsync(p->h_jobs, p->d_jobs, p->njobs * sizeof(Job), cudaMemcpyDeviceToHost, p->st));
  int rc = read_err(p);
  p->stage = ST_DONE;
  if (rc) return rc;
  if (out_count) *out_count = p->h_jobs[0].count;
  if (out_checksum) *out_checksum = p->h_jobs[0].checksum;
  if (pairs && p->h_jobs[0].count > pairs->capacity) return MPSM_ERR_CAPACITY;
  return MPSM_OK;
}

bool aligned16(const void* q) { return ((uintptr_t)q & 15u) == 0; }

int check_inputs(const mpsm_plan* p, const mpsm_tuple_t* R, u64 nR, const mpsm_tuple_t* S, u64 nS) {
  if (!p) return MPSM_ERR_INVALID_ARG;
  if ((nR && !R) || (nS && !S)) return MPSM_ERR_INVALID_ARG;
  if (!aligned16(R) || !aligned16(S)) return MPSM_ERR_INVALID_ARG;
  if (nR > p->max_nR || nS > p->max_nS) return MPSM_ERR_INVALID_ARG;
  return MPSM_OK;
}

}  // namespace

// ============================================================== C ABI

MPSM_API int mpsm_options_default(mpsm_options_t* opt) {
  if (!opt) return MPSM_ERR_INVALID_ARG;
  memset(opt, 0, sizeof(*opt));
  opt->splitter_mode = MPSM_SPLIT_HIST;
  opt->search_mode = MPSM_SEARCH_BINARY;
  opt->seed = 20120145ull;
  return MPSM_OK;
}

MPSM_API void mpsm_plan_destroy(mpsm_plan_t* p) {
  if (!p) return;
  if (p->st) cudaStreamSynchronize(p->st);
  dfree(p->xr);
  dfree(p->xs);
  dfree(p->y);
  dfree(p->stage_r);
  dfree(p->stage_s);
  dfree(p->d_jobs);
  hfree(p->h_jobs);
  dfree(p->d_runs);
  hfree(p->h_runs);
  dfree(p->d_split);
  hfree(p->h_segs);
  dfree(p->d_big[0]);
  dfree(p->d_big[1]);
  dfree(p->d_fin);
  dfree(p->d_cnt);
  hfree(p->h_cnt);
  dfree(p->d_ls);
  dfree(p->d_ls2);
  dfree(p->d_tot);
  dfree(p->d_hist_a);
  dfree(p->d_hist_b);
  dfree(p->d_bmin);
  dfree(p->d_bmax);
  dfree(p->d_fine_s);
  dfree(p->d_fine_min);
  dfree(p->d_fine_max);
  dfree(p->d_fine_r);
  dfree(p->d_rc);
  dfree(p->d_sp);
  dfree(p->d_fstart);
  dfree(p->d_part_off);
  dfree(p->d_win);
  dfree(p->d_tile_cnt);
  dfree(p->d_tile_out);
  dfree(p->d_chunk_off);
  hfree(p->h_scalar);
  dfree(p->d_lstat);
  dfree(p->d_fence);
  dfree(p->d_swin);
  dfree(p->d_models);
  dfree(p->d_tasks);
  hfree(p->h_tasks);
  if (p->d_leafacc) cudaFree(p->d_leafacc);
  dfree(p->d_tx);
  dfree(p->d_ty);
  dfree(p->d_partial);
  dfree(p->d_trainbar);
  dfree(p->d_fitk);
  dfree(p->d_fity);
  dfree(p->d_samp);
  dfree(p->d_samp_off);
  hfree(p->h_samp_off);
  dfree(p->d_samp_n);
  hfree(p->h_samp_n);
  dfree(p->d_bnd);
  dfree(p->d_brank);
  if (p->sub) mpsm_plan_destroy(p->sub);
  dfree(p->d_rl);
  dfree(p->d_rcell);
  dfree(p->d_rbnd);
  dfree(p->d_rsamp);
  dfree(p->d_rsamp_off);
  hfree(p->h_rsamp_off);
  dfree(p->d_rsamp_n);
  hfree(p->h_rsamp_n);
  if (p->rsub) mpsm_plan_destroy(p->rsub);
  for (auto& e : p->ev)
    if (e) cudaEventDestroy(e);
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->kt_ev) {
    for (u32 i = 0; i < 2 * KT_POOL; ++i) cudaEventDestroy(p->kt_ev[i]);
    delete[] p->kt_ev;
  }
  if (p->st_copy) {
    cudaStreamSynchronize(p->st_copy);
    cudaStreamDestroy(p->st_copy);
  }
  if (p->ev_run_copied) cudaEventDestroy(p->ev_run_copied);
  if (p->ev_part_copied) cudaEventDestroy(p->ev_part_copied);
  for (u32 i = 0; i < mpsm_plan::MAX_PIECES; ++i)
    if (p->ev_piece[i]) cudaEventDestroy(p->ev_piece[i]);
  if (p->own_stream && p->st) cudaStreamDestroy(p->st);
  delete p;
}

MPSM_API int mpsm_plan_create(mpsm_plan_t** out, uint64_t max_nR, uint64_t max_nS, uint32_t max_jobs,
                              const mpsm_options_t* opt, void* stream) {
  if (!out) return MPSM_ERR_INVALID_ARG;
  *out = nullptr;
  if (max_nR >= (1ull << 32) || max_nS >= (1ull << 32)) return MPSM_ERR_INVALID_ARG;
  if (max_jobs == 0) max_jobs = 1;
  mpsm_options_t o;
  if (opt) {
    o = *opt;
    for (int i = 0; i < 2; ++i)
      if (o.reserved[i]) return MPSM_ERR_INVALID_ARG;
    if (o.partition_side > MPSM_PART_SMALLER) return MPSM_ERR_INVALID_ARG;
    if (o.run_buckets > MPSM_RUNS_LEARNED) return MPSM_ERR_INVALID_ARG;
  } else {
    mpsm_options_default(&o);
  }
  if (o.fine_bits > 12 || (o.radix_bits && (o.radix_bits < 4 || o.radix_bits > 11))) return MPSM_ERR_INVALID_ARG;
  if (o.partitions_s > P_MAX || o.runs_r > RUNS_MAX || o.learn_steps > 100000) return MPSM_ERR_INVALID_ARG;
  if (o.join_tile && (o.join_tile < 256 || o.join_tile > TILE_MAX || o.join_tile % 256)) return MPSM_ERR_INVALID_ARG;
  if (o.splitter_mode != MPSM_SPLIT_HIST && o.splitter_mode != MPSM_SPLIT_LEARNED &&
      o.splitter_mode != MPSM_SPLIT_EQUI_HEIGHT)
    return MPSM_ERR_INVALID_ARG;
  if (o.search_mode != MPSM_SEARCH_BINARY && o.search_mode != MPSM_SEARCH_LEARNED &&
      o.search_mode != MPSM_SEARCH_INTERP)
    return MPSM_ERR_INVALID_ARG;
  mpsm_plan* p = new (std::nothrow) mpsm_plan();
  if (!p) return MPSM_ERR_OOM;
  p->opt = o;
  p->st = (cudaStream_t)stream;
  if (o.partition_side != MPSM_PART_S) max_nR = max_nS = std::max(max_nR, max_nS);  // either input may take either role
  p->max_nR = max_nR;
  p->max_nS = max_nS;
  p->max_jobs = max_jobs;
  p->tile = o.join_tile ? o.join_tile : TILE_MAX;
  p->timing = (o.flags & MPSM_FLAG_TIMING) != 0;
  int rc = MPSM_OK;
#define TRY(x)                 \
  do {                         \
    rc = (x);                  \
    if (rc) {                  \
      mpsm_plan_destroy(p);    \
      return rc;               \
    }                          \
  } while (0)
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return MPSM_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, p->device);
  if (p->nsm <= 0) p->nsm = 1;
  if (!p->st) {  // a stream of our own, synchronising with the legacy default stream like the caller's work
    if (cudaStreamCreate(&p->st) != cudaSuccess) {
      cudaGetLastError();
      delete p;
      return MPSM_ERR_CUDA;
    }
    p->own_stream = true;
  }
  init_attrs_pass();
  init_attrs_split();
  init_attrs_join();
  init_attrs_learn();
  const u64 nside = std::max(max_nR, max_nS);
  TRY(dalloc(&p->xr, max_nR));
  TRY(dalloc(&p->xs, max_nS));
  TRY(dalloc(&p->y, nside));
  p->runs_cap = max_jobs * RUNS_MAX;
  TRY(dalloc(&p->d_jobs, max_jobs));
  TRY(halloc(&p->h_jobs, max_jobs));
  TRY(dalloc(&p->d_runs, p->runs_cap));
  TRY(halloc(&p->h_runs, p->runs_cap));
  TRY(dalloc(&p->d_split, max_jobs));
  p->big_cap = (u32)(nside / NMAX + p->runs_cap + 1024);
  p->fin_cap = (u32)(nside / 256 + 65536 + p->runs_cap);
  TRY(dalloc(&p->d_big[0], p->big_cap));
  TRY(dalloc(&p->d_big[1], p->big_cap));
  TRY(dalloc(&p->d_fin, p->fin_cap));
  TRY(dalloc(&p->d_cnt, C_NUM));
  TRY(halloc(&p->h_cnt, C_NUM));
  TRY(dalloc(&p->d_ls, std::max<u64>(p->big_cap, max_jobs)));
  TRY(dalloc(&p->d_ls2, max_jobs));
  TRY(dalloc(&p->d_tot, T_NUM));
  const u64 s_chunks = 4ull * p->nsm + 2ull * max_jobs + 16;
  // radix passes: chunks x F <= n / 32 at the regular fan-out, plus n / 64 for the one-bucket-per-key passes
  p->hist_a_cap = std::max<u64>(nside / 32 + nside / 64 + (1u << 20), s_chunks * P_MAX);
  p->hist_b_cap = s_chunks * FINE_MAX;
  TRY(dalloc(&p->d_hist_a, p->hist_a_cap));
  TRY(dalloc(&p->d_hist_b, p->hist_b_cap));
  p->bucket_cap = nside / 64 + 65536 + (u64)max_jobs * 64;
  TRY(dalloc(&p->d_bmin, p->bucket_cap));
  TRY(dalloc(&p->d_bmax, p->bucket_cap));
  const u64 nf = (u64)max_jobs * FINE_MAX;
  TRY(dalloc(&p->d_fine_s, nf));
  TRY(dalloc(&p->d_fine_min, nf));
  TRY(dalloc(&p->d_fine_max, nf));
  TRY(dalloc(&p->d_fine_r, nf));
  TRY(dalloc(&p->d_rc, (u64)max_jobs * (FINE_MAX + 1)));
  TRY(dalloc(&p->d_sp, nf));
  TRY(dalloc(&p->d_fstart, (u64)max_jobs * (P_MAX + 1)));
  TRY(dalloc(&p->d_part_off, (u64)max_jobs * (P_MAX + 1)));
  TRY(halloc(&p->h_scalar, 16));
  TRY(dalloc(&p->d_lstat, 8));
  TRY(dalloc(&p->d_fence, max_nR / 64 + 2));
  if (o.splitter_mode == MPSM_SPLIT_LEARNED || o.search_mode == MPSM_SEARCH_LEARNED) TRY(alloc_learn(p));
  if (o.run_buckets == MPSM_RUNS_LEARNED) TRY(alloc_rlearn(p));
  {
    const u32 fl = o.flags;
    p->opt.flags = 0;
    TRY(mpsm_plan_set_flags(p, fl));
  }
#undef TRY
  *out = p;
  return MPSM_OK;
}

MPSM_API int mpsm_sort_runs(mpsm_plan_t* p, const mpsm_tuple_t* R, uint64_t nR) {
  int rc = check_inputs(p, R, nR, nullptr, 0);
  if (rc) return rc;
  if (split_learned(p) || search_learned(p)) return MPSM_ERR_INVALID_ARG;
  p->fused = false;
  Jobh j{reinterpret_cast<const Tuple*>(R), nullptr, nR, 0};
  rc = setup_jobs(p, &j, 1);
  if (rc) return rc;
  return phase_runs(p);
}

MPSM_API int mpsm_splitters(mpsm_plan_t* p, const mpsm_tuple_t* S, uint64_t nS) {
  if (!p) return MPSM_ERR_INVALID_ARG;
  if (p->stage < ST_RUNS || p->njobs != 1) return MPSM_ERR_STATE;
  int rc = check_inputs(p, nullptr, 0, S, nS);
  if (rc) return rc;
  // attach S to the single job and re-upload the S tables (R's state on the device is kept)
  const u64 tiles_need = (nS + p->tile - 1) / p->tile;
  const u64 win_need = tiles_need * p->h_jobs[0].runs;
  if (win_need * 2 > p->win_cap) {
    dfree(p->d_win);
    p->win_cap = std::max<u64>(win_need * 2, 1024);
    if (dalloc(&p->d_win, p->win_cap)) return MPSM_ERR_OOM;
  }
  if (tiles_need + 1 > p->tile_cap) {
    dfree(p->d_tile_cnt);
    dfree(p->d_tile_out);
    p->tile_cap = tiles_need + 1024;
    if (dalloc(&p->d_tile_cnt, p->tile_cap) || dalloc(&p->d_tile_out, p->tile_cap)) return MPSM_ERR_OOM;
  }
  u64 ch = (nS + 4ull * p->nsm - 1) / (4ull * p->nsm);
  ch = std::max<u64>(ch, 65536);
  p->ch_s = (ch + 4095) / 4096 * 4096;
  // device job: set S fields only (R fields were updated on the device by phase 1)
  CK(cudaMemcpyAsync(p->h_jobs, p->d_jobs, sizeof(Job), cudaMemcpyDeviceToHost, p->st));
  CK(cudaStreamSynchronize(p->st));
  p->h_jobs[0].S = reinterpret_cast<const Tuple*>(S);
  p->h_jobs[0].nS = nS;
  p->h_jobs[0].s_base = 0;
  p->h_jobs[0].parts_req = p->opt.partitions_s ? p->opt.partitions_s : auto_parts(nS);
  Seg sg{0, nS, 0, 0, 0, W_SIN};
  p->h_segs[0] = sg;
  p->h_cnt[C_SPLIT] = 1;
  CK(cudaMemcpyAsync(p->d_jobs, p->h_jobs, sizeof(Job), cudaMemcpyHostToDevice, p->st));
  CK(cudaMemcpyAsync(p->d_split, p->h_segs, sizeof(Seg), cudaMemcpyHostToDevice, p->st));
  CK(cudaMemcpyAsync(&p->d_cnt[C_SPLIT], &p->h_cnt[C_SPLIT], sizeof(u32), cudaMemcpyHostToDevice, p->st));
  CK(cudaStreamSynchronize(p->st));
  return phase_splitters(p);
}

MPSM_API int mpsm_scatter(mpsm_plan_t* p) {
  if (!p) return MPSM_ERR_INVALID_ARG;
  if (p->stage < ST_SPLIT) return MPSM_ERR_STATE;
  return phase_scatter(p);
}

MPSM_API int mpsm_sort_partitions(mpsm_plan_t* p) {
  if (!p) return MPSM_ERR_INVALID_ARG;
  if (p->stage < ST_SCATTER) return MPSM_ERR_STATE;
  return phase_sort_parts(p);
}

MPSM_API int mpsm_search(mpsm_plan_t* p) {
  if (!p) return MPSM_ERR_INVALID_ARG;
  if (p->stage < ST_SORTED) return MPSM_ERR_STATE;
  return phase_search(p);
}

MPSM_API int mpsm_merge_join(mpsm_plan_t* p, uint64_t* out_count, uint64_t* out_checksum, mpsm_pairs_t* pairs) {
  if (!p) return MPSM_ERR_INVALID_ARG;
  if (p->stage < ST_SEARCH) return MPSM_ERR_STATE;
  if (pairs && pairs->capacity && (!pairs->data || !aligned16(pairs->data))) return MPSM_ERR_INVALID_ARG;
  return phase_join(p, out_count, out_checksum, pairs);
}

static int join_device(mpsm_plan_t* p, const mpsm_tuple_t* R, uint64_t nR, const mpsm_tuple_t* S, uint64_t nS,
                       uint64_t* out_count, uint64_t* out_checksum, mpsm_pairs_t* pairs) {
  Jobh j{reinterpret_cast<const Tuple*>(R), reinterpret_cast<const Tuple*>(S), nR, nS};
  p->fused = !pairs && !(p->opt.flags & MPSM_FLAG_UNFUSED);
  int rc = setup_jobs(p, &j, 1);
  if (rc) return rc;
  if ((rc = phase_runs(p))) return rc;
  if ((rc = phase_learn(p))) return rc;
  if ((rc = phase_splitters(p))) return rc;
  if ((rc = phase_scatter(p))) return rc;
  if (p->fused) {
    if ((rc = phase_sort_join(p))) return rc;
    return fused_results(p, out_count, out_checksum);
  }
  if ((rc = phase_sort_parts(p))) return rc;
  if ((rc = phase_search(p))) return rc;
  return phase_join(p, out_count, out_checksum, pairs);
}

// Role reversal (Sec. 5.4): partition R and cut S into runs by joining S with R;
// count and checksum are symmetric, and the pairs get their columns swapped back.
static bool reverse_roles(const mpsm_plan* p, u64 nR, u64 nS) {
  return p->opt.partition_side == MPSM_PART_R || (p->opt.partition_side == MPSM_PART_SMALLER && nR < nS);
}

MPSM_API int mpsm_join(mpsm_plan_t* p, const mpsm_tuple_t* R, uint64_t nR, const mpsm_tuple_t* S, uint64_t nS,
                       uint64_t* out_count, uint64_t* out_checksum, mpsm_pairs_t* pairs) {
  int rc = check_inputs(p, R, nR, S, nS);
  if (rc) return rc;
  if (pairs && pairs->capacity && (!pairs->data || !aligned16(pairs->data))) return MPSM_ERR_INVALID_ARG;
  if (!reverse_roles(p, nR, nS)) return join_device(p, R, nR, S, nS, out_count, out_checksum, pairs);
  uint64_t cnt = 0;
  rc = join_device(p, S, nS, R, nR, &cnt, out_checksum, pairs);
  if (out_count) *out_count = cnt;
  if (rc == MPSM_OK && pairs && pairs->data && cnt) {
    launch_swap_pairs(reinterpret_cast<Tuple*>(pairs->data), std::min<u64>(cnt, pairs->capacity), p->st, p->nsm);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(p->st));
  }
  return rc;
}

// tuples of the partitioned side per piece of a host-buffer join: the side is cut
// into equal pieces of at most a quarter of the run side, within [2^26, 2^27]
constexpr u64 HOST_PIECE_MIN = 1ull << 26, HOST_PIECE_MAX = 1ull << 27;

// Host-buffer join with the partitioned side copied in pieces.  The run side is
// copied and sorted first; then piece i is range-partitioned, sorted and joined
// against the sorted runs while piece i + 1 is still on the host link.  Exact for
// any split of the partitioned side: each pair (r, s) is found by the piece that
// holds s, and count and checksum are sums over the pairs.  The join waits only
// for the last piece's copy, so the step ends one piece's work after the link.
// The step's tail is the last piece's work, and every piece's work includes a pass
// over all of the sorted runs, so the pieces are equal and as small as lets each
// piece's work end before the next piece's copy: a quarter of the run side (on a
// link of about 210 GB/s, a 100 Mi-tuple piece against 400 Mi runs takes about
// 7 ms of work and 8 ms of copy).  A short remainder piece would not shorten that
// work, and the piece before it would still be computing when its copy ends.
static int join_host_pieces(mpsm_plan* p, Tuple* run_dst, const Tuple* run_src, u64 n_run, Tuple* part_dst,
                            const Tuple* part_src, u64 n_part, uint64_t* out_count, uint64_t* out_checksum) {
  const u64 target = std::min(std::max(n_run / 4, HOST_PIECE_MIN), HOST_PIECE_MAX);
  u64 nk = (n_part + target - 1) / target;
  if (nk > mpsm_plan::MAX_PIECES) nk = mpsm_plan::MAX_PIECES;
  const u32 K = (u32)nk;
  const u64 piece = (n_part + K - 1) / K;
  for (u32 i = 0; i < K; ++i)
    if (!p->ev_piece[i]) CK(cudaEventCreateWithFlags(&p->ev_piece[i], cudaEventDisableTiming));
  if (n_run) CK(cudaMemcpyAsync(run_dst, run_src, n_run * sizeof(Tuple), cudaMemcpyHostToDevice, p->st));
  CK(cudaEventRecord(p->ev_run_copied, p->st));  // also after every earlier reader of the staging buffers
  CK(cudaStreamWaitEvent(p->st_copy, p->ev_run_copied, 0));
  for (u32 i = 0; i < K; ++i) {
    const u64 a = (u64)i * piece, len = std::min(piece, n_part - a);
    CK(cudaMemcpyAsync(part_dst + a, part_src + a, len * sizeof(Tuple), cudaMemcpyHostToDevice, p->st_copy));
    CK(cudaEventRecord(p->ev_piece[i], p->st_copy));
  }
  CK(cudaEventRecord(p->ev_part_copied, p->st_copy));
  p->part_copy_pending = false;  // each piece waits for its own copy
  int rc = MPSM_OK;
  do {
    Jobh j{run_dst, part_dst, n_run, std::min(piece, n_part)};
    p->fused = true;
    if ((rc = setup_jobs(p, &j, 1))) break;
    if ((rc = phase_runs(p))) break;
    for (u32 i = 0; i < K && rc == MPSM_OK; ++i) {
      const u64 a = (u64)i * piece, len = std::min(piece, n_part - a);
      p->runs_reused = i > 0;  // the run side's fences and per-bucket counts depend on the runs only
      if (i) {
        launch_set_part(p->d_jobs, p->d_split, part_dst + a, len, p->st);
        if ((rc = cuda_status(cudaGetLastError()))) break;
        p->h_jobs[0].S = part_dst + a;
        p->h_jobs[0].nS = len;
      }
      if ((rc = cuda_status(cudaStreamWaitEvent(p->st, p->ev_piece[i], 0)))) break;
      if ((rc = phase_learn(p)) || (rc = phase_splitters(p)) || (rc = phase_scatter(p)) ||
          (rc = phase_sort_join(p)))
        break;
    }
    if (rc == MPSM_OK) rc = fused_results(p, out_count, out_checksum);
  } while (false);
  p->runs_reused = false;
  // nothing later on the plan's stream may overlap the copies, on the error paths too
  CK(cudaStreamWaitEvent(p->st, p->ev_part_copied, 0));
  return rc;
}

MPSM_API int mpsm_join_host(mpsm_plan_t* p, const mpsm_tuple_t* R_host, uint64_t nR, const mpsm_tuple_t* S_host,
                            uint64_t nS, uint64_t* out_count, uint64_t* out_checksum) {
  if (!p) return MPSM_ERR_INVALID_ARG;
  if ((nR && !R_host) || (nS && !S_host) || nR > p->max_nR || nS > p->max_nS) return MPSM_ERR_INVALID_ARG;
  if (!p->stage_r && dalloc(&p->stage_r, p->max_nR)) return MPSM_ERR_OOM;
  if (!p->stage_s && dalloc(&p->stage_s, p->max_nS)) return MPSM_ERR_OOM;
  if (!p->st_copy) {
    CK(cudaStreamCreateWithFlags(&p->st_copy, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&p->ev_run_copied, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&p->ev_part_copied, cudaEventDisableTiming));
  }
  const bool rev = reverse_roles(p, nR, nS);
  // the run side first, on the plan's stream, where its sort follows; the partitioned
  // side after it on the copy stream (the host link is the bound: one copy at a time
  // gets all of it), so the run-side sort runs while the larger copy is in flight
  Tuple* run_dst = rev ? p->stage_s : p->stage_r;
  Tuple* part_dst = rev ? p->stage_r : p->stage_s;
  const void* run_src = rev ? static_cast<const void*>(S_host) : static_cast<const void*>(R_host);
  const void* part_src = rev ? static_cast<const void*>(R_host) : static_cast<const void*>(S_host);
  const u64 n_run = rev ? nS : nR, n_part = rev ? nR : nS;
  if (n_part >= 2 * HOST_PIECE_MAX && !split_learned(p) && !search_learned(p) && !(p->opt.flags & MPSM_FLAG_UNFUSED))
    return join_host_pieces(p, run_dst, static_cast<const Tuple*>(run_src), n_run, part_dst,
                            static_cast<const Tuple*>(part_src), n_part, out_count, out_checksum);
  if (n_run) CK(cudaMemcpyAsync(run_dst, run_src, n_run * sizeof(Tuple), cudaMemcpyHostToDevice, p->st));
  CK(cudaEventRecord(p->ev_run_copied, p->st));  // also after every earlier reader of the staging buffers
  CK(cudaStreamWaitEvent(p->st_copy, p->ev_run_copied, 0));
  if (n_part) CK(cudaMemcpyAsync(part_dst, part_src, n_part * sizeof(Tuple), cudaMemcpyHostToDevice, p->st_copy));
  CK(cudaEventRecord(p->ev_part_copied, p->st_copy));
  p->part_copy_pending = true;
  const mpsm_tuple_t* r = reinterpret_cast<const mpsm_tuple_t*>(p->stage_r);
  const mpsm_tuple_t* sd = reinterpret_cast<const mpsm_tuple_t*>(p->stage_s);
  const int rc = rev ? join_device(p, sd, nS, r, nR, out_count, out_checksum, nullptr)
                     : join_device(p, r, nR, sd, nS, out_count, out_checksum, nullptr);
  if (int rw = wait_part_copy(p)) return rw;  // an early error return never reached the wait
  return rc;
}

MPSM_API int mpsm_join_batch(mpsm_plan_t* p, const mpsm_job_t* jobs, uint32_t njobs, uint64_t* out_counts,
                             uint64_t* out_checksums) {
  if (!p || !jobs || !njobs || njobs > p->max_jobs) return MPSM_ERR_INVALID_ARG;
  std::vector<Jobh> jh(njobs);
  u64 tR = 0, tS = 0;
  for (u32 i = 0; i < njobs; ++i) {
    if ((jobs[i].nR && !jobs[i].R) || (jobs[i].nS && !jobs[i].S)) return MPSM_ERR_INVALID_ARG;
    if (!aligned16(jobs[i].R) || !aligned16(jobs[i].S)) return MPSM_ERR_INVALID_ARG;
    jh[i] = Jobh{reinterpret_cast<const Tuple*>(jobs[i].R), reinterpret_cast<const Tuple*>(jobs[i].S), jobs[i].nR,
                 jobs[i].nS};
    tR += jobs[i].nR;
    tS += jobs[i].nS;
  }
  if (tR > p->max_nR || tS > p->max_nS) return MPSM_ERR_INVALID_ARG;
  p->fused = !(p->opt.flags & MPSM_FLAG_UNFUSED);
  int rc = setup_jobs(p, jh.data(), njobs);
  if (rc) return rc;
  // same job sizes and pointers as the captured graph -> replay it
  std::vector<u64> sig;
  sig.reserve(4 * njobs + 1);
  sig.push_back(p->opt.flags);
  for (u32 i = 0; i < njobs; ++i) {
    sig.push_back((u64)(uintptr_t)jh[i].R);
    sig.push_back(jh[i].nR);
    sig.push_back((u64)(uintptr_t)jh[i].S);
    sig.push_back(jh[i].nS);
  }
  if (!p->gexec || sig != p->gsig) {
    if (p->gexec) {
      cudaGraphExecDestroy(p->gexec);
      p->gexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    p->graph_mode = true;
    const bool saved_timing = p->timing;
    p->timing = false;
    CK(cudaStreamBeginCapture(p->st, cudaStreamCaptureModeThreadLocal));
    int prc = MPSM_OK;
    if (!prc) prc = phase_runs(p);
    if (!prc) prc = phase_learn(p);
    if (!prc) prc = phase_splitters(p);
    if (!prc) prc = phase_scatter(p);
    if (!prc && p->fused) prc = phase_sort_join(p);
    if (!prc && !p->fused) prc = phase_sort_parts(p);
    if (!prc && !p->fused) {
      LAUNCH(K_TILES, launch_tiles(p->d_jobs, p->njobs, p->tile, p->d_tot + T_TILES, &p->d_cnt[C_ERR], p->st));
      LAUNCH(K_SEARCH, launch_search(p->d_jobs, p->njobs, p->d_runs, p->xr, p->xs, p->tile, p->d_tot + T_TILES, p->d_win,
                                     lctx(p, search_learned(p)), p->st, p->nsm));
      LAUNCH(K_JOIN, launch_join(JOIN_AGG, p->d_jobs, p->njobs, p->d_runs, p->xr, p->xs, p->tile, p->d_tot + T_TILES, p->d_win,
                  nullptr, nullptr, nullptr, &p->d_cnt[C_ERR], p->st, p->nsm));
    }
    cudaError_t ce = cudaStreamEndCapture(p->st, &g);
    p->graph_mode = false;
    p->timing = saved_timing;
    if (prc) {
      if (g) cudaGraphDestroy(g);
      return prc;
    }
    if (ce != cudaSuccess) return MPSM_ERR_CUDA;
    p->graph_launches = p->launches;
    ce = cudaGraphInstantiate(&p->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return MPSM_ERR_CUDA;
    p->gsig = sig;
  }
  record(p, EV_START);
  CK(cudaGraphLaunch(p->gexec, p->st));
  p->launches = p->graph_launches;
  record(p, EV_JOIN);
  CK(cudaMemcpyAsync(p->h_jobs, p->d_jobs, njobs * sizeof(Job), cudaMemcpyDeviceToHost, p->st));
  rc = read_err(p);
  p->stage = ST_DONE;
  if (rc) return rc;
  for (u32 i = 0; i < njobs; ++i) {
    if (out_counts) out_counts[i] = p->h_jobs[i].count;
    if (out_checksums) out_checksums[i] = p->h_jobs[i].checksum;
  }
  return MPSM_OK;
}

MPSM_API int mpsm_plan_stats(mpsm_plan_t* p, mpsm_stats_t* s) {
  if (!p || !s) return MPSM_ERR_INVALID_ARG;
  memset(s, 0, sizeof(*s));
  CK(cudaStreamSynchronize(p->st));
  if (p->njobs == 0) return MPSM_OK;
  CK(cudaMemcpy(p->h_jobs, p->d_jobs, sizeof(Job), cudaMemcpyDeviceToHost));
  const Job& J = p->h_jobs[0];
  s->runs_r = J.runs;
  s->partitions_s = J.parts;
  s->nfine = J.nfine;
  s->fine_shift = J.fine_shift;
  s->s_kept = J.s_kept;
  s->tiles = J.ntiles;
  s->levels_r = p->levels_r;
  s->levels_s = p->levels_s;
  s->launches = p->launches;
  if (J.parts) {
    std::vector<u64> po(J.parts + 1);
    CK(cudaMemcpy(po.data(), p->d_part_off + J.part_base, (J.parts + 1) * sizeof(u64), cudaMemcpyDeviceToHost));
    u64 mx = 0;
    for (u32 i = 0; i < J.parts; ++i) mx = std::max<u64>(mx, po[i + 1] - po[i]);
    s->part_max = mx;
    s->imbalance = po[J.parts] ? (double)mx * J.parts / (double)po[J.parts] : 0.0;
  }
  if (p->fused) s->tiles = 0;
  if (!p->fused && J.ntiles && J.runs && p->stage >= ST_SEARCH) {
    const u64 nw = J.ntiles * J.runs;
    std::vector<u32> w(2 * nw);
    CK(cudaMemcpy(w.data(), p->d_win + 2 * J.win_base, 2 * nw * sizeof(u32), cudaMemcpyDeviceToHost));
    double sum = 0;
    for (u64 i = 0; i < nw; ++i) sum += (double)(w[2 * i + 1] - w[2 * i]);
    s->mean_window = sum / (double)nw;
  }
  {
    u64 ls[8];
    CK(cudaMemcpy(ls, p->d_lstat, sizeof(ls), cudaMemcpyDeviceToHost));
    s->part_probes = ls[1] ? (double)ls[0] / (double)ls[1] : 0.0;
    s->search_probes = ls[3] ? (double)ls[2] / (double)ls[3] : 0.0;
    s->search_err = (ls[3] && search_learned(p)) ? (double)ls[4] / (double)ls[3] : 0.0;
    if (p->d_models && p->learn) {
      float l[2];
      CK(cudaMemcpy(l, &p->d_models[0].loss0, sizeof(l), cudaMemcpyDeviceToHost));
      s->loss_s0 = l[0];
      s->loss_s = l[1];
      CK(cudaMemcpy(l, &p->d_models[1].loss0, sizeof(l), cudaMemcpyDeviceToHost));
      s->loss_r0 = l[0];
      s->loss_r = l[1];
    }
  }
  if (p->timing) {
    auto el = [&](int a, int b) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, p->ev[a], p->ev[b]) != cudaSuccess) {
        cudaGetLastError();
        ms = 0;
      }
      return ms;
    };
    s->ms_sort_runs = el(EV_START, EV_RUNS);
    s->ms_learn = el(EV_RUNS, EV_LEARN);
    s->ms_splitters = el(EV_LEARN, EV_SPLIT);
    s->ms_scatter = el(EV_SPLIT, EV_SCATTER);
    s->ms_sort_partitions = el(EV_SCATTER, EV_SORTS);
    s->ms_search = el(EV_SORTS, EV_SEARCH);
    s->ms_join = el(EV_SEARCH, EV_JOIN);
    s->ms_total = el(EV_START, EV_JOIN);
  }
  return MPSM_OK;
}

MPSM_API int mpsm_plan_set_flags(mpsm_plan_t* p, uint32_t flags) {
  if (!p) return MPSM_ERR_INVALID_ARG;
  if (flags & ~(u32)(MPSM_FLAG_TIMING | MPSM_FLAG_KERNEL_TIMING | MPSM_FLAG_UNFUSED | MPSM_FLAG_BOUNDS_TEST))
    return MPSM_ERR_INVALID_ARG;
  if ((flags & MPSM_FLAG_TIMING) && !p->ev[0])
    for (auto& e : p->ev)
      if (cudaEventCreate(&e) != cudaSuccess) return MPSM_ERR_CUDA;
  if ((flags & MPSM_FLAG_KERNEL_TIMING) && !p->kt_ev) {
    p->kt_ev = new (std::nothrow) cudaEvent_t[2 * KT_POOL];
    if (!p->kt_ev) return MPSM_ERR_OOM;
    for (u32 i = 0; i < 2 * KT_POOL; ++i)
      if (cudaEventCreate(&p->kt_ev[i]) != cudaSuccess) return MPSM_ERR_CUDA;
  }
  p->opt.flags = flags;
  p->timing = (flags & MPSM_FLAG_TIMING) != 0;
  if (p->sub) {
    const int rc = mpsm_plan_set_flags(p->sub, flags & MPSM_FLAG_KERNEL_TIMING);
    if (rc) return rc;
  }
  if (p->rsub) {
    const int rc = mpsm_plan_set_flags(p->rsub, flags & MPSM_FLAG_KERNEL_TIMING);
    if (rc) return rc;
  }
  return MPSM_OK;
}

MPSM_API int mpsm_plan_kernel_times(mpsm_plan_t* p, mpsm_kernel_time_t* out, uint32_t cap, uint32_t* n) {
  if (!p || !n || (cap && !out)) return MPSM_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(p->st));
  float ms[K_NUM] = {};
  u32 cnt[K_NUM] = {};
  auto add = [&](const mpsm_plan* q) {
    for (u32 i = 0; i < q->kt_n; ++i) {
      float t = 0;
      if (cudaEventElapsedTime(&t, q->kt_ev[2 * i], q->kt_ev[2 * i + 1]) != cudaSuccess) {
        cudaGetLastError();
        t = 0;
      }
      ms[q->kt_id[i]] += t;
      cnt[q->kt_id[i]] += 1;
    }
  };
  add(p);
  if (p->learn && split_learned(p) && p->sub && p->sub->kt_ev) add(p->sub);  // the sample sort
  if (runs_learned(p) && p->rsub && p->rsub->kt_ev) add(p->rsub);              // the run-side sample sort
  u32 k = 0;
  for (u32 id = 0; id < K_NUM; ++id) {
    if (!cnt[id]) continue;
    if (k < cap) {
      memset(&out[k], 0, sizeof(out[k]));
      strncpy(out[k].name, KNAME[id], sizeof(out[k].name) - 1);
      out[k].launches = cnt[id];
      out[k].ms = ms[id];
    }
    ++k;
  }
  *n = k;
  return MPSM_OK;
}

MPSM_API int mpsm_plan_view(mpsm_plan_t* p, mpsm_view_t* v) {
  if (!p || !v) return MPSM_ERR_INVALID_ARG;
  memset(v, 0, sizeof(*v));
  CK(cudaStreamSynchronize(p->st));
  if (p->njobs == 0) return MPSM_ERR_STATE;
  CK(cudaMemcpy(p->h_jobs, p->d_jobs, sizeof(Job), cudaMemcpyDeviceToHost));
  const Job& J = p->h_jobs[0];
  // run boundaries of job 0 as one array (xr offsets)
  const u64 nchunks = J.nS ? (J.nS + p->ch_s - 1) / p->ch_s : 0;
  const u64 need = (u64)J.runs + 1 + nchunks + 1;
  if (need > p->chunk_off_cap) {
    dfree(p->d_chunk_off);
    p->chunk_off_cap = need + 64;
    if (dalloc(&p->d_chunk_off, p->chunk_off_cap)) return MPSM_ERR_OOM;
  }
  std::vector<u64> h(need);
  for (u32 j = 0; j < J.runs; ++j) h[j] = p->h_runs[J.run_base + j].off - J.r_base;
  h[J.runs] = J.nR;
  for (u64 c = 0; c <= nchunks; ++c) h[J.runs + 1 + c] = std::min<u64>(c * p->ch_s, J.nS);
  CK(cudaMemcpy(p->d_chunk_off, h.data(), need * sizeof(u64), cudaMemcpyHostToDevice));
  v->r_runs = reinterpret_cast<const mpsm_tuple_t*>(p->xr + J.r_base);
  v->run_offsets = reinterpret_cast<const uint64_t*>(p->d_chunk_off);
  v->runs_r = J.runs;
  v->key_min = J.kmin;
  v->key_max = J.kmax;
  v->nfine = J.nfine;
  v->fine_shift = J.fine_shift;
  v->fine_s = reinterpret_cast<const uint64_t*>(p->d_fine_s + J.fine_base);
  v->fine_r = reinterpret_cast<const uint64_t*>(p->d_fine_r + J.fine_base);
  v->splitters = p->d_sp + J.fine_base;
  v->partitions_s = J.parts;
  v->s_chunks = (u32)nchunks;
  v->s_chunk_offsets = reinterpret_cast<const uint64_t*>(p->d_chunk_off + J.runs + 1);
  v->chunk_offsets = p->d_hist_a;  // valid after mpsm_splitters / mpsm_scatter (job 0's chunks first)
  v->part_offsets = reinterpret_cast<const uint64_t*>(p->d_part_off + J.part_base);
  v->s_buffer = reinterpret_cast<const mpsm_tuple_t*>(p->xs + J.s_base);
  v->s_kept = J.s_kept;
  v->tiles = J.ntiles;
  v->join_tile = p->tile;
  v->windows = p->d_win + 2 * J.win_base;
  if (p->fused) {
    u32 nfin = 0;
    CK(cudaMemcpy(&nfin, &p->d_cnt[C_FIN], sizeof(u32), cudaMemcpyDeviceToHost));
    v->segments = reinterpret_cast<const mpsm_segment_t*>(p->d_fin);
    v->n_segments = std::min(nfin, p->fin_cap);
    v->window_stride = p->maxT;
    v->seg_windows = p->d_swin;
  }
  v->pass_buffer = reinterpret_cast<const mpsm_tuple_t*>(p->y);
  return MPSM_OK;
}

static_assert(sizeof(mpsm_segment_t) == sizeof(Seg) && offsetof(mpsm_segment_t, key_hi) == offsetof(Seg, kmax) &&
                  offsetof(mpsm_segment_t, flags) == offsetof(Seg, flags),
              "mpsm_segment_t mirrors the segment records");

static_assert(DERR_SEG_OVERFLOW == MPSM_DEVERR_LIST_OVERFLOW && DERR_SEG_TOO_BIG == MPSM_DEVERR_SEGMENT_TOO_BIG &&
                  DERR_TMA_TIMEOUT == MPSM_DEVERR_WAIT_TIMEOUT && DERR_LEVELS == MPSM_DEVERR_LEVELS &&
                  DERR_HIST_OVERFLOW == MPSM_DEVERR_HIST_OVERFLOW && DERR_LEARN == MPSM_DEVERR_LEARN &&
                  DERR_BOUNDS == MPSM_DEVERR_BOUNDS,
              "device check bits match the ABI");

MPSM_API int mpsm_plan_device_errors(const mpsm_plan_t* p, uint32_t* flags) {
  if (!p || !flags) return MPSM_ERR_INVALID_ARG;
  *flags = p->device_errors;
  return MPSM_OK;
}

MPSM_API int mpsm_selftest_wait_timeout(void* stream, uint32_t spin_limit, uint32_t* flags) {
  if (!flags) return MPSM_ERR_INVALID_ARG;
  *flags = 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  u32* d_flag = nullptr;
  if (cudaMalloc(&d_flag, sizeof(u32)) != cudaSuccess) return MPSM_ERR_OOM;
  u32 h = 0;
  cudaError_t e = cudaMemsetAsync(d_flag, 0, sizeof(u32), st);
  if (e == cudaSuccess) {
    launch_wait_selftest(d_flag, spin_limit ? spin_limit : 1000u, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_flag, sizeof(u32), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_flag);
  if (e != cudaSuccess) return MPSM_ERR_CUDA;
  *flags = h;
  return h ? MPSM_ERR_DEVICE : MPSM_OK;
}

MPSM_API int mpsm_selftest_log2_q16(const uint64_t* n, uint64_t count, uint64_t* out, uint32_t wide, void* stream) {
  if (count && (!n || !out)) return MPSM_ERR_INVALID_ARG;
  if ((((uintptr_t)n) | ((uintptr_t)out)) & 7u) return MPSM_ERR_INVALID_ARG;
  if (count == 0) return MPSM_OK;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MPSM_ERR_CUDA;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  launch_log2_selftest(reinterpret_cast<const u64*>(n), count, reinterpret_cast<u64*>(out), wide, st, nsm > 0 ? nsm : 1);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return MPSM_ERR_CUDA;
  return MPSM_OK;
}

MPSM_API const char* mpsm_strerror(int status) {
  switch (status) {
    case MPSM_OK: return "ok";
    case MPSM_ERR_INVALID_ARG: return "invalid argument";
    case MPSM_ERR_OOM: return "out of device memory";
    case MPSM_ERR_CUDA: return "CUDA error";
    case MPSM_ERR_CAPACITY: return "pair buffer too small";
    case MPSM_ERR_DEVICE: return "device-side check failed";
    case MPSM_ERR_STATE: return "phase called out of order";
    default: return "unknown status";
  }
}

// ============================================================== learned model on caller data

namespace {

// model slot 0 takes caller data (slot 1 is switched off)
int rmi_slot0(mpsm_plan* p, u32 n, u64 kmin, u64 kmax, bool init) {
  int rc = alloc_learn(p);
  if (rc) return rc;
  p->learn = false;  // the last join's learned state is gone
  p->h_tasks[0] = RmiTask{0, 0, kmin, kmax, 0, RMI_KIND_GIVEN, n, 1};
  p->h_tasks[1] = RmiTask{0, 0, 0, 0, 0, RMI_KIND_GIVEN, 0, 0};
  CK(cudaMemcpyAsync(p->d_tasks, p->h_tasks, 2 * sizeof(RmiTask), cudaMemcpyHostToDevice, p->st));
  launch_rmi_setup(p->d_models, p->d_tasks, 2, p->d_jobs, init, p->st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(p->st));
  return MPSM_OK;
}

// caller's training points into slot 0
int rmi_points(mpsm_plan* p, const float* x, const float* y, u32 n, const float* theta) {
  int rc = rmi_slot0(p, n, 0, 1, false);
  if (rc) return rc;
  CK(cudaMemcpyAsync(p->d_tx, x, n * sizeof(float), cudaMemcpyDeviceToDevice, p->st));
  CK(cudaMemcpyAsync(p->d_ty, y, n * sizeof(float), cudaMemcpyDeviceToDevice, p->st));
  CK(cudaMemcpyAsync(p->d_models[0].theta, theta, RMI_NP * sizeof(float), cudaMemcpyDeviceToDevice, p->st));
  u32* hn = reinterpret_cast<u32*>(p->h_scalar);
  hn[0] = n;
  CK(cudaMemcpyAsync(&p->d_models[0].train_n, hn, sizeof(u32), cudaMemcpyHostToDevice, p->st));
  CK(cudaStreamSynchronize(p->st));
  return MPSM_OK;
}

}  // namespace

MPSM_API int mpsm_rmi_loss_grad(mpsm_plan_t* p, const float* x, const float* y, uint32_t n, const float* theta,
                                float* grad, float* loss) {
  if (!p || !x || !y || !theta || !grad || !loss || n == 0 || n > RMI_TRAIN_MAX) return MPSM_ERR_INVALID_ARG;
  int rc = rmi_points(p, x, y, n, theta);
  if (rc) return rc;
  launch_rmi_grad(p->d_models, 1, p->d_tx, p->d_ty, p->d_partial, p->st);
  launch_rmi_reduce(p->d_partial, grad, &p->d_models[0].loss, p->st);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(loss, &p->d_models[0].loss, sizeof(float), cudaMemcpyDeviceToHost, p->st));
  CK(cudaStreamSynchronize(p->st));
  return MPSM_OK;
}

MPSM_API int mpsm_rmi_train(mpsm_plan_t* p, const float* x, const float* y, uint32_t n, uint32_t steps, float lr,
                            float* theta, float* losses) {
  if (!p || !x || !y || !theta || n == 0 || n > RMI_TRAIN_MAX || !(lr > 0.0f)) return MPSM_ERR_INVALID_ARG;
  int rc = rmi_points(p, x, y, n, theta);
  if (rc) return rc;
  if (losses && steps > p->fit_cap) return MPSM_ERR_INVALID_ARG;
  CK(cudaMemsetAsync(&p->d_cnt[C_ERR], 0, sizeof(u32), p->st));
  if ((rc = train_models(p, 1, steps, lr, losses ? p->d_fity : nullptr))) return rc;
  if ((rc = read_err(p))) return rc;
  CK(cudaMemcpyAsync(theta, p->d_models[0].theta, RMI_NP * sizeof(float), cudaMemcpyDeviceToDevice, p->st));
  if (losses && steps) CK(cudaMemcpyAsync(losses, p->d_fity, steps * sizeof(float), cudaMemcpyDeviceToHost, p->st));
  CK(cudaStreamSynchronize(p->st));
  return MPSM_OK;
}

MPSM_API int mpsm_rmi_fit(mpsm_plan_t* p, const uint64_t* keys, const float* y, uint32_t n, uint64_t kmin,
                          uint64_t kmax, uint32_t steps, float lr) {
  if (!p || !keys || !y || kmax < kmin || !(lr > 0.0f)) return MPSM_ERR_INVALID_ARG;
  int rc = alloc_learn(p);
  if (rc) return rc;
  if (n > p->fit_cap) return MPSM_ERR_INVALID_ARG;
  rc = rmi_slot0(p, n, kmin, kmax, true);
  if (rc) return rc;
  if (n) {
    CK(cudaMemcpyAsync(p->d_fitk, keys, n * sizeof(u64), cudaMemcpyDeviceToDevice, p->st));
    CK(cudaMemcpyAsync(p->d_fity, y, n * sizeof(float), cudaMemcpyDeviceToDevice, p->st));
  }
  launch_fit_data(p->d_models, p->d_tasks, 1, p->d_jobs, p->d_runs, p->xr, nullptr, p->d_fitk, p->d_fity, p->st, p->nsm);
  launch_train_data(p->d_models, 1, p->d_fitk, p->d_fity, p->d_tx, p->d_ty, p->st);
  CK(cudaMemsetAsync(&p->d_cnt[C_ERR], 0, sizeof(u32), p->st));
  if ((rc = train_models(p, 1, steps, lr, nullptr))) return rc;
  launch_rmi_tabulate(p->d_models, 1, p->st);
  launch_leaf_fit(p->d_models, 1, p->d_leafacc, p->d_fitk, p->d_fity, p->st, p->nsm);
  CK(cudaGetLastError());
  return read_err(p);
}

MPSM_API int mpsm_rmi_predict(mpsm_plan_t* p, uint32_t slot, const uint64_t* keys, uint64_t n, float* yhat,
                              uint32_t* leaf) {
  if (!p || slot > 1 || (n && (!keys || !yhat))) return MPSM_ERR_INVALID_ARG;
  if (!p->d_models) return MPSM_ERR_STATE;
  launch_rmi_predict(p->d_models + slot, reinterpret_cast<const u64*>(keys), n, yhat, leaf, p->st, p->nsm);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(p->st));
  return MPSM_OK;
}

MPSM_API int mpsm_rmi_export(mpsm_plan_t* p, uint32_t slot, mpsm_rmi_info_t* info, float* theta, uint16_t* cell_leaf,
                             uint64_t* leaf_base, float* leaf_a, float* leaf_b) {
  if (!p || slot > 1) return MPSM_ERR_INVALID_ARG;
  if (!p->d_models) return MPSM_ERR_STATE;
  RmiModel* h = new (std::nothrow) RmiModel;
  if (!h) return MPSM_ERR_OOM;
  CK(cudaStreamSynchronize(p->st));
  if (cudaMemcpy(h, p->d_models + slot, sizeof(RmiModel), cudaMemcpyDeviceToHost) != cudaSuccess) {
    delete h;
    return MPSM_ERR_CUDA;
  }
  if (info) {
    info->kmin = h->kmin;
    info->kmax = h->kmax;
    info->cshift = h->cshift;
    info->ncell = h->ncell;
    info->fit_n = h->fit_n;
    info->train_n = h->train_n;
    info->loss0 = h->loss0;
    info->loss = h->loss;
  }
  if (theta) memcpy(theta, h->theta, RMI_NP * sizeof(float));
  if (cell_leaf) memcpy(cell_leaf, h->tab, sizeof(h->tab));
  for (u32 l = 0; l < RMI_LEAVES; ++l) {
    if (leaf_base) leaf_base[l] = h->leaf[l].base;
    if (leaf_a) leaf_a[l] = h->leaf[l].a;
    if (leaf_b) leaf_b[l] = h->leaf[l].b;
  }
  delete h;
  return MPSM_OK;
}

// ============================================================== tuning

MPSM_API int mpsm_plan_set_tuning(mpsm_plan_t* p, const mpsm_tuning_t* t) {
  if (!p || !t) return MPSM_ERR_INVALID_ARG;
  if (t->radix_bits && (t->radix_bits < 4 || t->radix_bits > 11)) return MPSM_ERR_INVALID_ARG;
  if (t->join_tile && (t->join_tile < 256 || t->join_tile > TILE_MAX || t->join_tile % 256)) return MPSM_ERR_INVALID_ARG;
  if (t->partitions_s > P_MAX) return MPSM_ERR_INVALID_ARG;
  p->opt.radix_bits = t->radix_bits;
  p->opt.join_tile = t->join_tile;
  p->opt.run_len = t->run_len;
  p->opt.partitions_s = t->partitions_s;
  p->tile = t->join_tile ? t->join_tile : TILE_MAX;
  if (p->gexec) {
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  p->gsig.clear();
  return MPSM_OK;
}

MPSM_API int mpsm_autotune(mpsm_plan_t* p, const mpsm_job_t* jobs, uint32_t njobs, uint32_t reps, mpsm_tuning_t* best,
                           float* best_ms) {
  if (!p || !jobs || !njobs || !best || !best_ms) return MPSM_ERR_INVALID_ARG;
  if (reps == 0) reps = 1;
  std::vector<mpsm_tuning_t> cand;
  for (u32 rb : {11u, 9u})
    for (u32 tile : {4096u, 2048u})
      for (u32 rl : {0u, 1u << 23}) cand.push_back(mpsm_tuning_t{rb, tile, rl, p->opt.partitions_s});
  std::vector<uint64_t> c0(njobs), s0(njobs), c(njobs), s(njobs);
  float best_t = 0;
  int best_i = -1;
  for (size_t i = 0; i < cand.size(); ++i) {
    int rc = mpsm_plan_set_tuning(p, &cand[i]);
    if (rc) return rc;
    rc = mpsm_join_batch(p, jobs, njobs, c.data(), s.data());  // capture + warm-up
    if (rc) return rc;
    if (i == 0) {
      c0 = c;
      s0 = s;
    } else if (c != c0 || s != s0) {
      return MPSM_ERR_DEVICE;
    }
    const auto t0 = std::chrono::steady_clock::now();
    for (u32 r = 0; r < reps; ++r) {
      rc = mpsm_join_batch(p, jobs, njobs, c.data(), s.data());
      if (rc) return rc;
    }
    const float ms =
        std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count() / (float)reps;
    if (best_i < 0 || ms < best_t) {
      best_t = ms;
      best_i = (int)i;
    }
  }
  *best = cand[best_i];
  *best_ms = best_t;
  return mpsm_plan_set_tuning(p, best);
}
