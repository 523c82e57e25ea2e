// mpsm_launch.h -- host-side launchers of the MPSM kernels (one per kernel family).
#pragma once

#include <cuda_runtime.h>

#include "learn.cuh"
#include "mpsm_internal.cuh"

namespace mpsm {

// one-time kernel attribute setup (dynamic shared memory limits); call before any capture
void init_attrs_pass();
void init_attrs_split();
void init_attrs_join();
void init_attrs_learn();

// ---- partitioning passes (k_pass.cu)
void launch_sample_bounds(Seg* segs, const u32* nseg, u32 max_segs, Bufs bufs, const Job* jobs, cudaStream_t st);
void launch_level_plan(const Seg* segs, u32* nseg, u32 seg_cap, LSeg* ls, u64* totals, u32 mode, u64 chunk,
                       u32 radix_bits, const Job* jobs, u64 hist_cap, u64 bucket_cap, u32* err, cudaStream_t st,
                       u64 fill = 0,   // MODE_RADIX: target tuples per bucket, 0 = power-of-two buckets
                       const LearnCtx* lc = nullptr);  // MODE_RLEARN: the learned run bucket tables
void launch_init_buckets(u64* bmin, u64* bmax, u64* btot, const u64* totals, cudaStream_t st, int nsm);
void launch_hist(u32 mode, const Seg* segs, const u32* nseg, const LSeg* ls, const u64* totals, u64 chunk,
                 Bufs bufs, const Job* jobs, u32 src_where, u32* hist, u64* bmin, u64* bmax, u64* btot,
                 const LearnCtx& lc, cudaStream_t st, int nsm);
void launch_scan(u32 mode, const Seg* segs, const u32* nseg, const LSeg* ls, u32* hist, const u64* bmin,
                 const u64* bmax, const u32* part_fstart, Seg* big_out, u32* big_cnt, u32 big_cap, Seg* fin_out,
                 u32* fin_cnt, u32 fin_cap, u32 dst_where, Job* jobs, u64* part_off, u32* err, cudaStream_t st,
                 int nsm, bool keep_const = false,
                 const u64* lbnd = nullptr);  // MODE_LEARN: the learned boundaries (P_MAX per job)
void launch_scatter(u32 mode, const Seg* segs, const u32* nseg, const LSeg* ls, const u64* totals, u64 chunk,
                    Bufs bufs, const Job* jobs, u32 src_where, u32 dst_where, const u32* hist, const u32* sp,
                    u32* err, const LearnCtx& lc, cudaStream_t st, int nsm, bool big_tiles = false);
void launch_seg_sort(const Seg* segs, const u32* nseg, u32 cap, u32* work, Bufs bufs, const Job* jobs,
                     u32 dst_where, u32* err, cudaStream_t st, int nsm);
void launch_check_empty(const u32* cnt, u32* err, u32 flag, cudaStream_t st);
void launch_set_part(Job* jobs, Seg* split, const Tuple* S, u64 nS, cudaStream_t st);  // piecewise host join
void launch_narrow_bounds_test(Seg* segs, const u32* nseg, u32 cap, cudaStream_t st);  // MPSM_FLAG_BOUNDS_TEST
// phases 3 + 4 fused (k_pass.cu): fences of the sorted runs, per (segment, run) windows, sort-and-join
void launch_fences(const Tuple* xr, u64 n, u64* fence, cudaStream_t st, int nsm);
void launch_seg_search(const Seg* segs, const u32* nseg, u32 cap, const Job* jobs, const Run* runs, const Tuple* xr,
                       const u64* fence, u32* swin, u32 maxT, const LearnCtx& lc, cudaStream_t st, int nsm);
void launch_seg_sort_join(const Seg* segs, const u32* nseg, u32 cap, u32* work, Bufs bufs, const Job* jobs, u32* err,
                          const FuseCtx& fc, cudaStream_t st, int nsm);

// ---- splitters (k_split.cu)
void launch_run_bounds(Job* jobs, u32 njobs, const Run* runs, const Tuple* xr, cudaStream_t st);
void launch_run_cdf(const Job* jobs, u32 njobs, const Run* runs, const Tuple* xr, u64* rc, cudaStream_t st);
void launch_splitters(Job* jobs, u32 njobs, const u64* fine_s, const u64* rc, u64* fine_r, u32* sp,
                      u32* part_fstart, u32* err, cudaStream_t st, bool equi_height = false);
void launch_log2_selftest(const u64* n, u64 count, u64* out, u32 wide, cudaStream_t st, int nsm);
void launch_fold(const Seg* segs, const u32* nseg, const LSeg* ls_fine, const LSeg* ls_split, const u64* totals,
                 const Job* jobs, const u32* hist_fine, const u32* part_fstart, u32* hist_split, cudaStream_t st,
                 int nsm);

// ---- join (k_join.cu)
void launch_tiles(Job* jobs, u32 njobs, u32 tile, u64* totals, const u32* err, cudaStream_t st);
void launch_search(const Job* jobs, u32 njobs, const Run* runs, const Tuple* xr, const Tuple* xs, u32 tile,
                   const u64* totals, u32* win, const LearnCtx& lc, cudaStream_t st, int nsm);
void launch_join(u32 mode, Job* jobs, u32 njobs, const Run* runs, const Tuple* xr, const Tuple* xs, u32 tile,
                 const u64* totals, const u32* win, u64* tile_cnt, const u64* tile_out, Tuple* pairs,
                 u32* err, cudaStream_t st, int nsm);
void launch_swap_pairs(Tuple* pairs, u64 n, cudaStream_t st, int nsm);
void launch_wait_selftest(u32* flag, u32 limit, cudaStream_t st);  // bounded-wait self-test
void launch_pair_offsets(Job* jobs, u32 njobs, const u64* totals, const u64* tile_cnt, u64* tile_out,
                         u64* pair_total, cudaStream_t st);

// ---- learned CDF model (k_learn.cu)
enum RmiKind : u32 {
  RMI_KIND_SAMPLE = 0,  // a sorted sample of S (the sub-plan's runs); fit points = its slice inside R's range
  RMI_KIND_RUNS = 1,    // evenly spaced positions of the job's sorted R runs
  RMI_KIND_GIVEN = 2    // fit points written by the caller; range given in the RmiTask
};
struct RmiTask {
  u64 fit_off;          // first fit point (keys / CDF values) of the model
  u64 src_off;          // RMI_KIND_SAMPLE: first tuple of the job's sorted sample
  u64 kmin, kmax;       // RMI_KIND_GIVEN: normalisation range
  u32 job, kind;
  u32 cap;              // sample size / fit points
  u32 active;
};
size_t leaf_acc_bytes();
void launch_rmi_setup(RmiModel* models, const RmiTask* tasks, u32 nmodels, const Job* jobs, bool init,
                      cudaStream_t st);
void launch_fit_data(RmiModel* models, const RmiTask* tasks, u32 nmodels, const Job* jobs, const Run* runs,
                     const Tuple* xr, const Tuple* samp, u64* fitk, float* fity, cudaStream_t st, int nsm);
void launch_train_data(RmiModel* models, u32 nmodels, const u64* fitk, const float* fity, float* X, float* Y,
                       cudaStream_t st);
void launch_rmi_grad(const RmiModel* models, u32 nmodels, const float* X, const float* Y, float* partial,
                     cudaStream_t st);
void launch_rmi_adam(RmiModel* models, u32 nmodels, const float* partial, u32 step, float lr, cudaStream_t st);
// every Adam step in one cooperative launch when rmi_train_capacity(dev) >= RMI_GMAX * nmodels
u32 rmi_train_capacity(int dev);
cudaError_t launch_rmi_train(RmiModel* models, u32 nmodels, const float* X, const float* Y, float* partial, u32* bar,
                             u32 steps, float lr, float* losses, u32* err, cudaStream_t st);
void launch_rmi_reduce(const float* partial, float* grad, float* loss, cudaStream_t st);
void launch_rmi_tabulate(RmiModel* models, u32 nmodels, cudaStream_t st);
void launch_leaf_fit(RmiModel* models, u32 nmodels, void* acc, const u64* fitk, const float* fity, cudaStream_t st,
                     int nsm);
void launch_learn_bounds(Job* jobs, u32 njobs, const RmiModel* models, const u64* fitk, u64* bnd, u32* brank,
                         cudaStream_t st);
void launch_sample_s(const Job* jobs, u32 njobs, const u64* samp_off, const u32* samp_n, Tuple* samp,
                     cudaStream_t st, int nsm);
void launch_learn_cells(const Job* jobs, u32 njobs, const u64* bnd, u32* cell, cudaStream_t st);
// the learned run bucket function: run-side sample, then its tables from the sorted sample
void launch_sample_r(const Job* jobs, u32 njobs, const u64* samp_off, const u32* samp_n, Tuple* samp,
                     cudaStream_t st, int nsm);
void launch_rlearn_tables(const Job* jobs, u32 njobs, const Tuple* sorted, const u64* samp_off, const u32* samp_n,
                          RunLearn* rl, u32* rcell, u64* rbnd, cudaStream_t st);
void launch_rmi_predict(const RmiModel* M, const u64* keys, u64 n, float* yhat, u32* leaf, cudaStream_t st, int nsm);

enum JoinMode : u32 { JOIN_AGG = 0, JOIN_COUNT = 1, JOIN_WRITE = 2 };

}  // namespace mpsm
