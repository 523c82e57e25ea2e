/*
 * mpsm.h -- C ABI of libmpsm, a GB300 (sm_103a) implementation of the MPSM
 * massively parallel sort-merge equi-join (Albutiu, Kemper, Neumann, "Massively
 * Parallel Sort-Merge Joins in Main Memory Multi-Core Database Systems").
 *
 * The join R |><| S on 64-bit keys runs as the paper's range-partitioned P-MPSM
 * (Sec. 3.2, Fig. 5), with the two inputs in these roles:
 *   - R is cut into T_R chunks, each sorted independently into a run
 *     (phase 1, Sec. 2.1/3.2); runs are never merged (Sec. 2);
 *   - S is range-partitioned by splitters computed from histograms and prefix
 *     sums (phase 2, Sec. 3.2.1, 4.2, 4.3), then each partition is sorted
 *     (phase 3);
 *   - every sorted S partition is merge-joined against all R runs, a search
 *     locating where each run's relevant part starts (phase 4, Sec. 3.2.2).
 * This is the paper's role-reversal orientation (Sec. 3.2 last paragraph,
 * Sec. 5.4): the partitioned input is S, the run input is R.  The result does
 * not depend on the roles.
 *
 * Result (Sec. 5.1's query, with the aggregate every payload flows into):
 *   count    = |{(r, s) in R x S : r.key == s.key}|
 *   checksum = sum over those pairs of (r.payload + s.payload), modulo 2^64
 *   pairs    = optionally the pairs (r.payload, s.payload), in no particular order.
 *
 * Conventions for every entry point:
 *  - Tuples are 16-byte {key, payload} records, 16-byte aligned, in DEVICE
 *    memory unless the function says HOST.  R and S are read only.
 *  - All work is enqueued on the plan's CUDA stream.  Functions that return
 *    host values (counts, checksums, stats, views) synchronise that stream.
 *  - Return value: MPSM_OK (0) or an MPSM_ERR_* code; nothing aborts or prints.
 *    mpsm_strerror() names a code.  After MPSM_ERR_CUDA the plan must be
 *    destroyed.
 *  - A plan is not thread-safe; use one plan per host thread / stream.
 */
#ifndef MPSM_H
#define MPSM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { uint64_t key, payload; } mpsm_tuple_t;          /* 16 B */
typedef struct { uint64_t r_payload, s_payload; } mpsm_pair_t;    /* 16 B */
typedef struct { mpsm_pair_t* data; uint64_t capacity; } mpsm_pairs_t;
typedef struct mpsm_plan mpsm_plan_t;

enum {
  MPSM_OK = 0,
  MPSM_ERR_INVALID_ARG = 1,   /* null/misaligned pointer, size above the plan's maximum   */
  MPSM_ERR_OOM = 2,           /* device allocation failed                                  */
  MPSM_ERR_CUDA = 3,          /* a CUDA call failed                                        */
  MPSM_ERR_CAPACITY = 4,      /* pair buffer too small; *out_count holds the needed size   */
  MPSM_ERR_DEVICE = 5,        /* a kernel detected a violated invariant or gave up a wait  */
  MPSM_ERR_STATE = 6          /* a phase entry point called before the phase it needs      */
};

/* Splitters of S (Sec. 4.3): HIST minimises the largest split-relevant cost
 * |S_i| log|S_i| + T |S_i| + |R in range| over contiguous groups of the fine
 * buckets; EQUI_HEIGHT groups the same buckets by |S_i| alone, the equi-height
 * baseline of Sec. 5.6 (Fig. 16b); LEARNED takes sample quantiles (below). */
enum { MPSM_SPLIT_HIST = 0, MPSM_SPLIT_LEARNED = 1, MPSM_SPLIT_EQUI_HEIGHT = 2 };
/* Merge-start search in the sorted runs (Sec. 3.2.2): BINARY (with a fence index
 * of every 64th run key on the fused path), LEARNED (the R-side model's guess, then
 * exponential + binary search), INTERP (the paper's interpolation search: up to 16
 * rule-of-proportion probes between the known end keys, then binary search).  All
 * three find the exact bounds; they differ in probes and time only. */
enum { MPSM_SEARCH_BINARY = 0, MPSM_SEARCH_LEARNED = 1, MPSM_SEARCH_INTERP = 2 };
/* Role of the inputs (Sec. 3.2, Sec. 5.4 "role reversal"): which input is
 * range-partitioned; the other one is cut into sorted runs.  The result does not
 * depend on it (pairs keep their (r_payload, s_payload) order either way). */
enum { MPSM_PART_S = 0, MPSM_PART_R = 1, MPSM_PART_SMALLER = 2 };
/* Bucket function of the first sort pass over each run (Sec. 3.2.1 radix clustering):
 * RADIX takes equal-width ranges of the run's key range; LEARNED takes the quantiles of an
 * evenly spaced sample of the run-side input, sorted first (the empirical CDF the
 * learned splitters use, Sec. 4.1-4.2), so skewed or clustered keys still fill every
 * bucket evenly and the runs need fewer passes.  A key equal to several quantiles goes
 * whole to the first bucket they bound.  The sorted runs are the same. */
enum { MPSM_RUNS_RADIX = 0, MPSM_RUNS_LEARNED = 1 };
enum {
  MPSM_FLAG_TIMING = 1u,          /* record per-phase CUDA events (read by mpsm_plan_stats)        */
  MPSM_FLAG_KERNEL_TIMING = 2u,   /* record CUDA events around every kernel launch (read by
                                     mpsm_plan_kernel_times); adds a few microseconds per launch  */
  MPSM_FLAG_UNFUSED = 4u          /* mpsm_join / mpsm_join_batch: run phase 3 and phase 4 as separate
                                     kernels (sorted S written back, then searched and joined)
                                     instead of joining each S segment while its sort still holds
                                     it in shared memory; same results                            */,
  MPSM_FLAG_BOUNDS_TEST = 8u      /* test only: before phase 3's final in-shared-memory sorts, narrow
                                     the recorded key bounds of one S segment so that its largest
                                     key lies beyond them; the sort kernels then report
                                     MPSM_DEVERR_BOUNDS and the call returns MPSM_ERR_DEVICE.  It
                                     exercises the kernels' own check of those bounds; no access
                                     leaves its array                                          */
};

typedef struct {
  uint32_t runs_r;         /* T_R, runs cut from R (Sec. 2.1 "T chunks"); 0 = automatic       */
  uint32_t partitions_s;   /* P, partitions of S (at most 2^fine_bits); 0 = automatic        */
  uint32_t fine_bits;      /* B, bits of the fine S histogram (Sec. 4.2), 1..12; 0 = 12      */
  uint32_t radix_bits;     /* log2 of the largest sort fan-out per pass, 4..11; 0 = 11       */
  uint32_t join_tile;      /* S tuples per join tile, 256..4096, multiple of 256; 0 = 4096   */
  int32_t splitter_mode;   /* MPSM_SPLIT_*                                                   */
  int32_t search_mode;     /* MPSM_SEARCH_*                                                  */
  uint32_t flags;          /* MPSM_FLAG_*                                                    */
  uint64_t seed;           /* seed of the hash that spreads hot keys over learned partitions */
  uint32_t learn_steps;    /* Adam steps of the learned model; 0 = 200                       */
  uint32_t run_len;        /* target R tuples per run when runs_r = 0; 0 = automatic          */
  uint32_t partition_side; /* MPSM_PART_*: mpsm_join / mpsm_join_host partition S (default), R,
                              or the smaller input; the plan is then sized for either role.
                              The phase entry points and mpsm_join_batch use the default      */
  uint32_t run_buckets;    /* MPSM_RUNS_*: bucket function of the runs' first sort pass      */
  uint32_t reserved[2];    /* must be zero                                                   */
} mpsm_options_t;

/* Fills *opt with the defaults (all automatic, histogram splitters, binary search). */
int mpsm_options_default(mpsm_options_t* opt);

/* Creates a plan able to join up to max_nR R tuples with up to max_nS S tuples
 * (for mpsm_join_batch: the totals over all jobs, and at most max_jobs jobs).
 * The plan owns all scratch: about (max_nR + 2 max_nS) x 16 bytes plus small
 * tables.  `stream` is a cudaStream_t (NULL = the legacy default stream) on the
 * current device.  opt == NULL takes the defaults.  max_nR, max_nS < 2^32. */
int mpsm_plan_create(mpsm_plan_t** plan, uint64_t max_nR, uint64_t max_nS, uint32_t max_jobs,
                     const mpsm_options_t* opt, void* stream);

/* Frees the plan and its scratch (synchronises its stream first). */
void mpsm_plan_destroy(mpsm_plan_t* plan);

/* The whole join (phases 1-4).  R: nR tuples, S: nS tuples, device memory.
 * out_count / out_checksum: HOST pointers, written when the call returns.
 * opt_pairs: NULL, or a DEVICE buffer of capacity pairs; when the result has
 * more pairs than that, nothing is written to it, *out_count holds the required
 * capacity and the call returns MPSM_ERR_CAPACITY.  nR == 0 or nS == 0 give 0, 0. */
int mpsm_join(mpsm_plan_t* plan, const mpsm_tuple_t* R, uint64_t nR, const mpsm_tuple_t* S,
              uint64_t nS, uint64_t* out_count, uint64_t* out_checksum, mpsm_pairs_t* opt_pairs);

/* Same as mpsm_join with R and S in HOST memory (pinned memory copies fastest):
 * the plan copies them to device staging buffers (allocated on the first call)
 * and joins them there.  The run side is copied first and sorted while the
 * partitioned side is still on the host link.  When the partitioned side holds at
 * least 2^28 tuples (and no learned mode or MPSM_FLAG_UNFUSED is set), it is copied
 * in equal pieces of about a quarter of the run side, between 2^26 and 2^27 tuples
 * (larger once 64 pieces would not cover it), and each piece is range-partitioned,
 * sorted and joined against the sorted runs while the next one is in flight; the
 * result is the same, since the join sums over the pairs of each piece.
 * mpsm_plan_stats then describes the last piece's partitioning.
 * Synchronises the plan's stream. */
int mpsm_join_host(mpsm_plan_t* plan, const mpsm_tuple_t* R_host, uint64_t nR,
                   const mpsm_tuple_t* S_host, uint64_t nS, uint64_t* out_count,
                   uint64_t* out_checksum);

/* Host memory for mpsm_join_host's inputs (the paper has no counterpart: its inputs
 * start in memory).  Puts `bytes` (> 0) of zeroed, page-locked host memory in *out,
 * owned by the caller until mpsm_host_free.  It is an anonymous mapping advised for
 * transparent huge pages (Linux madvise MADV_HUGEPAGE, then MADV_POPULATE_WRITE and
 * MADV_COLLAPSE where the kernel has them) and registered with the CUDA driver
 * (cudaHostRegister).  A plain page-locked allocation made once host memory is
 * fragmented can hold regions that the host-to-device link reads at a tenth of its
 * rate; huge pages keep the whole buffer at the link's rate.  From one huge page up
 * (2 MiB under 4 KiB base pages, 512 MiB under 64 KiB ones) the mapping starts on a
 * huge-page boundary and spans whole huge pages, so up to one huge page more than
 * `bytes` is held.  Huge pages are advice: where host memory has just been fragmented
 * by other processes, part of the buffer can stay on base pages (a buffer made seconds
 * later usually gets huge pages throughout), and a kernel that splits underused huge
 * pages (Linux 6.12 and later) can split those of a buffer still all zeros when memory
 * runs short, so fill a buffer before making the next large one.  Where huge pages are unavailable the
 * memory is still page-locked, on base pages.  Errors:
 * MPSM_ERR_INVALID_ARG (null out, bytes == 0), MPSM_ERR_OOM (the mapping failed),
 * MPSM_ERR_CUDA (the registration failed; nothing stays allocated). */
int mpsm_host_alloc(uint64_t bytes, void** out);

/* Releases memory from mpsm_host_alloc (p and the same bytes); p == NULL is a no-op.
 * No copy from it may still be in flight.  MPSM_ERR_CUDA if the unregistration fails
 * (the mapping is released anyway). */
int mpsm_host_free(void* p, uint64_t bytes);

/* ---- phase entry points: mpsm_join == these five in order ---------------- */
/* They run the plain modes; on a plan created with a learned mode,
 * mpsm_sort_runs returns MPSM_ERR_INVALID_ARG. */

/* Phase 1 (Sec. 2.1, 3.2): R cut into T_R chunks [floor(j nR/T_R), floor((j+1) nR/T_R)),
 * each sorted by key into a run, kept in plan scratch (see mpsm_plan_view). */
int mpsm_sort_runs(mpsm_plan_t* plan, const mpsm_tuple_t* R, uint64_t nR);

/* Phase 2 (Sec. 3.2.1, 4.1-4.3): fine radix histograms of S over R's key range
 * (per S chunk = per worker), the run side's counts per fine bucket, the
 * cost-balanced splitters (fine bucket -> partition), and the prefix sums that
 * give every chunk its write position in every partition.  Needs phase 1. */
int mpsm_splitters(mpsm_plan_t* plan, const mpsm_tuple_t* S, uint64_t nS);

/* Phase 2, scatter (Sec. 4.3): every S tuple inside R's key range written to its
 * partition at its chunk's precomputed position; S tuples outside R's key range
 * cannot match and are dropped.  Needs mpsm_splitters. */
int mpsm_scatter(mpsm_plan_t* plan);

/* Phase 3: each S partition sorted by key.  Needs mpsm_scatter. */
int mpsm_sort_partitions(mpsm_plan_t* plan);

/* Phase 4, search (Sec. 3.2.2): for every S tile and R run, the run's window
 * [first key >= tile's first key, first key > tile's last key). Needs phase 3. */
int mpsm_search(mpsm_plan_t* plan);

/* Phase 4, merge join of every S tile against every run window; writes the
 * result like mpsm_join.  Needs mpsm_search. */
int mpsm_merge_join(mpsm_plan_t* plan, uint64_t* out_count, uint64_t* out_checksum,
                    mpsm_pairs_t* opt_pairs);

/* ---- batched joins -------------------------------------------------------- */

typedef struct {
  const mpsm_tuple_t* R; uint64_t nR;   /* device */
  const mpsm_tuple_t* S; uint64_t nS;   /* device */
} mpsm_job_t;

/* njobs independent joins in one launch sequence: all jobs' runs, partitions
 * and tiles are processed together by the same kernels, and the sequence is
 * captured once into a CUDA graph that later calls with the same job sizes
 * replay.  jobs: HOST array.  out_counts / out_checksums: HOST arrays of njobs. */
int mpsm_join_batch(mpsm_plan_t* plan, const mpsm_job_t* jobs, uint32_t njobs,
                    uint64_t* out_counts, uint64_t* out_checksums);

/* ---- tuning ------------------------------------------------------------------
 * The knobs the autotuner sets (0 = automatic, as in mpsm_options_t): the
 * largest radix fan-out (log2), S tuples per join tile, target R tuples per run,
 * and the number of S partitions. */
typedef struct {
  uint32_t radix_bits, join_tile, run_len, partitions_s;
} mpsm_tuning_t;

/* Replaces the plan's tunable options for later calls (invalid values:
 * MPSM_ERR_INVALID_ARG).  A captured batch graph is dropped. */
int mpsm_plan_set_tuning(mpsm_plan_t* plan, const mpsm_tuning_t* tuning);

/* Autotuner for batched joins (no counterpart in the paper): runs `jobs` through
 * mpsm_join_batch under each candidate tuning -- radix fan-out 2^9 or 2^11, join
 * tile 2048 or 4096, automatic runs or runs of about 2^23 tuples -- once to warm
 * up (capturing its graph) and `reps` times timed on the host clock, checks that
 * every candidate returns the same per-job results, and leaves the fastest set
 * on the plan.  Writes it to *best and its mean time per batch to *best_ms
 * (HOST).  Returns MPSM_ERR_DEVICE if two candidates disagree. */
int mpsm_autotune(mpsm_plan_t* plan, const mpsm_job_t* jobs, uint32_t njobs, uint32_t reps, mpsm_tuning_t* best,
                  float* best_ms);

/* ---- introspection --------------------------------------------------------- */

typedef struct {
  float ms_sort_runs, ms_splitters, ms_scatter, ms_sort_partitions, ms_search, ms_join, ms_learn;
  float ms_total;               /* per-phase device time of the last call (MPSM_FLAG_TIMING) */
  uint32_t runs_r;              /* T_R used                                                  */
  uint32_t partitions_s;        /* P used                                                    */
  uint32_t nfine, fine_shift;   /* fine histogram geometry                                   */
  uint64_t s_kept;              /* S tuples inside R's key range                             */
  uint64_t part_max;            /* largest partition                                         */
  double imbalance;             /* largest / mean partition size                             */
  double mean_window;           /* mean R tuples per (tile, run) window                      */
  uint64_t tiles;               /* S join tiles                                              */
  uint32_t levels_r, levels_s;  /* radix levels of phase 1 / phase 3 before the final sort   */
  uint64_t segments_r, segments_s; /* final in-shared-memory sort segments                   */
  uint32_t launches;            /* kernels launched by the last call                         */
  uint32_t pad;
  /* learned model (job 0; zero for the parts that ran in plain mode)                          */
  float loss_s0, loss_s;        /* S-side model: training loss (MSE of the CDF) at the first and */
  float loss_r0, loss_r;        /* the last Adam step; R-side model likewise                    */
  double part_probes;           /* boundary probes per partitioned S key (learned splitters)    */
  double search_probes;         /* probes per run-start search (binary or learned)              */
  double search_err;            /* mean |predicted - exact| run-start position (learned search) */
} mpsm_stats_t;

/* Statistics of the last join (job 0 of a batch).  Synchronises. */
int mpsm_plan_stats(mpsm_plan_t* plan, mpsm_stats_t* stats);

/* A final S segment of the fused path: `length` tuples at `offset` of the view's
 * s_buffer ((flags & 7) == 3) or pass_buffer ((flags & 7) == 4), every key in
 * [key_lo, key_hi] (the bounds its windows are searched for). */
typedef struct {
  uint64_t offset, length;
  uint64_t key_lo, key_hi;
  uint32_t job, flags;             /* the job; where the tuples are (bits 0-2) and internal flags */
} mpsm_segment_t;

typedef struct {
  const mpsm_tuple_t* r_runs;      /* device: nR tuples, the T_R sorted runs back to back      */
  const uint64_t* run_offsets;     /* device: T_R + 1 run boundaries                            */
  uint32_t runs_r;
  uint64_t key_min, key_max;       /* R's key range (valid when nR > 0)                         */
  uint32_t nfine, fine_shift;      /* fine bucket b = (key - key_min) >> fine_shift, b < nfine  */
  const uint64_t* fine_s;          /* device: nfine S counts                                    */
  const uint64_t* fine_r;          /* device: nfine R counts                                    */
  const uint32_t* splitters;       /* device: nfine entries, fine bucket -> partition            */
  uint32_t partitions_s;           /* P used                                                    */
  uint32_t s_chunks;               /* S chunks (workers) of phase 2                              */
  const uint64_t* s_chunk_offsets; /* device: s_chunks + 1 chunk boundaries in S                */
  const uint32_t* chunk_offsets;   /* device: s_chunks x P; ps_i[p], the s_buffer position where  */
                                   /* chunk i writes its first tuple of partition p (Sec. 3.2.1)  */
  const uint64_t* part_offsets;    /* device: P + 1 partition starts in s_buffer                 */
  const mpsm_tuple_t* s_buffer;    /* device: S after the last phase run (partitioned / sorted)  */
  uint64_t s_kept;
  uint64_t tiles;                  /* S tiles of phase 4                                         */
  uint32_t join_tile;              /* S tuples per tile (tile t = [t*join_tile, ...) of s_buffer) */
  const uint32_t* windows;         /* device: tiles x T_R x 2 (start, end) relative to the run    */
  /* the fused path (mpsm_join without pairs, Sec. 3.2 phases 3 and 4 in one pass): the final S
   * segments that its last pass sorted and joined in shared memory, and their windows */
  const mpsm_segment_t* segments;  /* device: n_segments records (order unspecified)             */
  uint32_t n_segments;
  uint32_t window_stride;          /* runs per row of seg_windows (>= T_R)                       */
  const uint32_t* seg_windows;     /* device: n_segments x window_stride x 2: for segment i and run
                                      j < T_R, [first position with key >= key_lo, first position
                                      with key > key_hi), relative to the run (Sec. 3.2.2)        */
  const mpsm_tuple_t* pass_buffer; /* device: the radix passes' ping-pong buffer                  */
} mpsm_view_t;

/* ---- learned CDF model (two-stage recursive model index) ----------------------
 * The learned modes (MPSM_SPLIT_LEARNED, MPSM_SEARCH_LEARNED) train, inside
 * every join, one model per job and side: a root MLP over the normalised key
 * (1 -> 32 -> 32 -> 1, ReLU, FP32 weights; Adam, 200 full-batch steps, learning
 * rate 3e-3, on up to 4096 evenly spaced points) and 4096 linear leaves (least squares on
 * the key's exact offset from the leaf's smallest key).  It stands in for the
 * paper's CDF of the runs (Sec. 4.1-4.2, Fig. 8): the S-side model is trained on
 * a sorted sample of S (1/64 of it, at most 2^21 keys) and its quantiles give
 * the partition boundaries; it predicts each S tuple's partition, which an exact
 * search over the boundaries then corrects (tuples of a key equal to several
 * boundaries spread over those partitions by a hash of their row).  The R-side
 * model is trained on positions of the sorted runs (exact ranks) and predicts
 * where each S tile's keys start in every run (Sec. 3.2.2), corrected by an
 * exponential then binary search.  Results are bit-identical to the plain modes.
 *
 * The entry points below run the same kernels on caller data, using model slot
 * 0 of the plan (slot 1 holds job 0's R-side model after a learned join).  All
 * pointers are DEVICE pointers unless marked HOST; x, y are FP32, n <= 4096
 * for the gradient and training calls.  The parameter vector theta has 1153
 * floats: W1[32], b1[32], W2[32][32] (row = output unit), b2[32], W3[32], b3. */

/* Loss (HOST *loss) = mean over i of (root(x_i) - y_i)^2 and its gradient (grad,
 * 1153 floats) at theta. */
int mpsm_rmi_loss_grad(mpsm_plan_t* plan, const float* x, const float* y, uint32_t n, const float* theta,
                       float* grad, float* loss);
/* `steps` full-batch Adam steps (beta 0.9 / 0.999, eps 1e-8) from theta, which is
 * updated in place; HOST losses[t] (may be NULL) = loss before step t + 1. */
int mpsm_rmi_train(mpsm_plan_t* plan, const float* x, const float* y, uint32_t n, uint32_t steps, float lr,
                   float* theta, float* losses);
/* Builds a whole model in slot 0 from n fit points (keys with their CDF values
 * y, n <= the plan's sample capacity): range [kmin, kmax], initial weights,
 * `steps` Adam steps on up to 4096 evenly spaced points, tabulation, leaves. */
int mpsm_rmi_fit(mpsm_plan_t* plan, const uint64_t* keys, const float* y, uint32_t n, uint64_t kmin, uint64_t kmax,
                 uint32_t steps, float lr);
/* Predicted CDF values (yhat, n floats) and leaves (leaf, n u32, may be NULL) of
 * `keys` under the model in `slot` (0 or 1). */
int mpsm_rmi_predict(mpsm_plan_t* plan, uint32_t slot, const uint64_t* keys, uint64_t n, float* yhat, uint32_t* leaf);

typedef struct {
  uint64_t kmin, kmax;          /* normalisation range                                       */
  uint32_t cshift, ncell;       /* cell = min((key - kmin) >> cshift, ncell - 1)             */
  uint32_t fit_n, train_n;      /* fit points, training points                               */
  float loss0, loss;            /* loss at the first and the last Adam step                  */
} mpsm_rmi_info_t;
/* Copies the model in `slot` to HOST buffers (each may be NULL): theta (1153
 * floats), cell_leaf (65536 u16: the tabulated root), leaf_base (4096 u64),
 * leaf_a, leaf_b (4096 floats each).  Synchronises. */
int mpsm_rmi_export(mpsm_plan_t* plan, uint32_t slot, mpsm_rmi_info_t* info, float* theta, uint16_t* cell_leaf,
                    uint64_t* leaf_base, float* leaf_a, float* leaf_b);

/* Replaces the plan's MPSM_FLAG_* flags (timing on/off) for later calls. */
int mpsm_plan_set_flags(mpsm_plan_t* plan, uint32_t flags);

typedef struct {
  char name[24];                /* kernel family, e.g. "scatter_split"                       */
  uint32_t launches;            /* launches in the last call                                 */
  float ms;                     /* summed device time of those launches (CUDA events)        */
} mpsm_kernel_time_t;

/* Per kernel family device time of the last call made with MPSM_FLAG_KERNEL_TIMING:
 * writes up to cap entries (families that launched) and their number to *n.
 * Synchronises. */
int mpsm_plan_kernel_times(mpsm_plan_t* plan, mpsm_kernel_time_t* out, uint32_t cap, uint32_t* n);

/* Device pointers into the plan's scratch after the last phase entry point
 * (valid until the next call on the plan).  Synchronises. */
int mpsm_plan_view(mpsm_plan_t* plan, mpsm_view_t* view);

const char* mpsm_strerror(int status);

/* ---- device-side checks -----------------------------------------------------
 * The paper has no counterpart.  Kernels never trap, assert or spin without end:
 * an invariant they find violated, an index they find out of bounds (the access
 * is skipped) or a wait that runs out (a bulk copy not complete after a bounded
 * number of polls of its shared-memory barrier) sets one of these bits, and the
 * call returns MPSM_ERR_DEVICE. */
enum {
  MPSM_DEVERR_LIST_OVERFLOW = 1u,   /* a segment work list ran out of capacity            */
  MPSM_DEVERR_SEGMENT_TOO_BIG = 2u, /* a final segment larger than a shared-memory sort    */
  MPSM_DEVERR_WAIT_TIMEOUT = 4u,    /* a bounded wait gave up                              */
  MPSM_DEVERR_LEVELS = 8u,          /* radix passes exhausted with big segments left       */
  MPSM_DEVERR_HIST_OVERFLOW = 16u,  /* a pass needed more histogram entries than allocated */
  MPSM_DEVERR_LEARN = 32u,          /* a learned-model invariant was violated              */
  MPSM_DEVERR_BOUNDS = 64u          /* an index check inside a kernel failed               */
};

/* The MPSM_DEVERR_* bits of the plan's last call that returned MPSM_ERR_DEVICE,
 * 0 after a call that did not (HOST). */
int mpsm_plan_device_errors(const mpsm_plan_t* plan, uint32_t* flags);

/* Self-test of the bounded waits, on `cuda_stream` (NULL = the default stream): one
 * block waits on a shared-memory barrier that nothing will complete, gives up
 * after spin_limit polls (0 = 1000), sets MPSM_DEVERR_WAIT_TIMEOUT and returns.
 * Returns MPSM_ERR_DEVICE with *flags = MPSM_DEVERR_WAIT_TIMEOUT; the CUDA context
 * stays usable.  Allocates and frees 4 bytes of device memory.  Synchronises. */
int mpsm_selftest_wait_timeout(void* cuda_stream, uint32_t spin_limit, uint32_t* flags);

/* Self-test of the splitter cost's logarithm.  Sec. 4.3 charges a partition of n
 * tuples n log n for its sort; the library evaluates that term as
 * n * floor(2^16 log2 n) in integers, so its splitters are reproducible bit for
 * bit.  For each of the `count` values n[i] (DEVICE array of uint64, 8-byte
 * aligned) this writes out[i] (DEVICE, count values) = floor(2^16 log2 n[i]), 0 for
 * n[i] <= 1, computed exactly as k_splitters computes it.  wide != 0 takes the
 * 126-bit path for every value (the library itself takes it only when the 62-bit
 * path cannot decide a bit); UINT64_MAX marks a value that the path used could not
 * decide.  Runs on cuda_stream (NULL = the default stream) and synchronises it.
 * Returns MPSM_ERR_INVALID_ARG for null or misaligned arrays. */
int mpsm_selftest_log2_q16(const uint64_t* n, uint64_t count, uint64_t* out, uint32_t wide, void* cuda_stream);

/* ---- allocation-free run sort ------------------------------------------------
 * The paper has no counterpart: this entry point exists for callers that must
 * not allocate device memory -- code that runs under a memory pool owned by
 * someone else (a framework's caching allocator, a fixed budget), or on a path
 * where cudaMalloc's implicit device-wide synchronisation is not acceptable.
 * It does phase 1 alone for a small input: R (nR tuples, device) is cut into
 * `runs` chunks [floor(j nR/runs), floor((j+1) nR/runs)) exactly like
 * mpsm_sort_runs, and each chunk is sorted by key into `out` (device, nR
 * tuples; may equal R) at the same positions.  No plan is needed and nothing is
 * allocated: the scratch lives in one fixed device array of about 41 KB inside
 * the library, which every GPU that loads the library keeps until exit.
 * Limits: 1 <= runs <= 1024 and every run at most 8192 tuples
 * (ceil(nR / runs) <= 8192); larger sizes return MPSM_ERR_INVALID_ARG.  Pointers
 * must be 16-byte aligned.  Work goes on `stream` (a cudaStream_t, NULL = legacy
 * default stream); every call reads its error flag back and synchronises that
 * stream before returning, so no call of it can be made inside a stream capture.
 * The first call on a device also looks up the array's address and sets kernel
 * attributes.  Every call shares the array: calls
 * whose work overlaps on the GPU (other streams, other host threads) race. */
int mpsm_sort_runs_noalloc(const mpsm_tuple_t* R, uint64_t nR, uint32_t runs, mpsm_tuple_t* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MPSM_H */
