/*
 * dtsort -- stable MSD integer sort with heavy-key detection and dovetail
 * merging, for NVIDIA GB300 (sm_103a).
 *
 * The operation (Sec. 2.3 of "Parallel Integer Sort: Theory and Practice",
 * Dong, Dhulipala, Gu, Sun, PPoPP'24): n records with unsigned integer keys
 * in [0, 2^w) are reordered into non-decreasing key order, STABLY (records
 * with equal keys keep their input order).  The result is written back into
 * the input arrays ("in place" refers to the interface; O(n) extra space is
 * used, passed in as a caller-owned workspace).  The method is DovetailSort
 * (Alg. 2): per subproblem, sample the keys and detect heavy (highly
 * duplicated) keys, distribute records into light buckets (one per MSD zone)
 * and heavy buckets (one per heavy key) with a stable counting sort, recurse
 * on light buckets only, and merge each zone's light and heavy runs (Alg. 3,
 * DTMerge).  A stable sort's output is unique, so every parameter below
 * (digit width, tile size, sample size, on-chip capacity, learned bucketing)
 * changes speed only, never the output.
 *
 * Conventions for every call:
 *   - Pointers named keys/values/offsets/workspace are DEVICE pointers on the
 *     handle's device.  The caller owns them; the library never frees them or
 *     keeps them after the call has been enqueued.  Keys and values are two
 *     separate arrays (structure of arrays); values == NULL means key-only.
 *     Values are opaque payload of the key's width, copied bit for bit.
 *   - Keys compare as unsigned integers.
 *   - Calls are asynchronous and stream-ordered on `stream` (a cudaStream_t;
 *     NULL is the legacy default stream).  The return value reports only what
 *     the host can check before launching.  Errors found on the device (a
 *     bounded wait that timed out, an exhausted internal table) are latched
 *     in the handle and read with dtsort_last_device_error().
 *   - No call allocates device memory, except dtsort_create() (a few KB) and
 *     the first sort with launch_mode 1 (a pinned host copy of a few KB).
 *   - n == 0 is a no-op returning DTSORT_OK; n >= 2^32 returns
 *     DTSORT_ERR_UNSUPPORTED.  n < 0, or a NULL pointer where
 *     n > 0 needs one, returns DTSORT_ERR_INVALID_ARG.  A workspace smaller
 *     than dtsort_workspace_bytes() returns DTSORT_ERR_WORKSPACE_TOO_SMALL.
 *     Keys/values must be aligned to their own width; the workspace to 256 B.
 *   - A handle is used by one host thread at a time.  Two sorts that use the
 *     same workspace must not overlap on the GPU.
 */
#ifndef DTSORT_H_
#define DTSORT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define DTSORT_API __attribute__((visibility("default")))
#else
#define DTSORT_API
#endif

/* Same type as cudaStream_t; declared here so that no CUDA header is needed. */
typedef struct CUstream_st *dtsort_stream;

typedef enum {
  DTSORT_OK = 0,
  DTSORT_ERR_INVALID_ARG = 1,
  DTSORT_ERR_WORKSPACE_TOO_SMALL = 2,
  DTSORT_ERR_CUDA = 3,             /* a CUDA runtime call failed */
  DTSORT_ERR_DEVICE_TIMEOUT = 4,   /* a bounded device-side wait expired */
  DTSORT_ERR_UNSUPPORTED = 5,      /* e.g. no sm_103a device */
  DTSORT_ERR_INTERNAL = 6          /* an internal device table overflowed */
} dtsort_status;

typedef enum {
  DTSORT_OP_U32 = 0,     /* 32-bit keys, key-only */
  DTSORT_OP_U32_KV = 1,  /* 32-bit keys, 32-bit values */
  DTSORT_OP_U64 = 2,     /* 64-bit keys, key-only */
  DTSORT_OP_U64_KV = 3   /* 64-bit keys, 64-bit values */
} dtsort_op;

typedef enum {
  DTSORT_BUCKETING_DIGIT = 0,   /* MSD zones = the next gamma key bits (Alg. 2) */
  DTSORT_BUCKETING_LEARNED = 1, /* zones from a CDF model fit on a sample, when a
                                   cost estimate from the sorted sample says they
                                   save more distribution passes than they cost;
                                   digit zones otherwise (decided on the device) */
  DTSORT_BUCKETING_LEARNED_ALWAYS = 2  /* the learned zones without the estimate */
} dtsort_bucketing;

/* Merging of a zone's sorted light bucket with its heavy buckets (Sec. 4).
 * Both give the same output. */
typedef enum {
  DTSORT_MERGE_DOVETAIL = 0, /* Alg. 3: every record's position in closed
                                form from the heavy buckets' sizes and one
                                binary search per heavy key; no key compares */
  DTSORT_MERGE_GENERIC = 1   /* a generic stable merge of the light bucket
                                with the heavy buckets' concatenation: merge
                                path, splitters found by key comparisons (the
                                paper's comparison against a standard
                                parallel merge) */
} dtsort_merge;

typedef struct dtsort_handle_s *dtsort_handle;

/* Tuning knobs.  Zero fields mean "default" (or "autotuned" where autotune is
 * on).  None of them changes the output. */
typedef struct {
  int32_t gamma_max;         /* largest digit width per level, 1..9 (default 9) */
  int32_t finisher_capacity; /* largest bucket the on-chip base case sorts,
                                in records (default: what fits on chip) */
  int32_t heavy_detection;   /* 1 on (default), -1 off (the paper's "Plain") */
  int32_t bucketing;         /* dtsort_bucketing (default DIGIT) */
  uint64_t seed;             /* sampler seed (default 1) */
  int32_t sample_log_factor; /* samples per level = 2^gamma * ceil(log2 n),
                                capped on chip; 0 = default */
  int32_t autotune;          /* 1: use the on-disk autotune cache (default 0) */
  int32_t learned_segments;  /* learned bucketing: knots of the CDF table
                                (default 1024) */
  int32_t learned_train_steps; /* learned bucketing: Adam steps (default 200) */
  int32_t wait_limit_ms;     /* bound of every device-side wait (default 2000);
                                when it expires the sort latches
                                DTSORT_ERR_DEVICE_TIMEOUT and writes nothing more */
  int32_t debug_fault;       /* testing only: 1 = the second look-back chunk of
                                the first distribution never publishes its
                                status, so its successors' waits expire */
  int32_t launch_mode;       /* 0 (default): the levels a uniformly
                                distributed input of n keys needs (n = the
                                total for a segmented call, which bounds every
                                array), and from 2^26 records on two more,
                                run as one launch per phase, queued
                                without host synchronisation (each phase checks
                                on the device whether it has work), then one
                                persistent cooperative launch takes any further
                                levels and the merges.  No host
                                synchronisation; capturable in a CUDA graph.
                                1: one launch per phase with the level loop on
                                the host (a profiling aid: every phase appears
                                as its own kernel; synchronises the stream).
                                2: the persistent launch alone. */
  int32_t block_tiles;       /* rows of the per-level count matrix cover
                                block_tiles tiles of the scatter (8K 32-bit or
                                4K 64-bit keys each); 1..8, default 8 */
  int32_t merge;             /* dtsort_merge: how each heavy zone's runs are
                                merged (default DOVETAIL) */
  int32_t heavy_min_share;   /* heavy keys are kept for a subproblem only when
                                they hold at least this many thousandths of its
                                sample (default 250; -1: any share).  Below
                                it the subproblem is distributed by its digit
                                alone, and deeper levels, where those keys
                                hold more of their smaller subproblems,
                                detect them */
  int32_t reserved[2];
} dtsort_options;

/* Statistics of the last completed sort on this handle (read after sync). */
typedef struct {
  int32_t levels;                 /* distribution levels executed */
  int32_t status;                 /* latched device status (dtsort_status) */
  int64_t segments[16];           /* subproblems distributed at level l */
  int64_t records[16];            /* records distributed at level l */
  int64_t heavy_keys[16];         /* heavy keys detected at level l */
  int64_t heavy_records[16];      /* records placed in heavy buckets at level l */
  int64_t overflow_records[16];   /* records in overflow buckets at level l */
  int64_t finisher_tasks;         /* buckets sorted by the on-chip base case */
  int64_t finisher_records;
  int64_t copy_records;           /* records moved by plain copies */
  int64_t merge_zones;            /* MSD zones that needed a dovetail merge */
  int64_t merge_records;          /* records written by dovetail merges */
  int64_t learned_fixup_records;  /* learned bucketing: records whose predicted
                                     bucket needed the exact fix-up */
  int64_t learned_fixup_steps;
  double learned_bucket_cv;       /* coefficient of variation of the level-0
                                     light bucket sizes (digit or learned
                                     zones; single-array sorts) */
  double learned_bucket_max_over_mean; /* largest / mean of the same */
  double phase_ms[8];             /* device time per phase kind: 0 setup,
                                     1 sample, 2 histogram, 3 scan, 4 scatter,
                                     5 finisher, 6 merge, 7 total */
  int64_t check_site;             /* first failed internal consistency check
                                     (0: none); the call then returned
                                     DTSORT_ERR_INTERNAL */
  int64_t check_values[2];        /* the two values that failed it */
  int64_t finisher_lsd_tasks;     /* base-case buckets that needed the LSD
                                     passes (a one-pass bin held too many
                                     equal-prefix keys) */
  int64_t kernel_launches;        /* kernels the last sort call launched
                                     (host count; memsets not included) */
  int64_t learned_zones_used;     /* 1: level 0 used learned zones; 0: digit
                                     zones (bucketing DIGIT, or LEARNED whose
                                     estimate chose digits) */
  double learned_estimate[2];     /* LEARNED: estimated record-passes below
                                     level 0 with digit zones, and with learned
                                     zones plus their extra cost */
  int64_t merge_free_zones;       /* MSD zones with heavy keys whose runs were
                                     already in key order (heavy keys below and
                                     above all of the zone's light keys): no
                                     merge */
} dtsort_stats;

DTSORT_API const char *dtsort_status_string(dtsort_status s);

/* Creates a handle on CUDA device `device`.  Allocates its small state
 * (status word, statistics, timing) on that device.  Fails with
 * DTSORT_ERR_UNSUPPORTED when the device is not compute capability 10.3. */
DTSORT_API dtsort_status dtsort_create(dtsort_handle *out, int device);
DTSORT_API dtsort_status dtsort_destroy(dtsort_handle h);

/* Fills *opt with the defaults. */
DTSORT_API dtsort_status dtsort_default_options(dtsort_options *opt);
/* opt == NULL restores the defaults.  Invalid values -> INVALID_ARG. */
DTSORT_API dtsort_status dtsort_set_options(dtsort_handle h, const dtsort_options *opt);
DTSORT_API dtsort_status dtsort_get_options(dtsort_handle h, dtsort_options *opt);

/* Workspace size in bytes for sorting n records (num_segments arrays for the
 * segmented calls, 1 otherwise) with the handle's current options.  The
 * workspace holds the second (ping-pong) copy of keys and values and the
 * per-level tables; it is about n * (key + value bytes) * 1.1 + 4 MB. */
DTSORT_API dtsort_status dtsort_workspace_bytes(dtsort_handle h, dtsort_op op, int64_t n,
                                     int64_t num_segments, size_t *bytes);

/* Stable sort of keys[0..n) (and values[0..n) alongside) in place. */
DTSORT_API dtsort_status dtsort_u32(dtsort_handle h, uint32_t *keys, int64_t n,
                         void *workspace, size_t workspace_bytes,
                         dtsort_stream stream);
DTSORT_API dtsort_status dtsort_u32_kv(dtsort_handle h, uint32_t *keys, uint32_t *values,
                            int64_t n, void *workspace, size_t workspace_bytes,
                            dtsort_stream stream);
DTSORT_API dtsort_status dtsort_u64(dtsort_handle h, uint64_t *keys, int64_t n,
                         void *workspace, size_t workspace_bytes,
                         dtsort_stream stream);
DTSORT_API dtsort_status dtsort_u64_kv(dtsort_handle h, uint64_t *keys, uint64_t *values,
                            int64_t n, void *workspace, size_t workspace_bytes,
                            dtsort_stream stream);

/* The same sort for records in HOST memory (Sec. 2's problem on host
 * buffers): copies the n keys (and values, if op has values) from keys_host /
 * values_host into the caller's DEVICE buffers dev_keys / dev_values, sorts
 * them there exactly as dtsort_u32 ... dtsort_u64_kv, and copies the result
 * back over the host arrays.  All three steps are enqueued on `stream`; the
 * host arrays hold the result once the stream has reached this point (host
 * memory should be pinned, e.g. cudaHostAlloc, for the copies to be
 * asynchronous; pageable memory works but the copies then synchronise).
 * values_host / dev_values must be NULL for a key-only op.  No allocation.
 * Errors: as the device entry points; DTSORT_ERR_CUDA if a copy cannot be
 * enqueued.  (The paper has no counterpart: it sorts in host memory.) */
DTSORT_API dtsort_status dtsort_sort_host(dtsort_handle h, dtsort_op op, void *keys_host,
                              void *values_host, int64_t n, void *dev_keys,
                              void *dev_values, void *workspace,
                              size_t workspace_bytes, dtsort_stream stream);

/* Segmented (batched) stable sort: every array s = [offsets[s], offsets[s+1])
 * of keys/values is sorted on its own, all in one persistent kernel launch.
 * offsets: DEVICE int64[num_segments + 1], offsets[0] == 0, non-decreasing,
 * offsets[num_segments] == n (not checked on the host; a violation is
 * reported as DTSORT_ERR_INVALID_ARG by dtsort_last_device_error()).  Empty
 * arrays are allowed.  The launch sequence contains no host synchronisation,
 * so it can be captured into a CUDA graph once the sizes are fixed. */
DTSORT_API dtsort_status dtsort_segmented_u32(dtsort_handle h, uint32_t *keys,
                                   const int64_t *offsets, int64_t num_segments,
                                   int64_t n, void *workspace,
                                   size_t workspace_bytes, dtsort_stream stream);
DTSORT_API dtsort_status dtsort_segmented_u32_kv(dtsort_handle h, uint32_t *keys,
                                      uint32_t *values, const int64_t *offsets,
                                      int64_t num_segments, int64_t n,
                                      void *workspace, size_t workspace_bytes,
                                      dtsort_stream stream);
DTSORT_API dtsort_status dtsort_segmented_u64(dtsort_handle h, uint64_t *keys,
                                   const int64_t *offsets, int64_t num_segments,
                                   int64_t n, void *workspace,
                                   size_t workspace_bytes, dtsort_stream stream);
DTSORT_API dtsort_status dtsort_segmented_u64_kv(dtsort_handle h, uint64_t *keys,
                                      uint64_t *values, const int64_t *offsets,
                                      int64_t num_segments, int64_t n,
                                      void *workspace, size_t workspace_bytes,
                                      dtsort_stream stream);

/* Synchronises `stream` and returns the device status latched by the sorts
 * enqueued on this handle since the previous call (then clears it). */
DTSORT_API dtsort_status dtsort_last_device_error(dtsort_handle h, dtsort_stream stream);

/* Copies the statistics of the most recent sort (synchronises the device). */
DTSORT_API dtsort_status dtsort_get_stats(dtsort_handle h, dtsort_stats *out);

/* ---- learned bucketing: the model's kernels ---------------------------------
 * The paper has no learned component.  With options.bucketing = LEARNED, a
 * single-array sort of n >= 2^20 keys first fits a CDF model on about 1% of
 * the keys (sampled, sorted, features x = log2(1 + key) / key_bits, targets
 * (i + 0.5) / m), trained by Adam on the GPU; the model's inverse gives the
 * level-0 zone boundaries, and each key's zone is predicted from the model and
 * then fixed up exactly by integer comparison with the boundaries.  The
 * output is the same as with digit zones.
 *
 * The model is a 1 -> 16 -> 16 -> 1 MLP with tanh hidden layers: 321 fp32
 * parameters laid out W1[16] b1[16] W2[16][16] (row j, column k multiplies
 * hidden unit k) b2[16] W3[16] b3.  These entry points run its kernels on
 * given data (all pointers DEVICE); they need no handle.
 *
 * dtsort_mlp_forward: y[i] = F(x[i]).
 * dtsort_mlp_grad:    grad_out[0..321) = gradient of (1/n) sum (F(x_i)-t_i)^2
 *                     over the parameters, grad_out[321] = that loss
 *                     (322 floats); partial: ceil(n/256) * 322 floats of
 *                     scratch.  Sums run in a fixed order (deterministic).
 * dtsort_mlp_adam:    one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at step
 *                     number `step` >= 1 on params, moments m, v (321 each)
 *                     with the gradient grad (322 floats as above).
 * dtsort_mlp_train:   `steps` Adam steps on batches of `batch` points; batch
 *                     k uses points ((k-1) mod S) + i*S, S = n / batch;
 *                     partial: ceil(batch/256) * 322 floats. */
DTSORT_API dtsort_status dtsort_mlp_forward(const float *params, const float *x, int64_t n,
                                            float *y, dtsort_stream stream);
DTSORT_API dtsort_status dtsort_mlp_grad(const float *params, const float *x, const float *t,
                                         int64_t n, float *partial, float *grad_out,
                                         dtsort_stream stream);
DTSORT_API dtsort_status dtsort_mlp_adam(float *params, float *m, float *v, const float *grad,
                                         int step, float lr, dtsort_stream stream);
DTSORT_API dtsort_status dtsort_mlp_train(float *params, float *m, float *v, const float *x,
                                          const float *t, int64_t n, int steps, int batch,
                                          float lr, float *partial, dtsort_stream stream);

/* ---- autotuning ------------------------------------------------------------
 * Picks the tuning knobs (digit width limit, base-case capacity, count-matrix
 * block size) for one problem class; the output never depends on them.  Each
 * candidate setting sorts a private copy of keys/values (+offsets) placed in
 * `scratch` (DEVICE, at least dtsort_autotune_scratch_bytes(), 256-byte
 * aligned); the caller's arrays are only read.  The fastest setting is
 * stored in the handle's options and written to the on-disk cache (the file
 * named by the environment variable DTSORT_AUTOTUNE_CACHE, else
 * $HOME/.cache/dtsort_autotune.tsv), keyed by (GPU name, op, floor(log2 n),
 * floor(log2 num_segments)).  Sorts on a handle whose options have
 * autotune = 1 use the cached setting of their class when there is one.
 * Synchronises `stream`.  best_out (optional) receives the chosen options. */
DTSORT_API dtsort_status dtsort_autotune_scratch_bytes(dtsort_handle h, dtsort_op op, int64_t n,
                                                       int64_t num_segments, size_t *bytes);
DTSORT_API dtsort_status dtsort_autotune(dtsort_handle h, dtsort_op op, const void *keys,
                                         const void *values, const int64_t *offsets,
                                         int64_t num_segments, int64_t n, void *scratch,
                                         size_t scratch_bytes, dtsort_stream stream,
                                         dtsort_options *best_out);

/* ---- sorting an array sharded over several GPUs ----------------------------
 * The rank-local steps of a sort with one exchange (no counterpart in the
 * paper's single-machine setting; it applies the distribution step of the
 * paper's counting sort (Sec. 2 preliminaries, "Counting Sort"; Alg. 2 step
 * 2) with one bucket per rank).  P ranks hold contiguous, index-ordered
 * shards of one array: rank r holds global records [gidx0_r, gidx0_r + n_r).
 * The stable order of the array is the order of the pairs (key, global
 * index) (Sec. 2.3), so:
 *   1. every rank draws a sample of such pairs (dtsort_shard_sample); the
 *      caller gathers all samples on every rank;
 *   2. dtsort_shard_splitters picks P-1 splitters from the gathered sample;
 *   3. every rank partitions its shard stably into P consecutive ranges,
 *      range p = the records with p splitters <= (key, global index)
 *      (dtsort_shard_partition); a key duplicated across a splitter is split
 *      by global index, which keeps the ranges balanced;
 *   4. the caller exchanges the ranges with one all-to-all (range p to rank
 *      p, received runs concatenated in source-rank order, i.e. in global
 *      index order);
 *   5. rank p sorts what it received with dtsort_u32[_kv]/dtsort_u64[_kv]
 *      and then holds the p-th consecutive part of the sorted array.
 * Keys compare as unsigned; 32-bit keys are widened to 64 bits in samples
 * and splitters. */
#define DTSORT_SHARD_MAX_PARTS 64

/* Draws `count` samples of the shard keys[0..n_local) (device, key_bytes 4 or
 * 8), uniformly with replacement: sample i is the record at position
 * x_i mod n_local, x_i the i-th output of SplitMix64 (Steele, Lea, Flood
 * 2014) started from seed ^ fmix64(gidx0 + 0x9E3779B97F4A7C15).  Writes its
 * key (widened to 64 bits) to sample_keys[i] and gidx0 + position to
 * sample_gidx[i] (device arrays, 8-byte aligned).  count = 0 is a no-op;
 * count > 0 needs n_local > 0.  Stream-ordered; INVALID_ARG on bad
 * arguments, DTSORT_ERR_CUDA if the launch fails. */
DTSORT_API dtsort_status dtsort_shard_sample(const void *keys, int key_bytes, int64_t n_local,
                                             int64_t gidx0, uint64_t seed, int64_t count,
                                             uint64_t *sample_keys, int64_t *sample_gidx,
                                             dtsort_stream stream);

/* Host only (no device, no stream): sorts the m gathered sample pairs
 * (sample_keys[i], sample_gidx[i]) (host arrays) and writes splitter j-1 =
 * the pair of rank floor(j m / parts), j = 1..parts-1, into split_keys /
 * split_gidx (host arrays of parts-1 entries, increasing).  With m = 0 every
 * splitter is (2^64-1, INT64_MAX): all records fall into range 0.
 * parts in [1, DTSORT_SHARD_MAX_PARTS]. */
DTSORT_API dtsort_status dtsort_shard_splitters(const uint64_t *sample_keys,
                                                const int64_t *sample_gidx, int64_t m, int parts,
                                                uint64_t *split_keys, int64_t *split_gidx);

/* Workspace of dtsort_shard_partition for n_local records and `parts`
 * ranges (256 + 8 * rows * parts bytes, rows <= 4096). */
DTSORT_API dtsort_status dtsort_shard_partition_workspace_bytes(int64_t n_local, int parts,
                                                                size_t *bytes);

/* Stable partition of the shard keys/values[0..n_local) (device; values NULL
 * for key-only; record i has global index gidx0 + i) into `parts`
 * consecutive ranges of out_keys/out_values (device, n_local records, not
 * overlapping the input): range p holds, in index order, the records with
 * exactly p of the splitters (split_keys[j], split_gidx[j]) (device, parts-1
 * increasing pairs) <= (key, gidx0 + i).  counts (device int64[parts])
 * receives each range's size.  ws: device, 256-byte aligned, at least
 * dtsort_shard_partition_workspace_bytes.  device_status (optional, device
 * int32): cleared, then set to DTSORT_ERR_INTERNAL if a self-check finds a
 * slot outside the shard (nothing is written there); NULL: kept in the
 * workspace, not observable.  Pointers aligned to the key width.
 * Stream-ordered; INVALID_ARG / WORKSPACE_TOO_SMALL / DTSORT_ERR_CUDA. */
DTSORT_API dtsort_status dtsort_shard_partition(const void *keys, const void *values,
                                                int key_bytes, int64_t n_local, int64_t gidx0,
                                                const uint64_t *split_keys,
                                                const int64_t *split_gidx, int parts,
                                                void *out_keys, void *out_values,
                                                int64_t *counts, void *ws, size_t ws_bytes,
                                                int32_t *device_status, dtsort_stream stream);

/* ---- sorting without any allocation ---------------------------------------
 * The paper has no counterpart of this entry point.  It serves callers that
 * may not allocate device memory at call time and cannot provide a workspace
 * either: plugin or callback code that gets a stream from a host framework
 * owning all device memory, real-time pipelines that forbid allocation after
 * start-up.
 *
 * Same operation as dtsort_u32_kv (stable sort of keys[0..n) with values
 * alongside, in place, default options), but every temporary lives in one
 * static device array of 12 MiB inside this library, which each GPU that
 * loads the library holds until the process exits; no cudaMalloc/cudaFree
 * and no allocating library routine is called.  n must not exceed
 * DTSORT_NOALLOC_MAX_N (larger n returns DTSORT_ERR_INVALID_ARG without
 * launching).  keys/values: device pointers on the current device, 4-byte
 * aligned.  device_status: optional device int32 the sort latches its device
 * status into (0 = OK; cleared at the start of the call).  With NULL the
 * status goes to a word inside the static array that the next call clears:
 * a device-side failure (a bounded wait that ran out, a failed self-check,
 * both leaving the records unsorted) then cannot be observed, so pass a
 * word whenever the result matters.
 * The first call on a device performs a one-time set-up on that device
 * (looks up the array's device address, sets the kernel's shared-memory
 * limit); make that first call before any stream capture.  All calls share
 * the one array (it keeps the last call's contents; the call clears what must
 * start at zero), so calls that overlap on the GPU race with each other:
 * order them on one stream. */
#define DTSORT_NOALLOC_MAX_N ((int64_t)1 << 20)
DTSORT_API dtsort_status dtsort_u32_kv_noalloc(uint32_t *keys, uint32_t *values, int64_t n,
                                               int32_t *device_status, dtsort_stream stream);

/* ---- diagnostics: single steps of the method, for testing ---------------- */

/* Alg. 2 step 1 on one subproblem keys[start .. start+size) of an array whose
 * original length is n_total: draws `count` sample keys at positions
 * start + (SplitMix64 output i mod size), where output i comes from the
 * SplitMix64 sequence (Steele, Lea, Flood 2014) started from
 *   seed ^ start ^ (size * 0x9E3779B97F4A7C15) ^ (hi << 57),
 * sorts them, keeps every L-th (S[L-1], S[2L-1], ...), and reports the keys
 * seen at least twice there (heavy keys, increasing) and the largest sample.
 * heavy_out: DEVICE uint64[count / 2 + 1]; nheavy_out, max_out: DEVICE.
 * count <= 8192.  key_bytes is 4 or 8. */
DTSORT_API dtsort_status dtsort_debug_sample(dtsort_handle h, const void *keys,
                                  int key_bytes, int64_t start, int64_t size,
                                  int hi, uint64_t seed, int64_t count,
                                  int64_t L, uint64_t *heavy_out,
                                  int64_t *nheavy_out, uint64_t *max_out,
                                  dtsort_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* DTSORT_H_ */
