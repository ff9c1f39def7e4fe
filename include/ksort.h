/*
 * libksort: K-sort on one GB300 GPU (CUDA, sm_103a), behind a plain C ABI.
 *
 * K-sort (Sundararajan, Pal, Chakraborty, Mahanti, arxiv 1107.3622, Section 1.1) is
 * the interchange-free Quick sort whose partition (Steps 1-4) takes the FIRST element
 * of a sub-array as the key, sends every element x with key <= x to the right of the
 * key and every other element to its left, and writes the key at its final index
 * i = left + #{x < key}; Steps 5-6 then sort the two sides the same way.
 *
 * Conventions for every entry point:
 *   - Pointers named *_dev are device pointers on the calling thread's current CUDA
 *     device; they must be aligned to the key size. The caller owns them.
 *   - Calls are asynchronous on `stream` (NULL = the legacy default stream) and return
 *     once the work is enqueued. Errors found on the host (bad pointer, size, dtype)
 *     return at once and enqueue nothing.
 *   - Errors found on the device (bad offsets, exhausted workspace, a wait that ran
 *     past its time limit) set a flag that ksort_get_device_error() reads. No kernel
 *     traps, asserts or spins without a bound.
 *   - Each (device, stream) pair owns a private workspace (scratch keys, work queue,
 *     look-back descriptors) that the library allocates on first use and grows as
 *     needed. Calls on the same stream are ordered; calls on different streams use
 *     different workspaces and may overlap. Growing a workspace is not allowed while
 *     the stream is being captured into a CUDA graph: reserve it first with
 *     ksort_reserve_workspace().
 *   - Float keys compare with IEEE `<=` (Step 3). A NaN is never >= the key, so it goes
 *     left; a NaN key sends every element left. +0 and -0 compare equal.
 *   - A single sub-array may hold at most 2^31 - 1 keys.
 */
#ifndef KSORT_H
#define KSORT_H

#include <stdint.h>

#if defined(__GNUC__)
#define KSORT_API __attribute__((visibility("default")))
#else
#define KSORT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st *ksort_stream_t;

typedef enum { KSORT_F32 = 0, KSORT_F64 = 1, KSORT_U32 = 2 } ksort_dtype_t;

typedef enum {
    KSORT_OK = 0,
    KSORT_ERR_INVALID_ARG = 1,        /* NULL/misaligned/host pointer, bad size       */
    KSORT_ERR_UNSUPPORTED_DTYPE = 2,
    KSORT_ERR_OUT_OF_MEMORY = 3,      /* workspace could not be allocated or grown    */
    KSORT_ERR_CUDA = 4,               /* a CUDA runtime call failed                   */
    KSORT_ERR_TIMEOUT = 5,            /* device: a bounded wait ran past its limit     */
    KSORT_ERR_BAD_OFFSETS = 6,        /* device: offsets decrease, leave [0, total],
                                         or one array exceeds 2^31 - 1 keys           */
    KSORT_ERR_WORKSPACE_EXHAUSTED = 7,/* device: the work queue or look-back arena was
                                         too small (adversarial, near-O(n^2) inputs)   */
    KSORT_ERR_INTERNAL = 8,
    KSORT_ERR_TOO_LARGE = 9           /* n above KSORT_NOALLOC_MAX_KEYS (the fixed
                                         scratch of ksort_partition_out_noalloc)      */
} ksort_status_t;

/* Steps 1-4 once, in place, on keys_dev[0..n-1] (Section 1.1, Steps 1-4).
 * After the call keys[0..i) < key, keys[i] == key (the original keys[0]) and
 * keys(i..n) >= key, with i = #{x in keys[1..n) : x < key}. The order inside each side
 * is not the paper's (only the index and the two multisets are defined).
 * *key_index_dev (device int64) receives i. n >= 1. */
KSORT_API ksort_status_t ksort_partition(ksort_dtype_t dtype, void *keys_dev, int64_t n,
                               int64_t *key_index_dev, ksort_stream_t stream);

/* The same partition, out of place: in_dev is read, out_dev (n keys, not overlapping
 * in_dev) receives the partitioned keys. The default form (the tuning's partition_form
 * 1-4, see ksort_partition_shape) is one launch that reads and writes every key once:
 * CTAs claim tiles in ascending order and stage them into shared memory by bulk copies;
 * data warps compact each tile there (less keys from the front, >= keys from the back)
 * and publish its less count; one warp per CTA adds, to the CTA's own running count, the
 * counts of the tiles that other CTAs claimed in between, which gives the tile's global
 * offsets; the data warps then write both runs with 128-bit stores.
 * With partition_form -1 the form follows tile_shape instead. Tile shapes 1-9: one launch
 * (CTAs take the tiles round-robin and chain their less counts by decoupled look-back).
 * Tile shapes 10-12 (the wave form): two launches with no waits between CTAs: every warp
 * counts the less keys of its run of warp tiles, then (under programmatic dependent
 * launch) moves them with the prefix of those counts; the keys are read twice. The order
 * within each side differs between forms, the key index and the two sides' contents do
 * not. */
KSORT_API ksort_status_t ksort_partition_out(ksort_dtype_t dtype, const void *in_dev, void *out_dev,
                                   int64_t n, int64_t *key_index_dev, ksort_stream_t stream);

/* Steps 1-4 once, out of place, in the paper's own element order (Section 1.1, Steps 1-4):
 * out_dev receives exactly the array the paper's hole scheme (temp, flag, the front and
 * back holes) leaves behind, not only the same key index and sides. That scheme has a
 * closed form. Take the elements after the key in order, let F_t be the t-th one >= key
 * from the front and B_t the t-th one < key from the back, and let T count the t with F_t
 * before B_t. Then B_t swaps places with F_t as the holes move, and F_0 ends at i + 1
 * (temp). The call computes it in four passes: tile counts, their scan, per-element
 * ranks and placement. Same arguments and checks as ksort_partition_out; the workspace
 * of (current device, stream) holds two int32 index arrays of n entries. It is meant for
 * layout-level checks, not for speed. */
KSORT_API ksort_status_t ksort_partition_exact(ksort_dtype_t dtype, const void *in_dev,
                                               void *out_dev, int64_t n,
                                               int64_t *key_index_dev, ksort_stream_t stream);

/* ksort_partition_out without any allocation. The paper has no counterpart: it is a
 * library form for callers that must not allocate device memory. Examples are a
 * process that has given all free HBM to its own pool allocator (cudaMalloc would
 * fail there), and a latency-bound caller that shares the GPU (cudaFree synchronises
 * the whole device, which would stall every other stream). Every other entry point
 * allocates a per-stream workspace on first use, of at least 2^21 look-back
 * descriptors (tens of MB).
 *
 * Arguments, result and checks are those of ksort_partition_out, for
 * 1 <= n <= KSORT_NOALLOC_MAX_KEYS. A larger n returns KSORT_ERR_TOO_LARGE and enqueues
 * nothing. The call allocates nothing: the scratch of the partition kernels (control
 * block, work item, look-back descriptors, ticket map: about 67 KB) is one
 * file-scope device array, one copy per device, and out_dev takes the keys directly.
 *
 * The first call on a device does set-up with that device current: it looks up the
 * array's device address (cudaGetSymbolAddress), reads the SM count and the kernel
 * occupancy, and clears the array on `stream`. Make that first call before any stream
 * capture.
 *
 * Every call on a device shares the one array, which keeps the last call's contents.
 * Each call clears the words that must start at zero (the sticky error word). A new
 * generation number retires the rest. Calls that overlap on the GPU race on the array
 * and give wrong results: different streams without an ordering event, or several host
 * threads. Order them, e.g. on one stream.
 *
 * Errors found on the device (a look-back wait past the tuned time limit, an
 * inconsistent descriptor) are not recorded for ksort_get_device_error(). Instead
 * *key_index_dev receives the negated status (for example -KSORT_ERR_TIMEOUT). */
#define KSORT_NOALLOC_MAX_KEYS (1LL << 24)
KSORT_API ksort_status_t ksort_partition_out_noalloc(ksort_dtype_t dtype, const void *in_dev,
                                           void *out_dev, int64_t n, int64_t *key_index_dev,
                                           ksort_stream_t stream);

/* Steps 1-6: sorts keys_dev[0..n-1] ascending, in place (Section 1.1). The recursion of
 * Steps 5-6 runs on the device (persistent kernel with a work queue); sub-arrays of at
 * most the tuned cutoff are finished inside shared memory by the same key rule.
 * n == 0 or 1 is a no-op. */
KSORT_API ksort_status_t ksort_sort(ksort_dtype_t dtype, void *keys_dev, int64_t n, ksort_stream_t stream);

/* Sorts num_arrays independent arrays in one launch: array r is
 * keys_dev[offsets_dev[r] .. offsets_dev[r+1]). offsets_dev is a device int64 array of
 * num_arrays + 1 nondecreasing entries within [0, total_keys]; total_keys bounds the
 * keys touched (it sizes the scratch). Offsets are checked on the device
 * (KSORT_ERR_BAD_OFFSETS). Capturable in a CUDA graph once the workspace is reserved. */
KSORT_API ksort_status_t ksort_sort_batched(ksort_dtype_t dtype, void *keys_dev, const int64_t *offsets_dev,
                                  int64_t num_arrays, int64_t total_keys, ksort_stream_t stream);

/* Makes sure the workspace of (current device, stream) can serve sorts of up to
 * max_total_keys keys of `dtype` in up to max_arrays arrays. Synchronises the stream
 * if it has to grow the workspace. */
KSORT_API ksort_status_t ksort_reserve_workspace(ksort_dtype_t dtype, int64_t max_total_keys,
                                       int64_t max_arrays, ksort_stream_t stream);

/* Frees the workspace of (current device, stream) after synchronising the stream. */
KSORT_API ksort_status_t ksort_release_workspace(ksort_stream_t stream);

/* Synchronises `stream`, then returns and clears the device error flag of its
 * workspace (KSORT_OK if none). A CUDA error found while synchronising is returned
 * as KSORT_ERR_CUDA. */
KSORT_API ksort_status_t ksort_get_device_error(ksort_stream_t stream);

/* Counters of the last ksort_sort / ksort_sort_batched on `stream` (synchronises). */
typedef struct {
    uint64_t large_items;   /* sub-arrays partitioned by multi-CTA tile passes        */
    uint64_t large_keys;    /* keys in those sub-arrays (each read once, written once) */
    uint64_t tiles;         /* tile passes run                                         */
    uint64_t small_items;   /* sub-arrays finished in shared memory                    */
    uint64_t small_keys;    /* keys in those sub-arrays                                */
    uint64_t smem_levels;   /* partition levels run inside shared memory (all items)   */
    uint64_t lookback_steps;/* 32-wide look-back windows examined                      */
    uint64_t items_pushed;  /* work-queue entries used                                 */
    uint64_t launches;      /* kernels the last sort or partition on `stream` enqueued */
} ksort_stats_t;
KSORT_API ksort_status_t ksort_get_stats(ksort_stream_t stream, ksort_stats_t *out);

/* Phase timing, for the roofline report (off by default). While enabled (enable != 0),
 * every ksort_sort, ksort_sort_batched, ksort_partition and ksort_partition_out call made
 * outside CUDA-graph capture records CUDA events on its stream at the boundaries of its
 * phases. A sort has three phases: the seed kernel; the partition passes (the tile
 * kernel, and the wave form's levels and hand-off); the shared-memory finisher. A
 * partition has one: its launch (two launches in the wave form). The events cost a few
 * microseconds of device time per call. */
KSORT_API ksort_status_t ksort_set_phase_timing(int32_t enable);
/* Synchronises `stream`, then writes the phase durations in milliseconds of up to
 * `max_calls` of the most recent timed calls on it (the last 64 are kept), oldest first,
 * three floats per call: out_ms[3 * c + i] is phase i of call c, and -1 for a phase the
 * call does not have (a partition has only phase 0). out_ms holds 3 * max_calls floats;
 * *calls receives the number of calls written (0 when none on `stream` was timed). */
KSORT_API ksort_status_t ksort_get_phase_times(ksort_stream_t stream, int32_t max_calls,
                                               float *out_ms, int32_t *calls);

/* Tuning for one dtype (process-wide; the autotuner sets it). Zero fields keep their
 * current value.
 *   cutoff:        sub-arrays with at most this many keys are finished in shared
 *                  memory (2 .. ksort_max_cutoff(dtype));
 *   ctas_per_sm:   shared-memory finisher CTAs per SM (capped by occupancy);
 *                  -1 = as many as fit (the default);
 *   spin_limit_ms: time limit of every device-side wait (1 .. 600000);
 *   tile_shape:    form of the partition passes, 1 .. 12 (1 = default); see
 *                  ksort_tile_shape(). Changing it may grow a stream's workspace on
 *                  the next call, so reserve again before capturing a graph.
 *   wave_levels:   tile shapes 10 .. 12 only: recursion levels run as level-synchronous
 *                  passes before the work queue takes over (1 .. 64); -1 = automatic
 *                  (about log2 of the mean array length over the cutoff, plus 2).
 *   medium_tiles:  tile shapes 1 .. 3 and 10 .. 12 (the register form's work queue): a
 *                  sub-array of 2 .. medium_tiles tile passes is taken by one CTA, which
 *                  counts every tile first and then moves them with the prefixes it
 *                  knows (no look-back); 1 .. 16, -1 = off (the default).
 *   partition_form: single partitions (ksort_partition, ksort_partition_out): 1 .. 6 the
 *                  one-pass ring partition in that configuration (5 = the default, see
 *                  ksort_partition_shape); -1 = the form that tile_shape names.
 *   sort_reserve:  sorts in tile shapes 1 .. 3 and 10 .. 12: 1 (the default) = each tile
 *                  pass takes its output ranges in its sub-array with one atomic add on
 *                  the sub-array's counter, so no tile waits for another; the order of
 *                  the tiles' runs inside each side then follows the order in which the
 *                  tiles finished (the sorted result does not change; only which key heads
 *                  each later sub-array does). -1 = decoupled look-back in tile order
 *                  (the layout depends on the input alone).
 *   finish_in_tiles: sorts in tile shape 3 only: W (1 .. 4096) = the CTAs of the tile
 *                  passes also finish small sub-arrays (the shared-memory finisher) while
 *                  the tile passes run: a CTA about to take a new tile takes a queued
 *                  small sub-array instead whenever other CTAs already wait for W or more
 *                  tiles of sub-arrays not yet queued. The finisher launch then takes the
 *                  small sub-arrays left; -1 = off (the default).
 *   finisher_threads: threads of a shared-memory finisher CTA: 256 (the default), 512
 *                  or 1024. More threads finish one sub-array sooner (fewer CTAs fit an
 *                  SM), which shortens sorts whose finisher is one round of sub-arrays.
 *   cluster_sort:  ksort_sort of one array that fits the shared memory of one thread-block
 *                  cluster (16 CTAs, else 8; about 390K 4-byte or 190K 8-byte keys) and
 *                  has fewer than 512 * (cutoff + 1) keys (cutoff >= 64): 1 = its levels
 *                  above the cutoff
 *                  run in that cluster, all sub-arrays of a level at once, exchanging keys
 *                  through distributed shared memory (one launch, then the finisher);
 *                  -1 = off (the default): the work queue.
 * A workspace reserved for one tuning serves any cutoff and finisher setting. */
typedef struct {
    int32_t cutoff;
    int32_t ctas_per_sm;
    int32_t spin_limit_ms;
    int32_t tile_shape;
    int32_t wave_levels;
    int32_t medium_tiles;
    int32_t partition_form;
    int32_t sort_reserve;
    int32_t finish_in_tiles;
    int32_t finisher_threads;
    int32_t cluster_sort;
} ksort_tuning_t;
KSORT_API ksort_status_t ksort_set_tuning(ksort_dtype_t dtype, const ksort_tuning_t *tuning);
KSORT_API ksort_status_t ksort_get_tuning(ksort_dtype_t dtype, ksort_tuning_t *out);
KSORT_API int32_t ksort_max_cutoff(ksort_dtype_t dtype);

/* Keys handled by one tile pass of the partition kernels for `dtype` under the current
 * tuning (threads x keys per thread of its tile shape). */
KSORT_API int32_t ksort_tile_keys(ksort_dtype_t dtype);

/* Form `shape` (1 .. 12) of the partition passes for `dtype`: CTAs of *threads threads,
 * whose tile-holding threads each hold *keys_per_thread keys (a multiple of the 128-bit
 * vector). Three CTA shapes come in four kinds (*form):
 *   0 (shapes 1-3):   every thread loads its keys of a tile straight into registers;
 *   1 (shapes 4-6):   a ring of shared-memory tiles: one warp stages tiles by bulk
 *                     copies, the data warps (threads - 64) compact them in place, and
 *                     one warp takes each tile's output ranges by reservation, so a CTA
 *                     keeps several tiles in flight and no tile waits for another;
 *   2 (shapes 7-9):   warp roles, with one warp loading tiles by bulk copies, one warp
 *                     running look-backs and completions, and the rest (threads - 64)
 *                     counting, scattering and writing, so consecutive tiles overlap;
 *   3 (shapes 10-12): the upper recursion levels (Steps 5-6) run level by level: all
 *                     sub-arrays of one depth are partitioned by two launches, one
 *                     counting and one moving keys, over equal spans of their keys per
 *                     CTA, with no waits between CTAs; the remaining levels then run as
 *                     form 0. Single partitions: see ksort_partition_out. */
KSORT_API ksort_status_t ksort_tile_shape(ksort_dtype_t dtype, int32_t shape, int32_t *threads,
                                          int32_t *keys_per_thread, int32_t *form);

/* Configuration `form` (1 .. 6) of the one-pass ring partition for `dtype`: CTAs of
 * *threads threads (one producer warp, the data warps, and in configurations 4 .. 6
 * two role warps) that stage tiles of *tile_keys keys, compiled for *ctas_per_sm CTAs
 * per SM. 1 .. 3: the last data warp of a tile takes its output ranges (one atomic add);
 * 4: two role warps take them by look-back, in tile order; 5, 6: two role warps take them
 * by the atomic add, so the data warps never wait on it. Every configuration moves the
 * same bytes per tile for 4- and 8-byte keys. */
KSORT_API ksort_status_t ksort_partition_shape(ksort_dtype_t dtype, int32_t form,
                                               int32_t *threads, int32_t *tile_keys,
                                               int32_t *ctas_per_sm);

/* Cluster form of ksort_sort (tuning cluster_sort) on the current device: the CTAs of
 * its thread-block cluster (16, else 8; 0 when no cluster of 1024-thread CTAs can run) and
 * the most keys of `dtype` it holds. Arrays above that, or of 512 * (cutoff + 1) keys or
 * more, take the work queue. */
KSORT_API ksort_status_t ksort_cluster_shape(ksort_dtype_t dtype, int32_t *cluster_ctas,
                                             int64_t *max_keys);

/* Failure-path check: runs one device-side wait, of the kind the partition's look-back
 * uses, on a flag that nothing ever sets. The wait gives up after limit_ms (1..60000),
 * records KSORT_ERR_TIMEOUT in the stream's workspace and returns; the next
 * ksort_get_device_error(stream) reports it. No fault, trap or endless loop. */
KSORT_API ksort_status_t ksort_selftest_wait_timeout(int32_t limit_ms, ksort_stream_t stream);

/* Failure-path check of ksort_partition_out_noalloc: runs the same bounded wait on a
 * look-back descriptor of the fixed device array that nothing publishes, then the
 * call's status step, so that *key_index_dev (device int64) receives
 * -KSORT_ERR_TIMEOUT after about limit_ms (1..60000). Allocates nothing; ordered on
 * `stream` like any ksort_partition_out_noalloc call, whose next call starts clean. */
KSORT_API ksort_status_t ksort_selftest_noalloc_timeout(int32_t limit_ms, int64_t *key_index_dev,
                                                        ksort_stream_t stream);

/* Diagnostics: while set, every tile pass of ksort_sort / ksort_sort_batched /
 * ksort_partition* writes 8 uint64 words per tile ticket into trace_dev[ticket * 8 ..]
 * for tickets < `tickets`: %globaltimer stamps (ns) of [0] ticket claimed, [1] ticket
 * issued, [2] keys loaded and counted, [3] look-back done, [4] written, [5] first
 * look-back window read (0 for tile 0), [6] completed; [7] = CTA index
 * | look-back windows << 20 | look-back polls << 40. In the cluster form (tuning
 * cluster_sort) entry k * 8 + j is level k instead: %globaltimer stamps of [0] level
 * start, [1] counts scanned, [2] counts of every CTA ready, [3] prefixes read,
 * [4] keys stored, [5] keys landed, [6] next table built, [7] active sub-arrays (CTA 0).
 * The caller owns the buffer (device memory); pass NULL / 0 to stop. Costs a little
 * time. */
KSORT_API ksort_status_t ksort_debug_trace(uint64_t *trace_dev, int64_t tickets);

/* Static text for a status code. */
KSORT_API const char *ksort_status_string(ksort_status_t status);

/* Text of the last CUDA runtime error seen by this thread inside the library. */
KSORT_API const char *ksort_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* KSORT_H */
