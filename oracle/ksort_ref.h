/*
 * K-sort oracle: a plain, slow, single-threaded C99 restatement of K-sort
 * (Sundararajan, Pal, Chakraborty, Mahanti, arxiv 1107.3622, Section 1.1, Steps 1-6).
 *
 * TEST INFRASTRUCTURE ONLY. This code exists to check the GPU library against the
 * paper. Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may build, load or call it. It shares no code, header, table or helper with the
 * CUDA library, and the library never calls it.
 *
 * Element types: float32 (f32), float64 (f64), uint32 (u32). Comparison is the native
 * C `key <= a[p]` of Step 3 for each type (IEEE for the floats).
 *
 * Parity status: every function here is pinned by the CPU test suite (the paper's
 * worked illustration of Section 1.2, brute force over all permutations and all
 * {0,1,2}-words up to length 8, partition postconditions, compare-count closed forms
 * and a library sort). None is "parity unpinned".
 */
#ifndef KSORT_REF_H
#define KSORT_REF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Counters over one sort (Steps 1-6). */
typedef struct {
    uint64_t calls;     /* executions of Steps 1-4 (one per sub-array of >= 2 elements) */
    uint64_t compares;  /* evaluations of the Step-3 test `key <= a[p]` */
    uint64_t max_depth; /* deepest recursion level reached; the whole array is level 1 */
} ksort_ref_stats_t;

/* Optional per-call record, in the order the calls execute (depth first, Step 5
 * before Step 6). Arrays are caller-owned with `capacity` entries; `count` receives
 * the number of calls (only the first `capacity` are stored). `key`, `temp` and
 * `snapshot` have the element type of the sort; `snapshot` (may be NULL) holds
 * `capacity * n` elements: the whole array after each call. */
typedef struct {
    int64_t capacity;
    int64_t count;
    int64_t *left;      /* sub-array first index */
    int64_t *right;     /* sub-array last index (inclusive, the paper's `right`) */
    int64_t *index;     /* the key's final index i (Step 4) */
    int32_t *flag;      /* Step-4 flag: 1 when temp was written to a[i+1] */
    void *key;          /* the key of the call (Step 1) */
    void *temp;         /* temp of the call; meaningful only when flag == 1 */
    void *snapshot;
} ksort_ref_trace_t;

/* Steps 1-4 on a[left..right] (inclusive, right > left). Returns the key's final
 * index i. When non-NULL: *flag_out gets the Step-4 flag, *temp_out the temp value
 * (unchanged when flag is 0), *compares_out the number of Step-3 comparisons. */
int64_t ksort_ref_partition_f32(float *a, int64_t left, int64_t right,
                                int32_t *flag_out, float *temp_out, uint64_t *compares_out);
int64_t ksort_ref_partition_f64(double *a, int64_t left, int64_t right,
                                int32_t *flag_out, double *temp_out, uint64_t *compares_out);
int64_t ksort_ref_partition_u32(uint32_t *a, int64_t left, int64_t right,
                                int32_t *flag_out, uint32_t *temp_out, uint64_t *compares_out);

/* Steps 1-6 on a[0..n-1], in place, ascending. n <= 1 is a no-op. stats and trace
 * may be NULL. Returns 0, or -1 if the explicit stack could not be allocated. */
int ksort_ref_sort_f32(float *a, int64_t n, ksort_ref_stats_t *stats, ksort_ref_trace_t *trace);
int ksort_ref_sort_f64(double *a, int64_t n, ksort_ref_stats_t *stats, ksort_ref_trace_t *trace);
int ksort_ref_sort_u32(uint32_t *a, int64_t n, ksort_ref_stats_t *stats, ksort_ref_trace_t *trace);

/* Sorts each array a[offsets[r] .. offsets[r+1]) independently with Steps 1-6.
 * Returns 0, or -1 on a bad offset or allocation failure. stats accumulate. */
int ksort_ref_sort_batched_f32(float *a, const int64_t *offsets, int64_t num_arrays,
                               ksort_ref_stats_t *stats);
int ksort_ref_sort_batched_f64(double *a, const int64_t *offsets, int64_t num_arrays,
                               ksort_ref_stats_t *stats);
int ksort_ref_sort_batched_u32(uint32_t *a, const int64_t *offsets, int64_t num_arrays,
                               ksort_ref_stats_t *stats);

#ifdef __cplusplus
}
#endif
#endif /* KSORT_REF_H */
