/*
 * Body of the K-sort oracle, written once and included by ksort_ref.c for each
 * element type. Before inclusion the includer defines
 *     KT         the element type (float, double, uint32_t)
 *     KNAME(x)   x with the type suffix appended (x##_f32, ...)
 *
 * TEST INFRASTRUCTURE ONLY (see ksort_ref.h).
 *
 * Variable names follow the paper (arxiv 1107.3622, Section 1.1): key, i, j, k, p,
 * temp, flag, left, right. Readings of the text used here:
 *   - Step 2 "repeat step 3 till (j-i) >= 2 is satisfied" is read as: repeat
 *     while (j - i) >= 2 (the other reading would never run Step 3).
 *   - The closing "decrease j by 1 and assign p = j" of Step 3.1 applies after
 *     either branch (or neither) of Step 3.1.
 *   - flag starts at 0 on every call; temp is only meaningful when flag == 1.
 *   - Step 5 recurses on [left, i-1] when left < i-1; Step 6 recurses on
 *     [i+1, right] when right > i+1 (the printed "left > i+1" can never hold; the
 *     illustration of Section 1.2 does recurse on the right part). The key at i is
 *     final and belongs to neither sub-array.
 *   - Recursion order: Step 5 (left part) is finished before Step 6 (right part).
 */

/* Steps 1-4 on a[left..right]. */
int64_t KNAME(ksort_ref_partition)(KT *a, int64_t left, int64_t right,
                                   int32_t *flag_out, KT *temp_out, uint64_t *compares_out)
{
    /* Step 1: the first element is the key; i = left, j = right + 1, k = p = left + 1. */
    KT key = a[left];
    int64_t i = left;
    int64_t j = right + 1;
    int64_t p = left + 1;
    int64_t k = p;
    KT temp = key;
    int32_t flag = 0;
    uint64_t compares = 0;

    /* Step 2: repeat Step 3 while (j - i) >= 2. */
    while (j - i >= 2) {
        /* Step 3: compare a[p] with the key. */
        compares++;
        if (key <= a[p]) {
            /* Step 3.1: a[p] belongs to the right of the key. */
            if (p != j && j != right + 1) {
                a[j] = a[p];
            } else if (j == right + 1) {
                temp = a[p];
                flag = 1;
            }
            j = j - 1;
            p = j;
        } else {
            /* Step 3.2: a[p] belongs to the left of the key. */
            a[i] = a[p];
            i = i + 1;
            k = k + 1;
            p = k;
        }
    }

    /* Step 4: the key goes to a[i]; a saved temp goes just after it. */
    a[i] = key;
    if (flag == 1) {
        a[i + 1] = temp;
    }

    if (flag_out) *flag_out = flag;
    if (flag_out && temp_out && flag == 1) *temp_out = temp;
    if (compares_out) *compares_out = compares;
    return i;
}

/* Steps 1-6 on a[0..n-1]. The recursion of Steps 5-6 is run with an explicit LIFO
 * stack so that depth n-1 (sorted input) does not overflow the C stack; pushing the
 * right part before the left part keeps the paper's order (left part first). */
int KNAME(ksort_ref_sort)(KT *a, int64_t n, ksort_ref_stats_t *stats, ksort_ref_trace_t *trace)
{
    int64_t cap, top;
    int64_t *lo_s, *hi_s, *depth_s;

    if (trace) trace->count = 0;
    if (n <= 1) return 0; /* a single value need not be processed (Section 1.2 note) */

    /* Every stacked range holds >= 2 elements and the ranges are disjoint. */
    cap = n / 2 + 2;
    lo_s = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
    hi_s = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
    depth_s = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
    if (!lo_s || !hi_s || !depth_s) {
        free(lo_s); free(hi_s); free(depth_s);
        return -1;
    }

    top = 0;
    lo_s[top] = 0; hi_s[top] = n - 1; depth_s[top] = 1; top++;

    while (top > 0) {
        int64_t left, right, depth, i;
        int32_t flag = 0;
        KT key, temp;
        uint64_t compares = 0;

        top--;
        left = lo_s[top]; right = hi_s[top]; depth = depth_s[top];

        key = a[left];
        temp = key;
        i = KNAME(ksort_ref_partition)(a, left, right, &flag, &temp, &compares);

        if (stats) {
            stats->calls++;
            stats->compares += compares;
            if ((uint64_t)depth > stats->max_depth) stats->max_depth = (uint64_t)depth;
        }
        if (trace) {
            int64_t c = trace->count;
            if (c < trace->capacity) {
                if (trace->left) trace->left[c] = left;
                if (trace->right) trace->right[c] = right;
                if (trace->index) trace->index[c] = i;
                if (trace->flag) trace->flag[c] = flag;
                if (trace->key) ((KT *)trace->key)[c] = key;
                if (trace->temp) ((KT *)trace->temp)[c] = temp;
                if (trace->snapshot) memcpy((KT *)trace->snapshot + c * n, a, (size_t)n * sizeof(KT));
            }
            trace->count = c + 1;
        }

        /* Step 6 (pushed first, so it runs after everything Step 5 starts). */
        if (right > i + 1) {
            lo_s[top] = i + 1; hi_s[top] = right; depth_s[top] = depth + 1; top++;
        }
        /* Step 5. */
        if (left < i - 1) {
            lo_s[top] = left; hi_s[top] = i - 1; depth_s[top] = depth + 1; top++;
        }
    }

    free(lo_s); free(hi_s); free(depth_s);
    return 0;
}

int KNAME(ksort_ref_sort_batched)(KT *a, const int64_t *offsets, int64_t num_arrays,
                                  ksort_ref_stats_t *stats)
{
    int64_t r;
    for (r = 0; r < num_arrays; r++) {
        int64_t b = offsets[r], e = offsets[r + 1];
        if (b < 0 || e < b) return -1;
        if (KNAME(ksort_ref_sort)(a + b, e - b, stats, NULL) != 0) return -1;
    }
    return 0;
}
