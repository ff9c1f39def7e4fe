"""Pins for the C oracle of K-sort (arxiv 1107.3622, Section 1.1, Steps 1-6).

Each check ties the oracle to something other than itself: the values the paper
prints for its worked example (Section 1.2), brute force over every permutation and
every {0,1,2}-word of length <= 8 against Python's ``sorted``, the partition
postconditions that define Steps 1-4, closed forms for the comparison count (n-1 per
call; n(n-1)/2 on sorted, reversed and constant input; 2(n+1)H_n - 4n on average for
distinct random keys, the Quick-sort recurrence that Section 1 appeals to), and
numpy's sort on large random inputs.

test_oracle_mutants.py re-runs this file against deliberately broken copies of the
oracle to show that these pins catch plausible mistakes.
"""
import itertools
import math
import os

import numpy as np
import pytest

import ksort_inputs as gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "illustration.txt")


def _read_golden():
    rows, inp, final = [], None, None
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tag, rest = line.split(" ", 1)
            if tag == "input":
                inp = [int(x) for x in rest.split()]
            elif tag == "sorted":
                final = [int(x) for x in rest.split()]
            elif tag == "row":
                key, arr, temp = (s.strip() for s in rest.split("|"))
                rows.append((int(key), [int(x) for x in arr.split()],
                             None if temp == "nil" else int(temp)))
    return inp, rows, final


@pytest.mark.parametrize("dtype", [np.uint32, np.float32, np.float64])
def test_illustration(ref, dtype):
    """Section 1.2: rows Key=55, 8, 50 match exactly (list and Temp). Row Key=66 is
    checked where the printed table agrees with the Steps (key index, Temp, the
    positions outside 7-8, and the multiset of 7-8). The final list matches."""
    inp, rows, final = _read_golden()
    a = np.array(inp, dtype)
    st, calls = ref.sort_traced(a)

    for (key, arr, temp), got in zip(rows[:3], calls[:3]):
        assert got["key"] == key
        assert list(got["array"]) == arr
        assert got["temp"] == temp

    key66, arr66, temp66 = rows[3]
    got = calls[3]
    assert got["key"] == key66 and got["index"] == 6 and got["temp"] == temp66
    assert list(got["array"][:7]) == arr66[:7] and got["array"][9] == arr66[9]
    assert sorted(got["array"][7:9]) == sorted(arr66[7:9])

    assert list(a) == final
    # The Steps make six calls (keys 55, 8, 50, 66, 75, 78) and 9+3+1+4+2+1 = 20 compares.
    assert [c["key"] for c in calls] == [55, 8, 50, 66, 75, 78]
    assert (st.calls, st.compares) == (6, 20)
    # The last printed row (Key=78, Temp=94) is also the Steps' last call.
    assert calls[-1]["temp"] == rows[4][2] and list(calls[-1]["array"]) == rows[4][1]


def _check_partition(ref, vals, dtype):
    a = np.array(vals, dtype)
    before = a.copy()
    i, flag, temp, cmp_ = ref.partition(a, 0, len(a) - 1)
    key = before[0]
    assert cmp_ == len(a) - 1                                   # n-1 compares
    assert i == int(np.sum(before[1:] < key))                   # key lands at #{x < key}
    assert a[i] == key
    assert np.all(a[:i] < key) and np.all(a[i + 1:] >= key)     # Step-3 predicate
    assert sorted(a.tolist()) == sorted(before.tolist())        # a permutation
    assert flag == int(np.any(before[1:] >= key))
    if flag:                                                    # temp = first x >= key
        first_ge = before[1:][before[1:] >= key][0]
        assert temp == first_ge and a[i + 1] == first_ge


def _check_sort(ref, vals, dtype):
    a = np.array(vals, dtype)
    st = ref.sort(a)
    assert a.tolist() == sorted(vals)
    return st


@pytest.mark.parametrize("n", range(1, 9))
def test_bruteforce_permutations(ref, n):
    for perm in itertools.permutations(range(n)):
        _check_sort(ref, list(perm), np.uint32)
        if n >= 2:
            _check_partition(ref, list(perm), np.uint32)


@pytest.mark.parametrize("n", range(1, 9))
def test_bruteforce_words_with_duplicates(ref, n):
    for word in itertools.product((0, 1, 2), repeat=n):
        _check_sort(ref, list(word), np.float32)
        if n >= 2:
            _check_partition(ref, list(word), np.float32)


@pytest.mark.parametrize("n", [2, 3, 10, 100, 2000])
@pytest.mark.parametrize("pattern", ["sorted", "reverse", "constant"])
def test_worst_case_closed_form(ref, n, pattern):
    """Sorted, reversed and constant inputs make every partition peel one element:
    n-1 calls, depth n-1 and n(n-1)/2 compares, the O(n^2) case of Sections 1 and 5."""
    if pattern == "sorted":
        vals = list(range(n))
    elif pattern == "reverse":
        vals = list(range(n, 0, -1))
    else:
        vals = [7] * n
    st = _check_sort(ref, vals, np.uint32)
    assert st.calls == n - 1
    assert st.max_depth == n - 1
    assert st.compares == n * (n - 1) // 2


def test_average_compares_closed_form(ref):
    """Mean compares over random distinct keys = 2(n+1)H_n - 4n (first-element key,
    n-1 compares per call, children uniformly random). 200 seeds at n = 1000; the
    standard deviation of one sort is about 0.65 n, so the mean is within +-250."""
    n, reps = 1000, 200
    total = 0
    for r in range(reps):
        vals = gen.splitmix64(gen.seed_for(0, 7, r), n)
        a = np.argsort(vals, kind="stable").astype(np.uint32)  # a random permutation
        total += ref.sort(a).compares
        assert np.array_equal(a, np.arange(n, dtype=np.uint32))
    h = sum(1.0 / k for k in range(1, n + 1))
    expected = 2 * (n + 1) * h - 4 * n
    assert abs(total / reps - expected) < 250, (total / reps, expected)


@pytest.mark.parametrize("dtype", ["f32", "f64", "u32"])
def test_matches_numpy_sort(ref, dtype):
    a = gen.make("uniform", dtype, 100_000, gen.seed_for(0, 0, 0))
    want = np.sort(a)
    st = ref.sort(a)
    assert a.tobytes() == want.tobytes()
    assert st.compares > 0 and st.calls < 100_000


@pytest.mark.parametrize("pattern", ["distinct16", "organ_pipe"])
def test_stress_patterns_match_numpy(ref, pattern):
    for dtype in ("f32", "u32"):
        a = gen.make(pattern, dtype, 3000, gen.seed_for(3, 1, 0))
        want = np.sort(a)
        ref.sort(a)
        assert a.tobytes() == want.tobytes()


def test_batched_equals_per_array(ref):
    lengths = np.array([0, 1, 2, 3, 17, 1000, 0, 5, 4096], np.int64)
    off = gen.offsets_from_lengths(lengths)
    flat = gen.uniform_f32(gen.seed_for(2, 0, 0), int(off[-1]))
    per = flat.copy()
    ref.sort_batched(flat, off)
    for r in range(len(lengths)):
        seg = per[off[r]:off[r + 1]]
        ref.sort(seg)
    assert flat.tobytes() == per.tobytes()
    for r in range(len(lengths)):
        assert np.all(np.diff(flat[off[r]:off[r + 1]]) >= 0)


def test_partition_on_subrange_leaves_rest(ref):
    a = gen.uniform_u32(gen.seed_for(0, 3, 0), 50)
    b = a.copy()
    i, *_ = ref.partition(a, 10, 39)
    assert np.array_equal(a[:10], b[:10]) and np.array_equal(a[40:], b[40:])
    assert 10 <= i <= 39 and i == 10 + int(np.sum(b[11:40] < b[10]))


def test_single_and_empty_are_noops(ref):
    for n in (0, 1):
        a = np.array([42] * n, np.uint32)
        st = ref.sort(a)
        assert st.calls == 0 and a.tolist() == [42] * n
