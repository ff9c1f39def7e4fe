"""GPU parity: libksort (through its C ABI) against the C oracle, on the same seeded
inputs. Sorts must be bit-identical; a first-level partition (Steps 1-4) must give
the oracle's key index and the same two multisets. Sizes span several tiles with
ragged tails, the shared-memory cutoff on both sides, misaligned starts, and the
paper's own example (Section 1.2)."""
import numpy as np
import pytest

import ksort_inputs as gen

pytestmark = pytest.mark.gpu

DTYPES = ["f32", "f64", "u32"]


@pytest.fixture(scope="module")
def ks():
    import torch
    import paper_1107_3622_gb300 as ks
    ks.load()
    torch.cuda.set_device(0)
    return ks


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def to_host(t):
    return t.cpu().numpy()


def gpu_sort(ks, a):
    t = to_dev(a)
    ks.sort_(t)
    assert ks.ksort_get_device_error() == 0
    return to_host(t)


def oracle_sort(ref, a):
    b = a.copy()
    ref.sort(b)
    return b


def check_partition(ref, ks, a, out_of_place=False):
    import torch
    t = to_dev(a)
    if out_of_place:
        dst = torch.empty_like(t)
        i = int(ks.partition_out(t, dst).item())
        got = to_host(dst)
        assert to_host(t).tobytes() == a.tobytes()  # input untouched
    else:
        i = ks.partition_(t)
        got = to_host(t)
    assert ks.ksort_get_device_error() == 0
    b = a.copy()
    ri, *_ = ref.partition(b)
    assert i == ri
    assert got[i] == a[0]
    assert np.sort(got[:i]).tobytes() == np.sort(b[:ri]).tobytes()
    assert np.sort(got[i + 1:]).tobytes() == np.sort(b[ri + 1:]).tobytes()


def test_illustration(ref, ks):
    for dt in (np.uint32, np.float32, np.float64):
        a = np.array(gen.ILLUSTRATION, dt)
        assert gpu_sort(ks, a).tobytes() == oracle_sort(ref, a).tobytes()
        check_partition(ref, ks, a)


PART_SIZES = [2, 3, 5, 31, 32, 33, 1000, 4095, 4096, 4097, 8191, 8192, 8193, 8194,
              65537, 100_000, 1_000_003]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", PART_SIZES)
def test_partition(ref, ks, dtype, n):
    a = gen.make("uniform", dtype, n, gen.seed_for(1, n % 977, 0))
    check_partition(ref, ks, a)
    check_partition(ref, ks, a, out_of_place=True)


@pytest.mark.parametrize("dtype", DTYPES)
def test_partition_misaligned_starts(ref, ks, dtype):
    """Sub-tensors that start 1..3 keys past a 16-byte boundary (for float64 an offset
    of 2 keys is aligned again, which is covered too)."""
    import torch
    base = gen.make("uniform", dtype, 50_003, gen.seed_for(1, 99, 1))
    for off in (1, 2, 3):
        a = base[off:]
        big = to_dev(base)
        view = big[off:]
        assert view.data_ptr() % 16 == (off * a.itemsize) % 16
        i = ks.partition_(view)
        b = a.copy()
        ri, *_ = ref.partition(b)
        got = to_host(view)
        assert i == ri and got[i] == a[0]
        assert np.sort(got[:i]).tobytes() == np.sort(b[:ri]).tobytes()
        assert to_host(big[:off]).tobytes() == base[:off].tobytes()
        t = to_dev(base)[off:]
        ks.sort_(t)
        assert to_host(t).tobytes() == oracle_sort(ref, a).tobytes()
    assert ks.ksort_get_device_error() == 0


SORT_SIZES = [0, 1, 2, 3, 17, 255, 4095, 4096, 4097, 8193, 20_000, 100_000, 1_000_000]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", SORT_SIZES)
def test_sort_uniform(ref, ks, dtype, n):
    a = gen.make("uniform", dtype, n, gen.seed_for(1, n % 1013, 2))
    assert gpu_sort(ks, a).tobytes() == oracle_sort(ref, a).tobytes()


@pytest.mark.parametrize("dtype", ["f32", "u32"])
@pytest.mark.parametrize("pattern", ["sorted", "reverse", "distinct16", "organ_pipe",
                                     "quantized15"])
@pytest.mark.parametrize("n", [20_000, 30_000, 50_000])
def test_sort_stress(ref, ks, dtype, pattern, n):
    """Input-structure stress at oracle-feasible sizes: the paper's worst cases for the
    first-element key (Section 1; O(n^2) on sorted input)."""
    a = gen.make(pattern, dtype, n, gen.seed_for(3, n, 0))
    assert gpu_sort(ks, a).tobytes() == oracle_sort(ref, a).tobytes()


@pytest.mark.parametrize("dtype,n", [("f32", 7_000_000), ("f64", 10_000_000),
                                     ("u32", 2_500_000)])
def test_sort_table1_sizes(ref, ks, dtype, n):
    """Whole-array parity at the paper's Table 1 sizes, in the launch configuration the
    benchmark times (one ksort_sort call on the default stream)."""
    a = gen.make("uniform", dtype, n, gen.seed_for(1, 6, 0))
    assert gpu_sort(ks, a).tobytes() == oracle_sort(ref, a).tobytes()


def test_repeated_calls_and_streams(ref, ks):
    import torch
    a = gen.uniform_f32(gen.seed_for(1, 3, 3), 300_000)
    want = oracle_sort(ref, a)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    t1, t2 = to_dev(a), to_dev(a[::-1].copy())
    torch.cuda.synchronize()
    for _ in range(3):
        with torch.cuda.stream(s1):
            ks.sort_(t1)
        with torch.cuda.stream(s2):
            ks.sort_(t2)
    torch.cuda.synchronize()
    assert ks.ksort_get_device_error(s1) == 0 and ks.ksort_get_device_error(s2) == 0
    assert to_host(t1).tobytes() == want.tobytes()
    assert to_host(t2).tobytes() == want.tobytes()


def test_stats_account_for_every_key(ks):
    n = 1_000_000
    t = to_dev(gen.uniform_f32(gen.seed_for(1, 4, 0), n))
    ks.sort_(t)
    st = ks.ksort_get_stats()
    # every key ends either as a large item's key or inside a small item or alone
    assert st["large_keys"] >= n and st["small_keys"] <= n
    assert st["tiles"] >= st["large_items"] >= 1
    assert st["items_pushed"] == st["large_items"] + st["small_items"]


@pytest.mark.parametrize("dtype", DTYPES)
def test_sort_duplicate_heavy(ref, ks, dtype):
    """U[0,1] on 2**15 levels (each value about n / 32768 times): long runs of keys equal
    to their sub-array's key, which Step 3 sends right one partition at a time."""
    a = gen.make("quantized15", dtype, 1_000_000, gen.seed_for(8, 0, 0))
    assert gpu_sort(ks, a).tobytes() == oracle_sort(ref, a).tobytes()


def _f64_specials(seed, n, with_nan):
    """float64 keys over the whole range: both signs, subnormals, extremes, infinities,
    +0 and -0 (and NaN when asked), mixed with normal values."""
    rng = np.random.default_rng(seed)
    pool = [0.0, np.inf, -np.inf, 5e-324, -5e-324, 2.2250738585072014e-308,
            -2.2250738585072014e-308, 1.7976931348623157e308, -1.7976931348623157e308,
            1.0, -1.0, 0.5]
    if with_nan:
        pool += [np.nan, -0.0]
    a = rng.standard_normal(n) * 10.0 ** rng.integers(-300, 300, n)
    pick = rng.random(n) < 0.3
    a[pick] = rng.choice(np.array(pool), int(pick.sum()))
    return a


@pytest.mark.parametrize("n", [2, 31, 5000, 70_001, 1_000_003])
def test_f64_special_values(ref, ks, n):
    """float64 classification (done on integer pipes) equals the IEEE compare of the
    oracle for every class of double: sorts bit-identical without NaN and -0 (where the
    sorted array is unique), and partitions with NaN and -0 give the oracle's key index
    and sides, for every choice of key class."""
    a = _f64_specials(gen.seed_for(8, 1, n), n, with_nan=False)
    assert gpu_sort(ks, a).tobytes() == oracle_sort(ref, a).tobytes()
    import torch
    bits = lambda v: np.sort(v.view(np.uint64)).tobytes()  # noqa: E731 (multiset of patterns)
    pool = [np.nan, -0.0, 0.0, np.inf, -np.inf, 5e-324, -1.0]
    for j, key in enumerate(pool):
        a = _f64_specials(gen.seed_for(8, 2 + j, n), n, with_nan=True)
        a[0] = key
        want = a.copy()
        ri, *_ = ref.partition(want)
        for out_of_place in (False, True):
            t = to_dev(a)
            if out_of_place:
                dst = torch.empty_like(t)
                i = int(ks.partition_out(t, dst).item())
                got = to_host(dst)
            else:
                i = ks.partition_(t)
                got = to_host(t)
            assert ks.ksort_get_device_error() == 0
            assert i == ri, (key, out_of_place)
            assert got[i:i + 1].tobytes() == a[:1].tobytes()
            assert bits(got[:i]) == bits(want[:ri]) and bits(got[i + 1:]) == bits(want[ri + 1:])


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_sort_with_nan_is_a_permutation(ks, dtype):
    """With NaN keys (Step 3's `key <= x` is false on either side of a NaN) the sort's
    order depends on element order, so it is not compared with the oracle; it must still
    be a permutation of its input, including inside the shared-memory leaves."""
    rng = np.random.default_rng(12)
    npdt = np.float32 if dtype == "f32" else np.float64
    for n in (2, 7, 31, 33, 1000, 5000, 100_003):
        for frac in (0.02, 0.5):
            a = rng.random(n).astype(npdt)
            a[rng.random(n) < frac] = np.nan
            got = gpu_sort(ks, a)
            bits = np.uint32 if dtype == "f32" else np.uint64
            assert np.array_equal(np.sort(got.view(bits)), np.sort(a.view(bits))), (n, frac)
            # The keys that are not NaN end in ascending order among themselves: a
            # partition around a number puts every smaller number before it and every
            # larger or equal one after it, and a NaN key sends all keys of its sub-array
            # before itself, so no step ever moves a larger number ahead of a smaller one.
            fin = got[~np.isnan(got)]
            assert np.all(fin[1:] >= fin[:-1]), (n, frac)
