"""The wave form (tile shapes 10-12). Sorts: the upper recursion levels run level by
level, each as a counting launch and a moving launch over equal key spans per CTA, then
the work queue finishes what remains. Every result must stay byte-identical to the
oracle whatever the number of wave levels (the hand-off to the queue can happen at any
depth), at both ends of the cutoff range, on degenerate and duplicate-heavy inputs, on
batches (many roots on one level list) and under CUDA-graph capture. Single partitions:
a counting launch and a moving launch over runs of warp tiles per warp, checked against
the oracle's key index and side multisets for every key type, from one warp tile to
many per warp, unaligned starts, in place, and interleaved with part_kernel calls."""
import numpy as np
import pytest

import ksort_inputs as gen

pytestmark = pytest.mark.gpu

DTYPES = {"f32": 0, "f64": 1, "u32": 2}
WAVE = (10, 11, 12)


@pytest.fixture(scope="module")
def ks():
    import torch
    import paper_1107_3622_gb300 as ks
    ks.load()
    torch.cuda.set_device(0)
    return ks


@pytest.fixture
def restore(ks):
    """Single partitions in this module follow the tile shape (the split partition for
    the wave form, part_kernel for shapes 1-3) instead of the ring partition."""
    saved = {c: ks.ksort_get_tuning(c) for c in DTYPES.values()}
    for c in DTYPES.values():
        ks.ksort_set_tuning(c, partition_form=-1)
    yield
    for c, t in saved.items():
        ks.ksort_set_tuning(c, cutoff=t["cutoff"], ctas_per_sm=t["ctas_per_sm"] or -1,
                            tile_shape=t["tile_shape"], wave_levels=t["wave_levels"],
                            partition_form=t["partition_form"])


def _dev(a):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


def _sort(ks, code, a):
    t = _dev(a)
    ks.ksort_sort(code, t, len(a))
    assert ks.ksort_get_device_error() == 0
    return t.cpu().numpy().view(a.dtype)


def _oracle(ref, a):
    b = a.copy()
    ref.sort(b)
    return b


@pytest.mark.parametrize("shape", WAVE)
@pytest.mark.parametrize("dtype", list(DTYPES))
def test_wave_sort_sizes(ref, ks, restore, dtype, shape):
    code = DTYPES[dtype]
    ks.ksort_set_tuning(code, tile_shape=shape, wave_levels=-1)
    assert ks.ksort_tile_shape(code, shape)[2] == 3
    tile = ks.ksort_tile_keys(code)
    for n in (2, 3, 100, tile - 1, tile + 1, 3 * tile + 5, 250_003, 1_000_000):
        a = gen.make("uniform", dtype, n, gen.seed_for(9, shape, n % 1009))
        assert _sort(ks, code, a).tobytes() == _oracle(ref, a).tobytes(), n


@pytest.mark.parametrize("levels", [1, 2, 3, 5, 8, 24])
def test_wave_levels_any_handoff_depth(ref, ks, restore, levels):
    """The hand-off from the level lists to the work queue at any depth, including
    after the lists have emptied (24 levels), gives the same bytes."""
    for dtype, code in DTYPES.items():
        ks.ksort_set_tuning(code, tile_shape=10, wave_levels=levels, cutoff=1024)
        a = gen.make("uniform", dtype, 700_001, gen.seed_for(9, 20 + levels, code))
        assert _sort(ks, code, a).tobytes() == _oracle(ref, a).tobytes(), dtype


@pytest.mark.parametrize("cutoff", [2, 33, 1024, 16384])
def test_wave_cutoff_extremes(ref, ks, restore, cutoff):
    for dtype, code in DTYPES.items():
        c = min(cutoff, ks.ksort_max_cutoff(code))
        ks.ksort_set_tuning(code, tile_shape=11, cutoff=c, wave_levels=-1)
        for pattern in ("uniform", "distinct16"):
            a = gen.make(pattern, dtype, 60_000, gen.seed_for(9, 30, c))
            assert _sort(ks, code, a).tobytes() == _oracle(ref, a).tobytes(), (dtype, pattern)


@pytest.mark.parametrize("pattern", ["sorted", "reverse", "distinct16", "organ_pipe",
                                     "quantized15"])
def test_wave_stress_patterns(ref, ks, restore, pattern):
    """Degenerate orders keep one large sub-array per level (every level a single
    shrinking item); duplicate runs peel one key per partition."""
    for dtype, code in DTYPES.items():
        ks.ksort_set_tuning(code, tile_shape=10, wave_levels=6)
        n = 50_000 if pattern in ("sorted", "reverse", "organ_pipe") else 400_000
        a = gen.make(pattern, dtype, n, gen.seed_for(9, 40, n))
        assert _sort(ks, code, a).tobytes() == _oracle(ref, a).tobytes(), (dtype, pattern)


@pytest.mark.parametrize("dtype", list(DTYPES))
def test_wave_table1_size(ref, ks, restore, dtype):
    code = DTYPES[dtype]
    ks.ksort_set_tuning(code, tile_shape=10, wave_levels=-1)
    n = {"f32": 7_000_000, "f64": 10_000_000, "u32": 2_500_000}[dtype]
    a = gen.make("uniform", dtype, n, gen.seed_for(9, 50, 0))
    assert _sort(ks, code, a).tobytes() == _oracle(ref, a).tobytes()


def test_wave_batched_and_graph(ref, ks, restore):
    import torch
    ks.ksort_set_tuning(ks.F32, tile_shape=10, wave_levels=-1)
    lengths = gen.batched_lengths(300, 2, 200_000, seed=gen.seed_for(9, 60, 0))
    lengths[5] = 0
    lengths[7] = 1
    lengths[11] = 1_000_000
    off = gen.offsets_from_lengths(lengths)
    flat = gen.uniform_f32(gen.seed_for(9, 61, 0), int(off[-1]))
    want = flat.copy()
    ref.sort_batched(want, off)
    pristine = _dev(flat)
    offs = _dev(off)
    keys = pristine.clone()
    ks.sort_batched_(keys, offs)
    assert ks.ksort_get_device_error() == 0
    assert keys.cpu().numpy().tobytes() == want.tobytes()
    # the same call captured once and replayed
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ks.ksort_reserve_workspace(ks.F32, int(off[-1]), len(lengths), stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    keys = pristine.clone()
    with torch.cuda.graph(g, stream=s):
        ks.sort_batched_(keys, offs, stream=s)
    for _ in range(3):
        keys.copy_(pristine)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert keys.cpu().numpy().tobytes() == want.tobytes()
    assert ks.ksort_get_device_error(s) == 0


def test_wave_stats_and_bad_offsets(ks, restore):
    ks.ksort_set_tuning(ks.F32, tile_shape=10, wave_levels=-1)
    n = 1_000_000
    t = _dev(gen.uniform_f32(gen.seed_for(9, 70, 0), n))
    ks.sort_(t)
    st = ks.ksort_get_stats()
    assert st["large_keys"] >= n and st["small_keys"] <= n
    assert st["tiles"] >= st["large_items"] >= 1
    # queue entries: the small items plus large items handed to the queue
    assert st["small_items"] <= st["items_pushed"] <= st["large_items"] + st["small_items"]
    # kernels per call as the library counts them: seed, two per wave level, hand-off,
    # queue, finisher; the queue form: seed, tile passes, finisher; a partition: one
    # (part_kernel) or two (the wave form's count and move)
    ks.ksort_set_tuning(ks.F32, wave_levels=5)
    ks.sort_(t)
    assert ks.ksort_get_stats()["launches"] == 2 * 5 + 4
    ks.ksort_set_tuning(ks.F32, tile_shape=1)
    ks.sort_(t)
    assert ks.ksort_get_stats()["launches"] == 3
    ks.partition_(t)
    assert ks.ksort_get_stats()["launches"] == 1
    ks.ksort_set_tuning(ks.F32, tile_shape=10)
    ks.partition_(t)
    assert ks.ksort_get_stats()["launches"] == 2
    ks.ksort_set_tuning(ks.F32, partition_form=1)  # the ring partition: one launch
    ks.partition_(t)
    assert ks.ksort_get_stats()["launches"] == 1
    ks.ksort_set_tuning(ks.F32, partition_form=-1)
    flat = _dev(gen.uniform_f32(1, 10_000))
    bad = _dev(np.array([0, 6000, 4000, 10_000], np.int64))
    ks.sort_batched_(flat, bad)
    assert ks.ksort_get_device_error() == 6
    good = _dev(np.array([0, 5000, 10_000], np.int64))
    ks.sort_batched_(flat, good)
    assert ks.ksort_get_device_error() == 0
    h = flat.cpu().numpy()
    assert np.all(np.diff(h[:5000]) >= 0) and np.all(np.diff(h[5000:]) >= 0)


def _bits(v):
    """Multiset of bit patterns (uint32 or uint64 view), sorted, as bytes."""
    return np.sort(v.view(np.uint64 if v.dtype.itemsize == 8 else np.uint32)).tobytes()


def _check_partition(ref, ks, code, a, offset=0, in_place=False):
    """One wave-form partition of `a` (placed `offset` keys into a larger device buffer,
    so the start is not 16-byte aligned for offset % 4 != 0) against the oracle: the key
    index, the key, and both side multisets bit for bit."""
    import torch
    n = len(a)
    big = np.zeros(n + offset + 3, a.dtype)
    big[offset:offset + n] = a
    t = _dev(big)
    src = t[offset:offset + n]
    idx = torch.empty(1, dtype=torch.int64, device="cuda")
    if in_place:
        ks.ksort_partition(code, src, n, idx)
        got = src.cpu().numpy().view(a.dtype)
    else:
        dst = torch.empty_like(src)
        ks.ksort_partition_out(code, src, dst, n, idx)
        got = dst.cpu().numpy().view(a.dtype)
        assert src.cpu().numpy().view(a.dtype).tobytes() == a.tobytes()  # input untouched
    assert ks.ksort_get_device_error() == 0
    i = int(idx.item())
    b = a.copy()
    ri, *_ = ref.partition(b)
    assert i == ri
    assert got[i:i + 1].tobytes() == a[:1].tobytes()
    assert _bits(got[:i]) == _bits(b[:ri]) and _bits(got[i + 1:]) == _bits(b[ri + 1:])


@pytest.mark.parametrize("shape", WAVE)
@pytest.mark.parametrize("dtype", list(DTYPES))
def test_wave_partition_split(ref, ks, restore, dtype, shape):
    """Single partitions of the wave form (count, then move): a single warp tile, fewer
    warp tiles than warps, and many warp tiles per warp."""
    code = DTYPES[dtype]
    ks.ksort_set_tuning(code, tile_shape=shape)
    for n in (2, 3, 31, 4097, 100_003, 1_000_001, 7_000_000):
        a = gen.make("uniform", dtype, n, gen.seed_for(9, 80 + shape, n % 1013))
        _check_partition(ref, ks, code, a)
    a = gen.make("uniform", dtype, 250_001, gen.seed_for(9, 90, shape))
    for offset in (1, 2, 3):
        _check_partition(ref, ks, code, a, offset=offset)
    _check_partition(ref, ks, code, a, in_place=True)


def test_wave_partition_alternates_with_part_kernel(ref, ks, restore):
    """Calls of the split partition and of part_kernel interleave on one stream (the
    counts of one and the descriptors of the other share a workspace), including key
    classes the IEEE compare treats specially."""
    for rep in range(6):
        for shape in (10, 1, 12, 3):
            ks.ksort_set_tuning(ks.F32, tile_shape=shape)
            a = gen.make("distinct16" if rep % 2 else "uniform", "f32", 300_007,
                         gen.seed_for(9, 100 + rep, shape))
            _check_partition(ref, ks, ks.F32, a)
    ks.ksort_set_tuning(ks.F64, tile_shape=11)
    rng = np.random.default_rng(5)
    a = rng.standard_normal(200_003) * 10.0 ** rng.integers(-300, 300, 200_003)
    pick = rng.random(len(a)) < 0.2
    a[pick] = rng.choice(np.array([np.nan, -0.0, 0.0, np.inf, -np.inf, 5e-324]), int(pick.sum()))
    for key in (np.nan, -0.0, np.inf, 1.0):
        a[0] = key
        _check_partition(ref, ks, ks.F64, a)


def test_wave_partition_in_graph(ref, ks, restore):
    """The split partition captured in a CUDA graph (the move launch depends on the count
    launch programmatically) and replayed, with the output cleared between replays."""
    import torch
    ks.ksort_set_tuning(ks.F32, tile_shape=10)
    n = 1_000_003
    a = gen.make("uniform", "f32", n, gen.seed_for(9, 110, 0))
    src = _dev(a)
    dst = torch.empty_like(src)
    idx = torch.empty(1, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ks.ksort_reserve_workspace(ks.F32, n, 1, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ks.ksort_partition_out(ks.F32, src, dst, n, idx, stream=s)
    b = a.copy()
    ri, *_ = ref.partition(b)
    for _ in range(3):
        dst.zero_()
        idx.fill_(-1)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert int(idx.item()) == ri
        got = dst.cpu().numpy()
        assert got[ri:ri + 1].tobytes() == a[:1].tobytes()
        assert _bits(got[:ri]) == _bits(b[:ri]) and _bits(got[ri + 1:]) == _bits(b[ri + 1:])
    assert ks.ksort_get_device_error(s) == 0
