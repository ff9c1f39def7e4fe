"""Whole-item CTAs of the register form's work queue (tuning medium_tiles): a sub-array of
2 .. medium_tiles tile passes takes one ticket, and the CTA that draws it counts every
tile and then moves them with the prefixes it has summed itself, without look-back.
Every result must stay byte-identical to the oracle for each limit, key type and input
class (random, duplicate-heavy, presorted), in single sorts, batches and the wave form's
queue. (Single partitions run part_kernel or the split partition, never the queue.)"""
import numpy as np
import pytest

import ksort_inputs as gen

pytestmark = pytest.mark.gpu

DTYPES = {"f32": 0, "f64": 1, "u32": 2}


@pytest.fixture(scope="module")
def ks():
    import torch
    import paper_1107_3622_gb300 as ks
    ks.load()
    torch.cuda.set_device(0)
    return ks


@pytest.fixture
def restore(ks):
    """Whole-item CTAs lay tiles out as the multi-tile passes do in tile order, so this
    module compares them under the look-back form of the tile passes (sort_reserve -1),
    whose layout depends on the input alone."""
    saved = {c: ks.ksort_get_tuning(c) for c in DTYPES.values()}
    for c in DTYPES.values():
        ks.ksort_set_tuning(c, sort_reserve=-1)
    yield
    for c, t in saved.items():
        ks.ksort_set_tuning(c, cutoff=t["cutoff"], ctas_per_sm=t["ctas_per_sm"] or -1,
                            tile_shape=t["tile_shape"], wave_levels=t["wave_levels"],
                            medium_tiles=t["medium_tiles"], sort_reserve=t["sort_reserve"])


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


def test_medium_tuning_roundtrip(ks, restore):
    for code in DTYPES.values():
        ks.ksort_set_tuning(code, medium_tiles=4)
        assert ks.ksort_get_tuning(code)["medium_tiles"] == 4
        ks.ksort_set_tuning(code, medium_tiles=-1)
        assert ks.ksort_get_tuning(code)["medium_tiles"] == -1


@pytest.mark.parametrize("medium", [2, 4, 16])
@pytest.mark.parametrize("shape", [1, 2, 3, 10])
@pytest.mark.parametrize("dtype", list(DTYPES))
def test_medium_sort_sizes(ref, ks, restore, dtype, shape, medium):
    code = DTYPES[dtype]
    ks.ksort_set_tuning(code, tile_shape=shape, medium_tiles=medium, wave_levels=-1)
    tile = ks.ksort_tile_keys(code)
    cut = ks.ksort_get_tuning(code)["cutoff"]
    # just above the cutoff, one to medium + 1 tiles (unaligned starts inside), and sizes
    # whose recursion passes through every class
    for n in (cut + 1, tile + 1, 2 * tile - 1, medium * tile, medium * tile + 7,
              (medium + 1) * tile + 3, 250_003, 2_000_000):
        a = gen.make("uniform", dtype, n, gen.seed_for(11, shape * 17 + medium, n % 1009))
        assert _sort(ks, code, a).tobytes() == _oracle(ref, a).tobytes(), n


@pytest.mark.parametrize("pattern", ["sorted", "reverse", "distinct16", "organ_pipe",
                                     "quantized15"])
def test_medium_stress_patterns(ref, ks, restore, pattern):
    """Degenerate orders make every medium item a one-sided partition; duplicate runs
    put many keys equal to the item's key on the >= side."""
    for dtype, code in DTYPES.items():
        ks.ksort_set_tuning(code, tile_shape=1, medium_tiles=16)
        n = 60_000 if pattern in ("sorted", "reverse", "organ_pipe") else 500_000
        a = gen.make(pattern, dtype, n, gen.seed_for(11, 40, n))
        assert _sort(ks, code, a).tobytes() == _oracle(ref, a).tobytes(), (dtype, pattern)


def test_medium_f64_specials(ref, ks, restore):
    """Every class of double in medium items. Without NaN and -0 the sorted array is
    unique: bit-identical to the oracle. With them the order depends on element order
    (Step 3's compare is false on both sides of a NaN), so the result must be a
    permutation of the input and byte-identical to the same sort run tile by tile
    (a whole-item CTA lays out every tile exactly as the multi-tile passes do)."""
    import torch
    rng = np.random.default_rng(17)
    n = 400_003
    pool = np.array([0.0, np.inf, -np.inf, 5e-324, -5e-324, 2.2250738585072014e-308,
                     1.7976931348623157e308, -1.7976931348623157e308, 1.0, -1.0])
    a = rng.standard_normal(n) * 10.0 ** rng.integers(-300, 300, n)
    pick = rng.random(n) < 0.2
    a[pick] = rng.choice(pool, int(pick.sum()))
    ks.ksort_set_tuning(ks.F64, tile_shape=1, medium_tiles=8)
    assert _sort(ks, ks.F64, a).tobytes() == _oracle(ref, a).tobytes()
    pick = rng.random(n) < 0.1
    a[pick] = rng.choice(np.array([np.nan, -0.0]), int(pick.sum()))
    got = {}
    for m in (-1, 8):
        ks.ksort_set_tuning(ks.F64, medium_tiles=m)
        got[m] = _sort(ks, ks.F64, a)
        torch.cuda.synchronize()
    assert np.sort(got[8].view(np.uint64)).tobytes() == np.sort(a.view(np.uint64)).tobytes()
    assert got[8].tobytes() == got[-1].tobytes()


@pytest.mark.parametrize("shape", [1, 10])
def test_medium_batched(ref, ks, restore, shape):
    ks.ksort_set_tuning(ks.F32, tile_shape=shape, medium_tiles=16, wave_levels=-1)
    lengths = gen.batched_lengths(400, 2, 120_000, seed=gen.seed_for(11, 60, shape))
    lengths[3] = 0
    lengths[9] = 1
    off = gen.offsets_from_lengths(lengths)
    flat = gen.uniform_f32(gen.seed_for(11, 61, shape), int(off[-1]))
    want = flat.copy()
    ref.sort_batched(want, off)
    keys = _dev(flat)
    ks.sort_batched_(keys, _dev(off))
    assert ks.ksort_get_device_error() == 0
    assert keys.cpu().numpy().tobytes() == want.tobytes()


def test_medium_counts_tiles(ks, restore):
    """A medium item still counts every tile pass in the statistics: the totals of the
    same sort with and without whole-item CTAs agree."""
    import torch
    ks.ksort_set_tuning(ks.F32, tile_shape=1)
    pristine = _dev(gen.uniform_f32(gen.seed_for(11, 70, 0), 1_000_000))
    got = {}
    for m in (-1, 16):
        ks.ksort_set_tuning(ks.F32, medium_tiles=m)
        t = pristine.clone()
        ks.sort_(t)
        torch.cuda.synchronize()
        got[m] = ks.ksort_get_stats()
    for k in ("tiles", "large_items", "large_keys", "small_items", "small_keys"):
        assert got[-1][k] == got[16][k], k
