"""The fused finisher (tuning finish_in_tiles, tile shape 3): the CTAs of the tile passes
take small sub-arrays while enough other CTAs wait for future tiles; the finisher launch
that follows takes the rest of the small list.
Every sort must stay bit-identical to the oracle for each park threshold, key type and
input class, in single sorts and batches; the statistics must still count every key, and
graph replay and two streams at once must work."""
import numpy as np
import pytest

import ksort_inputs as gen

pytestmark = pytest.mark.gpu

DTYPES = {"f32": 0, "f64": 1, "u32": 2}
PARKS = [1, 8, 64, 4096]


@pytest.fixture(scope="module")
def ks():
    import torch
    import paper_1107_3622_gb300 as ks
    ks.load()
    torch.cuda.set_device(0)
    return ks


@pytest.fixture
def fused(ks):
    """Tile shape 3 with the given park threshold for every dtype; restored afterwards."""
    saved = {c: ks.ksort_get_tuning(c) for c in DTYPES.values()}

    def use(park, code=None):
        for c in (DTYPES.values() if code is None else [code]):
            ks.ksort_set_tuning(c, tile_shape=3, finish_in_tiles=park)
    yield use
    for c, t in saved.items():
        ks.ksort_set_tuning(c, cutoff=t["cutoff"], tile_shape=t["tile_shape"],
                            finish_in_tiles=t["finish_in_tiles"],
                            spin_limit_ms=t["spin_limit_ms"])


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


def test_tuning_roundtrip(ks, fused):
    fused(16)
    for code in DTYPES.values():
        assert ks.ksort_get_tuning(code)["finish_in_tiles"] == 16
    fused(-1)
    for code in DTYPES.values():
        assert ks.ksort_get_tuning(code)["finish_in_tiles"] == -1


@pytest.mark.parametrize("park", PARKS)
@pytest.mark.parametrize("dtype", list(DTYPES))
def test_fused_sort_sizes(ref, ks, fused, dtype, park):
    code = DTYPES[dtype]
    fused(park, code)
    cut = ks.ksort_get_tuning(code)["cutoff"]
    tile = ks.ksort_tile_keys(code)
    for n in (2, cut, cut + 1, tile + 1, 3 * tile + 7, 100_003, 1_000_003):
        a = gen.make("uniform", dtype, n, gen.seed_for(13, park % 97, n % 1009))
        assert _sort(ks, code, a).tobytes() == _oracle(ref, a).tobytes(), n


@pytest.mark.parametrize("pattern", ["sorted", "reverse", "distinct16", "organ_pipe",
                                     "quantized15"])
def test_fused_stress_patterns(ref, ks, fused, pattern):
    """Degenerate orders make long chains of one-sided partitions (few small items until
    the end); duplicate runs give many equal keys on the >= side. Sizes stay within the
    look-back arena of tile shape 3 (16 distinct values peel one key per level off each
    run of equal keys, so their tile count grows with the square of the run length)."""
    fused(8)
    for dtype, code in DTYPES.items():
        n = {"sorted": 60_000, "reverse": 60_000, "organ_pipe": 60_000,
             "distinct16": 150_000}.get(pattern, 600_000)
        a = gen.make(pattern, dtype, n, gen.seed_for(13, 40, n))
        assert _sort(ks, code, a).tobytes() == _oracle(ref, a).tobytes(), (dtype, pattern)


def test_fused_full_size(ref, ks, fused):
    """The 7e6-key float32 size that bench.py times."""
    fused(8, ks.F32)
    a = gen.uniform_f32(gen.seed_for(1, 6, 0), 7_000_000)
    assert _sort(ks, ks.F32, a).tobytes() == _oracle(ref, a).tobytes()


def test_fused_nan_is_a_permutation(ks, fused):
    """Items holding a NaN take the finisher's level-by-level path inside the tile
    kernel: the result is a permutation with the non-NaN keys in ascending order."""
    fused(8, ks.F32)
    rng = np.random.default_rng(3622)
    a = rng.random(500_001).astype(np.float32)
    a[rng.random(a.size) < 0.01] = np.nan
    got = _sort(ks, ks.F32, a)
    assert np.sort(got.view(np.uint32)).tobytes() == np.sort(a.view(np.uint32)).tobytes()
    v = got[~np.isnan(got)]
    assert np.all(v[1:] >= v[:-1])


@pytest.mark.parametrize("park", [1, 64])
def test_fused_batched(ref, ks, fused, park):
    fused(park, ks.F32)
    lengths = gen.batched_lengths(600, 2, 300_000, seed=gen.seed_for(13, 60, park))
    lengths[5] = 0
    lengths[11] = 1
    off = gen.offsets_from_lengths(lengths)
    flat = gen.uniform_f32(gen.seed_for(13, 61, park), int(off[-1]))
    want = flat.copy()
    ref.sort_batched(want, off)
    keys = _dev(flat)
    ks.sort_batched_(keys, _dev(off))
    assert ks.ksort_get_device_error() == 0
    assert keys.cpu().numpy().tobytes() == want.tobytes()


def test_fused_stats_and_phases(ks, fused):
    """Under look-back tile offsets (the recursion then depends on the input alone) the
    fused sort counts the same items and keys as with the finisher launch alone, and the
    same result; both make three launches (seed, tile passes, finisher)."""
    import torch
    pristine = _dev(gen.uniform_f32(gen.seed_for(13, 70, 0), 2_000_000))
    ks.ksort_set_tuning(ks.F32, sort_reserve=-1)
    got = {}
    try:
        for park in (-1, 8):
            fused(park, ks.F32)
            t = pristine.clone()
            ks.ksort_set_phase_timing(True)
            ks.sort_(t)
            torch.cuda.synchronize()
            ph = ks.ksort_get_phase_times()
            ks.ksort_set_phase_timing(False)
            got[park] = (ks.ksort_get_stats(), ph, t)
    finally:
        ks.ksort_set_tuning(ks.F32, sort_reserve=1)
    for k in ("tiles", "large_items", "large_keys", "small_items", "small_keys"):
        assert got[-1][0][k] == got[8][0][k], k
    assert got[8][0]["small_keys"] > 0
    assert got[-1][0]["launches"] == 3 and got[8][0]["launches"] == 3
    assert len(got[8][1]) == 3
    assert torch.equal(got[-1][2], got[8][2])


def test_fused_graph_replay(ref, ks, fused):
    import torch
    fused(8, ks.F32)
    n = 1_500_001
    s = torch.cuda.Stream()
    keys = torch.empty(n, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(s):
        ks.ksort_reserve_workspace(ks.F32, n, 1, stream=s)
        keys.copy_(torch.from_numpy(gen.uniform_f32(1, n)))
        ks.ksort_sort(ks.F32, keys, n, stream=s)  # set-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ks.ksort_sort(ks.F32, keys, n, stream=s)
    for rep in range(3):
        a = gen.uniform_f32(gen.seed_for(13, 80, rep), n)
        keys.copy_(torch.from_numpy(a))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert ks.ksort_get_device_error(s) == 0
        assert keys.cpu().numpy().tobytes() == _oracle(ref, a).tobytes()


def test_fused_two_streams_at_once(ref, ks, fused):
    """Two fused sorts overlap on two streams, each with a grid that fills the GPU
    alone; a CTA only ever waits for tiles that running CTAs hold, so both finish."""
    import torch
    fused(8, ks.F32)
    ks.ksort_set_tuning(ks.F32, spin_limit_ms=500)
    arrays = [gen.uniform_f32(gen.seed_for(13, 90, r), 3_000_017) for r in range(2)]
    streams = [torch.cuda.Stream() for _ in arrays]
    bufs = [_dev(a) for a in arrays]
    for s, b in zip(streams, bufs):
        ks.ksort_reserve_workspace(ks.F32, b.numel(), 1, stream=s)
    torch.cuda.synchronize()
    for s, b in zip(streams, bufs):
        ks.ksort_sort(ks.F32, b, b.numel(), stream=s)
    torch.cuda.synchronize()
    for s, b, a in zip(streams, bufs, arrays):
        assert ks.ksort_get_device_error(s) == 0
        assert b.cpu().numpy().tobytes() == _oracle(ref, a).tobytes()
