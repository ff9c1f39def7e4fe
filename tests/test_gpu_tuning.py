"""Every tuning the autotuner may pick keeps GPU results bit-identical to the oracle:
each compiled tile shape of the partition passes (sort and first-level partition),
cutoffs at both ends of their range, and a capped finisher. Then the autotuner itself:
it searches, applies its choice, caches it, and a second call reads the cache."""
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
    saved = {c: ks.ksort_get_tuning(c) for c in DTYPES.values()}
    yield
    for c, t in saved.items():
        ks.ksort_set_tuning(c, cutoff=t["cutoff"], ctas_per_sm=t["ctas_per_sm"] or -1,
                            tile_shape=t["tile_shape"], partition_form=t["partition_form"],
                            sort_reserve=t["sort_reserve"], finish_in_tiles=t["finish_in_tiles"],
                            finisher_threads=t["finisher_threads"],
                            cluster_sort=t["cluster_sort"])


def _sort(ks, a):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ks.sort_(t)
    assert ks.ksort_get_device_error() == 0
    return t.cpu().numpy()


def _oracle(ref, a):
    b = a.copy()
    ref.sort(b)
    return b


@pytest.mark.parametrize("shape", list(range(1, 13)))
@pytest.mark.parametrize("dtype", list(DTYPES))
def test_tile_shapes_sort_and_partition(ref, ks, restore, dtype, shape):
    import torch
    code = DTYPES[dtype]
    # single partitions follow the tile shape (part_kernel or the split partition)
    ks.ksort_set_tuning(code, tile_shape=shape, partition_form=-1)
    nt, ipt, form = ks.ksort_tile_shape(code, shape)
    # the keys of one tile pass: the data warps' share (warp roles: two warps load and
    # look back; the ring: one warp loads, one reserves)
    tile = (nt - 64 if form in (1, 2) else nt) * ipt
    assert ks.ksort_tile_keys(code) == tile
    for n in (tile - 1, tile + 1, 3 * tile + 5, 250_003):
        a = gen.make("uniform", dtype, n, gen.seed_for(6, shape, n % 1009))
        assert _sort(ks, a).tobytes() == _oracle(ref, a).tobytes()
        t = torch.from_numpy(a).cuda()
        i = ks.partition_(t)
        b = a.copy()
        ri, *_ = ref.partition(b)
        got = t.cpu().numpy()
        assert i == ri and got[i] == a[0]
        assert np.sort(got[:i]).tobytes() == np.sort(b[:ri]).tobytes()
        assert np.sort(got[i + 1:]).tobytes() == np.sort(b[ri + 1:]).tobytes()


@pytest.mark.parametrize("shape", list(range(1, 13)))
def test_tile_shapes_batched(ref, ks, restore, shape):
    import torch
    ks.ksort_set_tuning(0, tile_shape=shape)
    lengths = gen.batched_lengths(64, 2, 60_000, seed=gen.seed_for(6, 9, shape))
    off = gen.offsets_from_lengths(lengths)
    a = gen.uniform_f32(gen.seed_for(6, 10, shape), int(off[-1]))
    t = torch.from_numpy(a).cuda()
    ks.sort_batched_(t, torch.from_numpy(off).cuda())
    got = t.cpu().numpy()
    assert ks.ksort_get_device_error() == 0
    for r in range(len(lengths)):
        seg = a[off[r]:off[r + 1]]
        assert got[off[r]:off[r + 1]].tobytes() == _oracle(ref, seg).tobytes()


@pytest.mark.parametrize("cutoff,ctas", [(2, 0), (16384, -1), (1024, 1)])
def test_cutoff_and_finisher_extremes(ref, ks, restore, cutoff, ctas):
    for dtype, code in DTYPES.items():
        c = min(cutoff, ks.ksort_max_cutoff(code))
        ks.ksort_set_tuning(code, cutoff=c, ctas_per_sm=ctas)
        for pattern in ("uniform", "distinct16"):
            a = gen.make(pattern, dtype, 40_000, gen.seed_for(6, 11, c))
            assert _sort(ks, a).tobytes() == _oracle(ref, a).tobytes(), (dtype, pattern)


@pytest.mark.parametrize("threads", [256, 512, 1024])
@pytest.mark.parametrize("cutoff", [2, 33, 2048, 16384])
def test_finisher_threads(ref, ks, restore, threads, cutoff):
    """Finisher CTAs of every size, from the smallest cutoff to the largest (where the
    CTA-wide partitions run before the warps take over), on random and duplicate-heavy
    inputs and on batches with empty and one-key arrays."""
    for dtype, code in DTYPES.items():
        c = min(cutoff, ks.ksort_max_cutoff(code))
        ks.ksort_set_tuning(code, cutoff=c, finisher_threads=threads)
        assert ks.ksort_get_tuning(code)["finisher_threads"] == threads
        for pattern in ("uniform", "distinct16", "quantized15"):
            a = gen.make(pattern, dtype, 60_001, gen.seed_for(6, 12, c + threads))
            assert _sort(ks, a).tobytes() == _oracle(ref, a).tobytes(), (dtype, pattern)
    ks.ksort_set_tuning(ks.F32, cutoff=min(cutoff, 16384), finisher_threads=threads)
    lengths = gen.batched_lengths(300, 1, 40_000, seed=gen.seed_for(6, 13, threads))
    lengths[0] = 0
    lengths[7] = 1
    off = gen.offsets_from_lengths(lengths)
    flat = gen.uniform_f32(gen.seed_for(6, 14, threads), int(off[-1]))
    want = flat.copy()
    ref.sort_batched(want, off)
    import torch
    keys = torch.from_numpy(flat.copy()).cuda()
    ks.sort_batched_(keys, torch.from_numpy(off).cuda())
    assert ks.ksort_get_device_error() == 0
    assert keys.cpu().numpy().tobytes() == want.tobytes()


@pytest.mark.parametrize("threads", [512, 1024])
def test_finisher_threads_nan(ks, restore, threads):
    """Items holding a NaN take the level-by-level path with the larger CTA as well."""
    ks.ksort_set_tuning(ks.F32, finisher_threads=threads)
    rng = np.random.default_rng(threads)
    a = rng.random(300_001).astype(np.float32)
    a[rng.random(a.size) < 0.02] = np.nan
    got = _sort(ks, a)
    assert np.sort(got.view(np.uint32)).tobytes() == np.sort(a.view(np.uint32)).tobytes()
    v = got[~np.isnan(got)]
    assert np.all(v[1:] >= v[:-1])


def test_autotuner_searches_applies_and_caches(ks, restore, tmp_path, monkeypatch):
    from paper_1107_3622_gb300 import autotune
    monkeypatch.setenv("KSORT_TUNE_CACHE", str(tmp_path / "tune.json"))
    e = autotune.autotune("sort", ks.F32, n=300_000, reps=2, max_rounds=1)
    assert not e["cached"] and e["ms"] > 0
    t = ks.ksort_get_tuning(ks.F32)
    assert t["tile_shape"] == e["tuning"]["tile_shape"]
    assert t["cutoff"] == e["tuning"]["cutoff"]
    assert len(e["candidates"]) >= len(autotune.SHAPES)
    # a candidate replaces the incumbent only when at least 0.5 % faster
    assert e["ms"] <= min(c["ms"] for c in e["candidates"]) / 0.995 + 1e-9
    autotune.reset(ks.F32)
    e2 = autotune.autotune("sort", ks.F32, n=300_000)
    assert e2["cached"] and e2["tuning"] == e["tuning"]
    assert ks.ksort_get_tuning(ks.F32)["tile_shape"] == e["tuning"]["tile_shape"]
    lengths = gen.batched_lengths(128, 100, 100_000, seed=gen.seed_for(6, 12, 0))
    eb = autotune.autotune("batched", ks.F32, lengths=lengths, reps=2, max_rounds=1)
    assert eb["workload"].startswith("batched:f32:128x")


def test_autotuner_limited_shapes(ks, restore, tmp_path, monkeypatch):
    """A search limited to some tile shapes measures and picks only those, and caches
    its choice apart from an unlimited search of the same workload."""
    from paper_1107_3622_gb300 import autotune
    monkeypatch.setenv("KSORT_TUNE_CACHE", str(tmp_path / "tune.json"))
    lengths = np.array([round(10 ** (3 + 4 * (i + 0.5) / 8)) for i in range(8)], np.int64)
    ks.ksort_set_tuning(ks.F32, tile_shape=12)  # the incumbent lies outside the limit
    e = autotune.autotune("batched", ks.F32, lengths=lengths, reps=2, max_rounds=1,
                          shapes=(1, 2, 3))
    assert {c["tile_shape"] for c in e["candidates"]} <= {1, 2, 3}
    assert e["tuning"]["tile_shape"] in (1, 2, 3)
    assert ks.ksort_get_tuning(ks.F32)["tile_shape"] == e["tuning"]["tile_shape"]
    again = autotune.autotune("batched", ks.F32, lengths=lengths, shapes=(1, 2, 3))
    assert again["cached"] and again["tuning"] == e["tuning"]
    assert autotune.apply_cached("batched", ks.F32, lengths=lengths) is None


def test_autotuner_partition_kind(ks, restore, tmp_path, monkeypatch):
    from paper_1107_3622_gb300 import autotune
    monkeypatch.setenv("KSORT_TUNE_CACHE", str(tmp_path / "tune.json"))
    e = autotune.autotune("partition", ks.F32, n=500_000, reps=2, max_rounds=1)
    assert e["workload"] == "partition:f32:2^19"
    # only the form of the partition is searched for a single partition
    assert {c["cutoff"] for c in e["candidates"]} == {e["tuning"]["cutoff"]}
    # every ring configuration, and the tile shape's own form (-1)
    assert {c["partition_form"] for c in e["candidates"]} == set(autotune.PARTITION_FORMS)
    if e["tuning"]["partition_form"] == -1:
        # then the three CTA shapes of part_kernel and of the split partition
        assert {c["tile_shape"] for c in e["candidates"]} >= {1, 2, 3, 10, 11, 12}
    t = ks.ksort_get_tuning(ks.F32)
    assert t["partition_form"] == e["tuning"]["partition_form"]
    assert t["tile_shape"] == e["tuning"]["tile_shape"]


@pytest.mark.parametrize("reserve", [-1, 1])
@pytest.mark.parametrize("shape", [1, 2, 3, 10])
@pytest.mark.parametrize("dtype", list(DTYPES))
def test_sort_offsets_by_reservation_or_lookback(ref, ks, restore, dtype, shape, reserve):
    """Tile passes that take their output ranges by reservation (the order of tiles'
    runs follows completion) and by look-back (tile order) both sort bit for bit as the
    oracle does, across tile edges, presorted input and duplicate-heavy input."""
    code = DTYPES[dtype]
    ks.ksort_set_tuning(code, tile_shape=shape, sort_reserve=reserve)
    assert ks.ksort_get_tuning(code)["sort_reserve"] == reserve
    for pattern, n in (("uniform", 300_007), ("uniform", 2_000_003), ("sorted", 40_000),
                       ("distinct16", 200_001), ("quantized15", 1_000_000)):
        a = gen.make(pattern, dtype, n, gen.seed_for(6, 20 + shape, n % 997))
        assert _sort(ks, a).tobytes() == _oracle(ref, a).tobytes(), (pattern, n)
