"""The seeded input generators (SplitMix64) against the published stream and
against each other (numpy vs torch)."""
import numpy as np
import pytest

import ksort_inputs as gen


def test_splitmix64_published_vector():
    # First outputs for seed 1234567 of the reference splitmix64.c (Vigna), as widely
    # used to check SplitMix64 implementations.
    assert list(map(int, gen.splitmix64(1234567, 5))) == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


def test_stream_offsets_are_consistent():
    full = gen.splitmix64(77, 100)
    assert np.array_equal(full[40:], gen.splitmix64(77, 60, start=40))


@pytest.mark.parametrize("dtype", ["f32", "f64", "u32"])
def test_torch_matches_numpy(dtype):
    a = gen.uniform_torch(dtype, gen.seed_for(1, 2, 3), 5000, chunk=777).numpy()
    if dtype == "u32":
        a = a.view(np.uint32)
    b = gen.make("uniform", dtype, 5000, gen.seed_for(1, 2, 3))
    assert a.tobytes() == b.tobytes()


def test_value_ranges():
    f = gen.uniform_f32(5, 100_000)
    assert f.dtype == np.float32 and f.min() >= 0 and f.max() < 1
    assert not np.any(np.signbit(f)) and not np.any(np.isnan(f))
    d = gen.uniform_f64(5, 100_000)
    assert d.min() >= 0 and d.max() < 1
    assert set(np.unique(gen.distinct16_u32(5, 10_000)).tolist()) == set(range(16))


def test_patterns():
    s = gen.make("sorted", "f32", 1000, 1)
    assert np.all(np.diff(s) >= 0)
    r = gen.make("reverse", "u32", 1000, 1)
    assert np.all(np.diff(r.astype(np.int64)) <= 0)
    o = gen.make("organ_pipe", "f32", 7, 0)
    assert o.tolist() == [0, 1, 2, 3, 2, 1, 0]
    q = gen.make("quantized15", "f32", 200_000, 3)
    assert q.min() >= 0 and q.max() < 1 and len(np.unique(q)) <= 32768
    assert np.all(q * 32768 == np.floor(q * 32768))        # on the 2**-15 grid
    u = gen.uniform_f64(3, 200_000)                          # the same stream, truncated
    assert np.array_equal(q, (np.floor(u * 32768) / 32768).astype(np.float32))


def test_batched_lengths():
    L = gen.batched_lengths()
    assert len(L) == 4096 and L.min() >= 100 and L.max() <= 1_000_000
    off = gen.offsets_from_lengths(L)
    assert off[0] == 0 and off[-1] == L.sum() and np.all(np.diff(off) == L)
    # log-uniform on [100, 1e6]: E[len] = (1e6 - 100) / ln(1e4) ~ 108,561 and the
    # standard deviation of one length is ~2.06e5, so the mean of 4096 is within
    # ~3.2e3 (1 sigma); allow 4 sigma.
    assert abs(L.mean() - 108_561) < 4 * 3_220
