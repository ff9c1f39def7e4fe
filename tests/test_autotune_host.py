"""The autotuner's search on the host, with the device work replaced by a cost function
of the tuning the library holds (no GPU): coordinate descent over the axes in order,
the 0.5 % rule for replacing the incumbent, the axes that apply only to some forms, a
search limited to some tile shapes, the cache, and the restore when the chosen tuning
fails its check."""
import sys

import pytest

import paper_1107_3622_gb300 as ks
from paper_1107_3622_gb300 import autotune


def _cost(t):
    """ms of a fake workload: separable, with its minimum at tile shape 3, cutoff 8192,
    finisher CTAs 2 per SM, 512-thread finisher; the wave form is slow, cluster off."""
    c = 10.0
    c += {3: 0.0, 2: 1.0, 1: 2.0}.get(t["tile_shape"], 3.0)
    c += {8192: 0.0, 4096: 0.5}.get(t["cutoff"], 1.0)
    c += 0.0 if t["ctas_per_sm"] == 2 else 0.3
    c += 0.0 if t["finisher_threads"] == 512 else 0.2
    c += 0.0 if t["cluster_sort"] == -1 else 5.0
    c += 0.0 if t["finish_in_tiles"] == -1 else 4.0
    return c


class _FakeRunner:
    bad = False

    def __init__(self, kind, dtype, n, lengths, seed):
        self.kind, self.dtype, self.total = kind, dtype, n or int(sum(lengths))
        self.calls = 0

    def time(self, reps):
        self.calls += 1
        return _cost(ks.ksort_get_tuning(self.dtype))

    def check_sorted(self):
        return not _FakeRunner.bad


@pytest.fixture
def fake(monkeypatch, tmp_path):
    ks.load()
    before = ks.ksort_get_tuning(ks.F32)
    monkeypatch.setenv("KSORT_TUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(autotune, "_Runner", _FakeRunner)
    monkeypatch.setattr(autotune, "device_key", lambda: "fake-device")
    _FakeRunner.bad = False
    autotune.reset(ks.F32)
    yield
    ks.ksort_set_tuning(ks.F32, cutoff=before["cutoff"],
                        ctas_per_sm=before["ctas_per_sm"] or -1,
                        tile_shape=before["tile_shape"], wave_levels=before["wave_levels"],
                        partition_form=before["partition_form"],
                        finish_in_tiles=before["finish_in_tiles"],
                        finisher_threads=before["finisher_threads"],
                        cluster_sort=before["cluster_sort"])


def test_search_finds_the_separable_minimum_and_caches_it(fake):
    e = autotune.autotune("sort", ks.F32, n=1_000_000, reps=1)
    t = e["tuning"]
    assert not e["cached"]
    assert (t["tile_shape"], t["cutoff"], t["ctas_per_sm"], t["finisher_threads"],
            t["cluster_sort"], t["finish_in_tiles"]) == (3, 8192, 2, 512, -1, -1)
    assert e["ms"] == pytest.approx(10.0)
    held = ks.ksort_get_tuning(ks.F32)
    assert held["tile_shape"] == 3 and held["cutoff"] == 8192 and held["finisher_threads"] == 512
    # wave levels are searched only under a wave shape, which never led here
    assert {c["wave_levels"] for c in e["candidates"]} == {-1}
    autotune.reset(ks.F32)
    again = autotune.autotune("sort", ks.F32, n=1_000_000)
    assert again["cached"] and again["tuning"] == t
    assert ks.ksort_get_tuning(ks.F32)["cutoff"] == 8192


def test_incumbent_kept_unless_half_a_percent_faster(fake, monkeypatch):
    # shape 2 is 0.2 % faster than the incumbent shape 3: not enough to replace it
    monkeypatch.setattr(autotune, "SHAPES", (3, 2))
    base = _cost

    def cost(t):
        return base(dict(t, tile_shape=3)) * (0.998 if t["tile_shape"] == 2 else 1.0)

    monkeypatch.setattr(sys.modules[__name__], "_cost", cost)
    ks.ksort_set_tuning(ks.F32, tile_shape=3)
    e = autotune.autotune("sort", ks.F32, n=2_000_000, reps=1, max_rounds=1)
    assert 2 in {c["tile_shape"] for c in e["candidates"]}
    assert e["tuning"]["tile_shape"] == 3


def test_limited_shapes_and_batched_axes(fake):
    lengths = [1_000, 20_000, 300_000]
    e = autotune.autotune("batched", ks.F32, lengths=lengths, reps=1, shapes=(1, 2))
    assert {c["tile_shape"] for c in e["candidates"]} <= {1, 2}
    assert e["tuning"]["tile_shape"] == 2
    # the cluster form is a single-sort axis: never tried for a batch
    assert {c["cluster_sort"] for c in e["candidates"]} == {-1}
    # nor the fused finisher outside tile shape 3
    assert {c["finish_in_tiles"] for c in e["candidates"]} == {-1}
    assert autotune.apply_cached("batched", ks.F32, lengths=lengths) is None
    assert autotune.apply_cached("batched", ks.F32, lengths=lengths, shapes=(1, 2)) is not None


def test_failed_check_restores_the_previous_tuning(fake):
    ks.ksort_set_tuning(ks.F32, tile_shape=1, cutoff=2048)
    _FakeRunner.bad = True
    with pytest.raises(RuntimeError):
        autotune.autotune("sort", ks.F32, n=500_000, reps=1, max_rounds=1)
    t = ks.ksort_get_tuning(ks.F32)
    assert t["tile_shape"] == 1 and t["cutoff"] == 2048
