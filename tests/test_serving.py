"""Serving form: the admission/batching planner, the HBM arena and the Poisson request
stream on CPU; on the GPU, a continuous-batching run (keys copied in from page-locked
host memory and back) whose every result must equal the same request sorted alone (bit
for bit), with batches overlapping on the device, also under an HBM budget small enough
to refuse admissions."""
import math

import numpy as np
import pytest

from paper_1107_3622_gb300 import serving


def _reqs_with_offsets(reqs):
    off = {"f32": 0, "u32": 0}
    for r in reqs:
        r.pool_off = off[r.dtype]
        off[r.dtype] += r.n
    return reqs


def test_poisson_stream_shape():
    reqs = serving.poisson_requests(20_000, rate_per_s=1000.0)
    arr = np.array([r.arrival_s for r in reqs])
    gaps = np.diff(arr)
    assert arr[0] == 0.0 and (gaps >= 0).all()
    assert abs(gaps.mean() - 1e-3) < 5e-5          # exponential gaps, mean 1/rate
    assert abs(np.median(gaps) - math.log(2) * 1e-3) < 5e-5
    n = np.array([r.n for r in reqs])
    assert n.min() >= 1_000 and n.max() <= 10_000_000
    # log-uniform: ln n is uniform on [ln 1e3, ln 1e7]
    ln = np.log(n)
    assert abs(ln.mean() - (math.log(1e3) + math.log(1e7)) / 2) < 0.05
    frac_f32 = np.mean([r.dtype == "f32" for r in reqs])
    assert 0.48 < frac_f32 < 0.52
    assert abs(n.mean() - serving.mean_length()) / serving.mean_length() < 0.05
    assert len({r.seed for r in reqs}) == len(reqs)


def test_planner_fifo_contiguous_and_bounded():
    reqs = _reqs_with_offsets(serving.poisson_requests(400, 100.0, lo=10, hi=5000))
    p = serving.Planner(slot_keys=20_000, max_arrays=16)
    for r in reqs:
        p.arrive(r)
    seen = []
    while p.waiting():
        b = p.next_batch()
        assert 1 <= len(b.reqs) <= 16 and b.total <= 20_000
        assert all(r.dtype == b.dtype for r in b.reqs)
        assert b.total == sum(r.n for r in b.reqs)
        # one contiguous range of the type's pool, in arrival order
        pos = b.base
        for r in b.reqs:
            assert r.pool_off == pos
            pos += r.n
            assert r.batch == b.bid
        seen.extend(r.rid for r in b.reqs)
    assert sorted(seen) == list(range(400))


def test_planner_serves_oldest_type_first():
    reqs = _reqs_with_offsets([
        serving.Request(0, 0.0, "u32", 10, 1), serving.Request(1, 0.1, "f32", 10, 2),
        serving.Request(2, 0.2, "u32", 10, 3)])
    p = serving.Planner(slot_keys=15, max_arrays=8)
    for r in reqs:
        p.arrive(r)
    order = []
    while p.waiting():
        order.append([r.rid for r in p.next_batch().reqs])
    assert order == [[0], [1], [2]]  # capacity 15 admits one 10-key request per batch


def test_planner_rejects_oversized_and_gaps():
    p = serving.Planner(slot_keys=100, max_arrays=4)
    with pytest.raises(ValueError):
        p.arrive(serving.Request(0, 0.0, "f32", 101, 1))
    p.arrive(serving.Request(1, 0.0, "f32", 10, 1, pool_off=0))
    with pytest.raises(ValueError):
        p.arrive(serving.Request(2, 0.0, "f32", 10, 1, pool_off=11))


def test_arena_first_fit_merges_and_reuses():
    a = serving.Arena(4096, align=256)
    x = a.alloc(1)        # rounds up to one 256-byte block
    y = a.alloc(1000)     # 1024
    z = a.alloc(512)
    assert (x, y, z) == (0, 256, 1280)
    assert a.in_use == 256 + 1024 + 512 and a.largest_free() == 4096 - 1792
    assert a.alloc(4096) is None
    a.free(y)             # a hole of 1024 between x and z
    assert a.alloc(1024) == 256  # first fit takes the hole again
    a.free(256)
    a.free(x)
    a.free(z)             # every block back: one free block spanning the arena
    assert a.in_use == 0 and a.blocks() == 0 and a.largest_free() == 4096
    assert a.peak_in_use == 1792
    with pytest.raises(KeyError):
        a.free(z)


def test_arena_random_alloc_free_invariants():
    """Random traffic: blocks never overlap, stay aligned and inside the arena, and the
    free space plus the blocks in use always add up to the arena."""
    rng = np.random.default_rng(3622)
    a = serving.Arena(1 << 20, align=256)
    live = {}
    for step in range(4000):
        if live and (rng.random() < 0.45 or len(live) > 40):
            off = int(rng.choice(list(live)))
            a.free(off)
            del live[off]
        else:
            n = int(rng.integers(1, 60_000))
            off = a.alloc(n)
            if off is None:
                assert a.largest_free() < serving.align_up(n, 256)
                continue
            assert off % 256 == 0 and off + n <= a.size
            live[off] = serving.align_up(n, 256)
        spans = sorted(live.items())
        for (o1, l1), (o2, _) in zip(spans, spans[1:]):
            assert o1 + l1 <= o2
        assert a.in_use == sum(live.values())
        assert a.in_use + sum(a._free_len) == a.size
    for off in list(live):
        a.free(off)
    assert a.largest_free() == a.size


def test_planner_budget_refuses_then_admits_after_completion():
    """A byte budget of 4096 B (1024 four-byte keys): the first batch takes 600 keys,
    the next request (600 keys, 2400 B) does not fit the 1600 B left, so nothing is
    admitted (a refusal) until the first batch completes and gives its buffer back."""
    reqs = _reqs_with_offsets([
        serving.Request(0, 0.0, "f32", 600, 1), serving.Request(1, 0.1, "f32", 600, 2),
        serving.Request(2, 0.2, "u32", 100, 3)])
    p = serving.Planner(slot_keys=1000, max_arrays=8, budget_bytes=4096)
    for r in reqs:
        p.arrive(r)
    b0 = p.next_batch()
    assert [r.rid for r in b0.reqs] == [0] and b0.nbytes == 2400 and b0.dev_off == 0
    assert p.arena.in_use == serving.align_up(2400)
    # request 1 is the oldest waiting: it does not fit, and the younger u32 request
    # behind it is not admitted ahead of it either
    assert p.next_batch() is None and p.refusals == 1 and p.waiting() == 2
    p.complete(b0)
    assert p.arena.in_use == 0 and b0.dev_off == -1
    b1 = p.next_batch()
    assert [r.rid for r in b1.reqs] == [1] and b1.dev_off == 0
    b2 = p.next_batch()     # 400 B fit beside b1
    assert [r.rid for r in b2.reqs] == [2] and b2.dev_off == serving.align_up(2400)
    assert p.arena.peak_in_use == serving.align_up(2400) + serving.align_up(400)
    p.complete(b1)
    p.complete(b2)
    assert p.arena.in_use == 0 and not p.waiting()


def test_planner_budget_trims_batch_to_free_block():
    """A batch takes the FIFO prefix that fits the largest free block of the arena."""
    reqs = _reqs_with_offsets([serving.Request(i, 0.01 * i, "f32", 100, i) for i in range(10)])
    p = serving.Planner(slot_keys=10_000, max_arrays=64, budget_bytes=2048)
    for r in reqs:
        p.arrive(r)
    b = p.next_batch()
    assert [r.rid for r in b.reqs] == [0, 1, 2, 3, 4]   # 5 x 400 B = 2000 B <= 2048 B
    assert p.next_batch() is None
    p.complete(b)
    assert [r.rid for r in p.next_batch().reqs] == [5, 6, 7, 8, 9]


def test_planner_rejects_request_over_budget():
    p = serving.Planner(slot_keys=10_000, max_arrays=4, budget_bytes=1024)
    with pytest.raises(ValueError):
        p.arrive(serving.Request(0, 0.0, "u32", 257, 1))   # 1028 B > 1024 B
    p.arrive(serving.Request(1, 0.0, "u32", 256, 1))


def _check_alone(reqs, pools):
    import torch
    for r in reqs:
        got = pools.keys(r).cuda()
        alone = serving.sort_alone(r)
        assert torch.equal(got.view(torch.int32), alone.view(torch.int32)), r.rid


@pytest.mark.gpu
def test_serving_results_equal_alone_and_overlap():
    import torch
    import paper_1107_3622_gb300 as ks
    ks.load()
    torch.cuda.set_device(0)
    # a burst: 300 requests within ~3 ms, so several batches are in flight at once
    reqs = serving.poisson_requests(300, rate_per_s=100_000.0, lo=1_000, hi=1_000_000,
                                    seed=0x5E7)
    with serving.build_pools(reqs) as pools:
        srv = serving.Server(slots=4, slot_keys=1 << 24, max_arrays=64)
        res = srv.run(reqs, pools)
        summ = res.summary()
        assert summ["requests"] == 300 and res.keys == sum(r.n for r in reqs)
        assert res.max_in_flight >= 2
        assert len(res.batches) >= 4
        assert all(r.batch >= 0 and math.isfinite(r.done_s) for r in reqs)
        assert all(r.arrival_s <= r.admit_s <= r.done_s + 1e-3 for r in reqs)
        assert (res.latencies_s > -1e-3).all()
        assert summ["p50_ms"] <= summ["p99_ms"]
        assert summ["blocks_outstanding"] == 0
        assert 0 < summ["peak_bytes_in_use"] <= summ["budget_bytes"]
        assert summ["h2d_bytes"] == 4 * res.keys
        _check_alone(reqs, pools)
        srv.close()
    assert ks.ksort_get_device_error() == 0


@pytest.mark.gpu
def test_serving_tight_budget_refuses_and_stays_identical():
    """An arena of 8 MiB (2M keys) against requests of up to 1M keys on four slots:
    admissions are refused while buffers are out, every request is still served, and
    every result equals the request sorted alone."""
    import torch
    import paper_1107_3622_gb300 as ks
    ks.load()
    torch.cuda.set_device(0)
    reqs = serving.poisson_requests(200, rate_per_s=200_000.0, lo=10_000, hi=1_000_000,
                                    seed=0xB0D)
    with serving.build_pools(reqs) as pools:
        srv = serving.Server(slots=4, slot_keys=1 << 21, max_arrays=64, budget_bytes=8 << 20)
        res = srv.run(reqs, pools)
        summ = res.summary()
        assert summ["budget_bytes"] == 8 << 20
        assert summ["refusals"] > 0
        assert summ["peak_bytes_in_use"] <= 8 << 20
        assert summ["blocks_outstanding"] == 0
        assert all(r.batch >= 0 for r in reqs)
        _check_alone(reqs, pools)
        srv.close()
    assert ks.ksort_get_device_error() == 0


@pytest.mark.gpu
def test_serving_matches_oracle_on_sample(ref):
    import paper_1107_3622_gb300 as ks
    ks.load()
    reqs = serving.poisson_requests(24, rate_per_s=50_000.0, lo=1_000, hi=200_000, seed=0xA1)
    with serving.build_pools(reqs) as pools:
        srv = serving.Server(slots=2, slot_keys=1 << 22, max_arrays=16)
        srv.run(reqs, pools)
        for r in reqs:
            got = pools.keys(r).numpy().copy()
            a = serving.request_keys(r, device="cpu").numpy()
            if r.dtype == "u32":
                a, got = a.view(np.uint32).copy(), got.view(np.uint32)
            ref.sort(a)
            assert got.tobytes() == a.tobytes()
        srv.close()
