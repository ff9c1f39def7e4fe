"""Serving form: the admission/batching planner and the Poisson request stream on CPU;
on the GPU, a continuous-batching run whose every result must equal the same request
sorted alone (bit for bit), with batches overlapping on the device."""
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


@pytest.mark.gpu
def test_serving_results_equal_alone_and_overlap():
    import torch
    import paper_1107_3622_gb300 as ks
    ks.load()
    torch.cuda.set_device(0)
    # a burst: 300 requests within ~3 ms, so several batches are in flight at once
    reqs = serving.poisson_requests(300, rate_per_s=100_000.0, lo=1_000, hi=1_000_000,
                                    seed=0x5E7)
    pools = serving.build_pools(reqs)
    srv = serving.Server(slots=4, slot_keys=1 << 24, max_arrays=64)
    res = srv.run(reqs, pools)
    summ = res.summary()
    assert summ["requests"] == 300 and res.keys == sum(r.n for r in reqs)
    assert res.max_in_flight >= 2
    assert len(res.batches) >= 4
    assert all(r.batch >= 0 and math.isfinite(r.done_s) for r in reqs)
    assert (res.latencies_s > -1e-3).all()
    assert summ["p50_ms"] <= summ["p99_ms"]
    for r in reqs:
        got = pools[r.dtype][r.pool_off:r.pool_off + r.n]
        alone = serving.sort_alone(r)
        assert torch.equal(got.view(torch.int32), alone.view(torch.int32)), r.rid
    assert ks.ksort_get_device_error() == 0


@pytest.mark.gpu
def test_serving_matches_oracle_on_sample(ref):
    import torch
    import paper_1107_3622_gb300 as ks
    ks.load()
    reqs = serving.poisson_requests(24, rate_per_s=50_000.0, lo=1_000, hi=200_000, seed=0xA1)
    pools = serving.build_pools(reqs)
    serving.Server(slots=2, slot_keys=1 << 22, max_arrays=16).run(reqs, pools)
    for r in reqs:
        got = pools[r.dtype][r.pool_off:r.pool_off + r.n].cpu().numpy()
        a = serving.request_keys(r, device="cpu").numpy()
        if r.dtype == "u32":
            a, got = a.view(np.uint32).copy(), got.view(np.uint32)
        ref.sort(a)
        assert got.tobytes() == a.tobytes()
