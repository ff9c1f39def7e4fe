"""Phase timing (ksort_set_phase_timing / ksort_get_phase_times): a timed sort reports
its seed, partition-pass and finisher durations, a timed partition its one phase, each
within the call's own CUDA-event time; graph-captured calls are not timed; disabling
stops the recording."""
import numpy as np
import pytest

import ksort_inputs as gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ks():
    import torch
    import paper_1107_3622_gb300 as ks
    ks.load()
    torch.cuda.set_device(0)
    return ks


@pytest.fixture
def timing(ks):
    saved = ks.ksort_get_tuning(ks.F32)
    ks.ksort_set_phase_timing(True)
    yield
    ks.ksort_set_phase_timing(False)
    ks.ksort_set_tuning(ks.F32, cutoff=saved["cutoff"], ctas_per_sm=saved["ctas_per_sm"] or -1,
                        tile_shape=saved["tile_shape"], wave_levels=saved["wave_levels"])


def _timed(fn):
    import torch
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


@pytest.mark.parametrize("shape", [1, 10])
def test_sort_and_partition_phases(ks, timing, shape):
    import torch
    ks.ksort_set_tuning(ks.F32, tile_shape=shape)
    a = gen.uniform_f32(gen.seed_for(12, 1, shape), 2_000_000)
    t = torch.from_numpy(a).cuda()
    ms = _timed(lambda: ks.sort_(t))
    ph = ks.ksort_get_phase_times()
    assert len(ph) == 3 and min(ph) >= 0.0
    assert ph[1] > 0.0 and ph[2] > 0.0  # partition passes and finisher both ran
    assert sum(ph) <= ms * 1.02 + 0.01
    assert bool((t[1:] >= t[:-1]).all())
    src = torch.from_numpy(a).cuda()
    dst = torch.empty_like(src)
    idx = torch.empty(1, dtype=torch.int64, device="cuda")
    ms = _timed(lambda: ks.ksort_partition_out(ks.F32, src, dst, len(a), idx))
    ph = ks.ksort_get_phase_times()
    assert len(ph) == 1 and 0.0 < ph[0] <= ms * 1.02 + 0.01
    assert int(idx.item()) == int((a[1:] < a[0]).sum())
    assert ks.ksort_get_device_error() == 0


def test_capture_and_disable_are_not_timed(ks, timing):
    import torch
    a = gen.uniform_f32(gen.seed_for(12, 2, 0), 300_000)
    s = torch.cuda.Stream()
    t = torch.from_numpy(a).cuda()
    with torch.cuda.stream(s):
        ks.ksort_reserve_workspace(ks.F32, len(a), 1, stream=s)
    torch.cuda.synchronize()
    assert ks.ksort_get_phase_times(s) == []  # nothing timed on this stream yet
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ks.sort_(t, stream=s)
    t.copy_(torch.from_numpy(a).cuda())
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert ks.ksort_get_phase_times(s) == []  # the captured call recorded no events
    assert np.array_equal(t.cpu().numpy(), np.sort(a))
    ks.ksort_set_phase_timing(False)
    t.copy_(torch.from_numpy(a).cuda())
    torch.cuda.synchronize()
    ks.sort_(t, stream=s)
    assert ks.ksort_get_phase_times(s) == []
    assert ks.ksort_get_device_error(s) == 0


def test_history_of_back_to_back_calls(ks, timing):
    """Calls enqueued back to back without a sync keep their own phases (the last 64
    timed calls are kept); a partition between sorts shows as its one phase."""
    import torch
    ks.ksort_set_tuning(ks.F32, tile_shape=1)
    s = torch.cuda.Stream()
    a = gen.uniform_f32(gen.seed_for(12, 3, 0), 1_000_000)
    bufs = [torch.from_numpy(a).cuda() for _ in range(3)]
    dst = torch.empty_like(bufs[0])
    idx = torch.empty(1, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    ks.sort_(bufs[0], stream=s)
    ks.ksort_partition_out(ks.F32, bufs[1], dst, len(a), idx, stream=s)
    ks.sort_(bufs[2], stream=s)
    h = ks.ksort_get_phase_history(s, 3)
    assert [len(p) for p in h] == [3, 1, 3]
    assert all(min(p) >= 0.0 for p in h) and h[0][1] > 0.0 and h[1][0] > 0.0
    assert len(ks.ksort_get_phase_history(s, 64)) == 3  # only what was timed on s
    for _ in range(70):
        ks.ksort_partition_out(ks.F32, bufs[1], dst, len(a), idx, stream=s)
    assert len(ks.ksort_get_phase_history(s, 100)) == 64
    assert ks.ksort_get_device_error(s) == 0
