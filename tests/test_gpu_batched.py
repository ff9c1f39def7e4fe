"""GPU: batched sort (many arrays, one launch) against the oracle and against the
per-array path; CUDA-graph capture and replay; device-side error reporting."""
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


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


RAGGED = [0, 1, 2, 3, 4096, 4097, 10_000, 100, 0, 1, 8193, 65_536, 2, 5, 300_000]


@pytest.mark.parametrize("dtype", ["f32", "f64", "u32"])
def test_batched_ragged_matches_oracle(ref, ks, dtype):
    off = gen.offsets_from_lengths(np.array(RAGGED, np.int64))
    flat = gen.make("uniform", dtype, int(off[-1]), gen.seed_for(2, 1, 0))
    t = _dev(flat)
    ks.sort_batched_(t, _dev(off))
    assert ks.ksort_get_device_error() == 0
    want = flat.copy()
    ref.sort_batched(want, off)
    assert t.cpu().numpy().tobytes() == want.tobytes()


def test_batched_equals_per_array_loop(ks):
    import torch
    lengths = gen.batched_lengths(256, 100, 200_000, seed=gen.seed_for(3, 5, 0))
    off = gen.offsets_from_lengths(lengths)
    flat = gen.uniform_f32(gen.seed_for(3, 5, 1), int(off[-1]))
    a = _dev(flat)
    b = a.clone()
    ks.sort_batched_(a, _dev(off))
    for r in range(len(lengths)):
        ks.sort_(b[int(off[r]):int(off[r + 1])])
    torch.cuda.synchronize()
    assert ks.ksort_get_device_error() == 0
    assert torch.equal(a, b)


def test_batched_graph_capture_replay(ref, ks):
    import torch
    lengths = np.array([5000, 1, 70_000, 0, 12_345, 2], np.int64)
    off = gen.offsets_from_lengths(lengths)
    flat = gen.uniform_f32(gen.seed_for(3, 6, 0), int(off[-1]))
    want = flat.copy()
    ref.sort_batched(want, off)
    pristine = _dev(flat)
    keys = pristine.clone()
    offs = _dev(off)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ks.ksort_reserve_workspace(ks.F32, int(off[-1]), len(lengths), stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ks.sort_batched_(keys, offs, stream=s)
    for _ in range(3):
        keys.copy_(pristine)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert keys.cpu().numpy().tobytes() == want.tobytes()
    assert ks.ksort_get_device_error(s) == 0


def test_bad_offsets_reported_not_faulted(ks):
    import torch
    flat = _dev(gen.uniform_f32(1, 1000))
    bad = _dev(np.array([0, 600, 400, 1000], np.int64))  # decreasing
    ks.sort_batched_(flat, bad)
    assert ks.ksort_get_device_error() == 6
    out_of_range = _dev(np.array([0, 500, 2000], np.int64))
    ks.sort_batched_(flat, out_of_range)
    assert ks.ksort_get_device_error() == 6
    # the stream's workspace is still usable afterwards
    good = _dev(np.array([0, 500, 1000], np.int64))
    ks.sort_batched_(flat, good)
    assert ks.ksort_get_device_error() == 0
    h = flat.cpu().numpy()
    assert np.all(np.diff(h[:500]) >= 0) and np.all(np.diff(h[500:]) >= 0)
    torch.cuda.synchronize()


def test_bounded_wait_times_out_cleanly(ks):
    """A device wait on a flag that nothing sets gives up after its limit and reports
    KSORT_ERR_TIMEOUT; the context stays usable."""
    import time
    t0 = time.time()
    ks.ksort_selftest_wait_timeout(200)
    assert ks.ksort_get_device_error() == 5
    assert time.time() - t0 < 30
    t = _dev(gen.uniform_f32(2, 10_000))
    ks.sort_(t)
    assert ks.ksort_get_device_error() == 0
    assert np.all(np.diff(t.cpu().numpy()) >= 0)


def test_host_side_argument_errors(ks):
    import torch
    t = _dev(gen.uniform_f32(3, 100))
    with pytest.raises(ks.KSortError) as e:
        ks.ksort_sort(ks.F32, t.data_ptr() + 1, 50)  # misaligned
    assert e.value.status == 1
    host = torch.zeros(100)
    with pytest.raises(ks.KSortError) as e:
        ks.ksort_sort(ks.F32, host.data_ptr(), 100)  # host pointer
    assert e.value.status == 1
    with pytest.raises(ks.KSortError):
        ks.ksort_partition_out(ks.F32, t, t, 100, _dev(np.zeros(1, np.int64)))  # overlap
