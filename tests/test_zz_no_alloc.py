"""ksort_partition_out_noalloc: the partition of Steps 1-4 (Section 1.1) with the kernels'
scratch in one fixed device array, so that a call allocates nothing. It runs the sort's
seed kernel and tile_kernel (tile shape 1, whatever the tuning) and a status kernel:
three launches. Its results are checked against ksort_partition_out on two calls in a row
that share the array: the oracle's key index and the same two sides (as multisets, the
partition's contract) against the default form, and byte for byte against the form that
follows tile shape 1 (part_kernel), which lays tiles out the way tile_kernel does.

This file is collected last on purpose. It must pass in a fresh process, where its first
call does the per-device set-up, and after every other test has used the library."""
import numpy as np
import pytest

import ksort_inputs as gen

pytestmark = pytest.mark.gpu

DTYPES = ["f32", "f64", "u32"]


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


def _poisoned(like):
    import torch
    t = torch.empty_like(like)
    t.view(torch.uint8).fill_(0xAB)
    return t


def _host(t):
    return t.cpu().numpy()


def _oracle_index(ref, a):
    b = a.copy()
    i, *_ = ref.partition(b)
    return i


def _same_sides(got, want, i):
    """Same key at i and the same multisets on both sides of it."""
    return got[i:i + 1].tobytes() == want[i:i + 1].tobytes() and \
        np.sort(got[:i]).tobytes() == np.sort(want[:i]).tobytes() and \
        np.sort(got[i + 1:]).tobytes() == np.sort(want[i + 1:]).tobytes()


@pytest.fixture
def tile_layout_form(ks):
    """ksort_partition_out under partition_form -1 and tile shape 1 runs part_kernel,
    whose tiles have tile_kernel's layout; the tuning is restored afterwards."""
    saved = {c: ks.ksort_get_tuning(c) for c in (ks.F32, ks.F64, ks.U32)}
    yield lambda code: ks.ksort_set_tuning(code, partition_form=-1, tile_shape=1)
    for c, t in saved.items():
        ks.ksort_set_tuning(c, partition_form=t["partition_form"], tile_shape=t["tile_shape"])


@pytest.mark.parametrize("dtype", DTYPES)
def test_two_calls_in_a_row_match_partition_out(ref, ks, tile_layout_form, dtype):
    """Two back-to-back calls on one stream (the second smaller than the first, with a
    misaligned start), then the same two inputs through ksort_partition_out: the default
    form (same index and sides) and the tile-layout form (same bytes)."""
    import torch
    code = {"f32": ks.F32, "f64": ks.F64, "u32": ks.U32}[dtype]
    a1 = gen.make("uniform", dtype, 1_000_003, gen.seed_for(5, 1, 0))
    big = gen.make("uniform", dtype, 70_002, gen.seed_for(5, 2, 0))
    a2 = big[1:]
    s1 = _dev(a1)
    s2 = _dev(big)[1:]
    g1, g2 = _poisoned(s1), _poisoned(s2)
    w1, w2 = _poisoned(s1), _poisoned(s2)
    b1, b2 = _poisoned(s1), _poisoned(s2)
    idx = torch.full((6,), -99, dtype=torch.int64, device="cuda")
    ks.ksort_partition_out_noalloc(code, s1, g1, a1.size, idx[0:1])
    ks.ksort_partition_out_noalloc(code, s2, g2, a2.size, idx[1:2])
    ks.ksort_partition_out(code, s1, w1, a1.size, idx[2:3])
    ks.ksort_partition_out(code, s2, w2, a2.size, idx[3:4])
    tile_layout_form(code)
    ks.ksort_partition_out(code, s1, b1, a1.size, idx[4:5])
    ks.ksort_partition_out(code, s2, b2, a2.size, idx[5:6])
    torch.cuda.synchronize()
    assert ks.ksort_get_device_error() == 0
    i1, i2, j1, j2, k1, k2 = idx.tolist()
    assert (i1, i2) == (j1, j2) == (k1, k2)
    assert i1 == _oracle_index(ref, a1) and i2 == _oracle_index(ref, a2)
    assert _same_sides(_host(g1), _host(w1), i1)
    assert _same_sides(_host(g2), _host(w2), i2)
    assert _host(g1).tobytes() == _host(b1).tobytes()
    assert _host(g2).tobytes() == _host(b2).tobytes()
    assert _host(s1).tobytes() == a1.tobytes()  # inputs untouched
    assert _host(s2).tobytes() == a2.tobytes()


def test_largest_size_and_one_key(ref, ks, tile_layout_form):
    """n = KSORT_NOALLOC_MAX_KEYS float64 keys from a start that is not tile-aligned
    (the most tile tickets the fixed array must hold), then n = 1."""
    import torch
    n = ks.KSORT_NOALLOC_MAX_KEYS
    big = gen.make("uniform", "f64", n + 1, gen.seed_for(5, 3, 0))
    src = _dev(big)[1:]
    got, want, same = _poisoned(src), _poisoned(src), _poisoned(src)
    idx = torch.full((3,), -99, dtype=torch.int64, device="cuda")
    ks.ksort_partition_out_noalloc(ks.F64, src, got, n, idx[0:1])
    ks.ksort_partition_out(ks.F64, src, want, n, idx[1:2])
    tile_layout_form(ks.F64)
    ks.ksort_partition_out(ks.F64, src, same, n, idx[2:3])
    torch.cuda.synchronize()
    i, j, k = idx.tolist()
    assert i == j == k == _oracle_index(ref, big[1:])
    assert _same_sides(_host(got), _host(want), i)
    assert torch.equal(got.view(torch.int64), same.view(torch.int64))
    one_in = _dev(np.array([0.25], np.float64))
    one_out = _poisoned(one_in)
    ks.ksort_partition_out_noalloc(ks.F64, one_in, one_out, 1, idx[0:1])
    torch.cuda.synchronize()
    assert int(idx[0].item()) == 0 and float(one_out.item()) == 0.25


def test_rejects_beyond_the_maximum_and_enqueues_nothing(ks):
    import torch
    n = ks.KSORT_NOALLOC_MAX_KEYS + 1
    src = torch.zeros(n, dtype=torch.float32, device="cuda")
    dst = _poisoned(src)
    idx = torch.full((1,), -99, dtype=torch.int64, device="cuda")
    with pytest.raises(ks.KSortError) as e:
        ks.ksort_partition_out_noalloc(ks.F32, src, dst, n, idx)
    assert e.value.status == ks.KSORT_ERR_TOO_LARGE
    assert "KSORT_NOALLOC_MAX_KEYS" in str(e.value)
    torch.cuda.synchronize()
    assert int(idx.item()) == -99
    assert bool((dst.view(torch.uint8) == 0xAB).all())


def test_calls_leave_free_device_memory_unchanged(ks):
    """After the set-up call, further calls take no device memory."""
    import torch
    a = gen.make("uniform", "f32", 300_000, gen.seed_for(5, 4, 0))
    src = _dev(a)
    dst = torch.empty_like(src)
    idx = torch.zeros(1, dtype=torch.int64, device="cuda")
    ks.ksort_partition_out_noalloc(ks.F32, src, dst, a.size, idx)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        ks.ksort_partition_out_noalloc(ks.F32, src, dst, a.size, idx)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert int(idx.item()) == int((torch.from_numpy(a[1:]) < float(a[0])).sum())


def test_device_error_reaches_key_index_and_next_call_is_clean(ref, ks):
    """A device wait of the call's kind that runs past its limit on the fixed array
    (a look-back descriptor that nothing publishes) leaves -KSORT_ERR_TIMEOUT in the key
    index, reports nothing through ksort_get_device_error, and the next call on the same
    stream starts clean and is right."""
    import time
    import torch
    idx = torch.full((1,), -99, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.time()
    ks.ksort_selftest_noalloc_timeout(100, idx)
    torch.cuda.synchronize()
    assert time.time() - t0 < 30
    assert int(idx.item()) == -ks.KSORT_ERR_TIMEOUT
    assert ks.ksort_get_device_error() == 0
    a = gen.make("uniform", "f32", 500_003, gen.seed_for(5, 5, 0))
    src = _dev(a)
    got = _poisoned(src)
    ks.ksort_partition_out_noalloc(ks.F32, src, got, a.size, idx)
    torch.cuda.synchronize()
    i = int(idx.item())
    assert i == _oracle_index(ref, a)
    want = a.copy()
    ref.partition(want)
    assert _same_sides(_host(got), want, i)


def test_captured_in_a_graph_and_replayed(ref, ks):
    """Calls captured in a CUDA graph (after a first call has done the set-up) replay
    with no allocation; each replay partitions the inputs' current contents."""
    import torch
    n1, n2 = 800_001, 65_537
    s = torch.cuda.Stream()
    src1 = torch.empty(n1, dtype=torch.float32, device="cuda")
    src2 = torch.empty(n2, dtype=torch.float64, device="cuda")
    dst1, dst2 = torch.empty_like(src1), torch.empty_like(src2)
    idx = torch.full((2,), -99, dtype=torch.int64, device="cuda")
    with torch.cuda.stream(s):
        ks.ksort_partition_out_noalloc(ks.F32, src1, dst1, n1, idx[0:1], stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ks.ksort_partition_out_noalloc(ks.F32, src1, dst1, n1, idx[0:1], stream=s)
        ks.ksort_partition_out_noalloc(ks.F64, src2, dst2, n2, idx[1:2], stream=s)
    free0, _ = torch.cuda.mem_get_info()
    for rep in range(3):
        a1 = gen.make("uniform", "f32", n1, gen.seed_for(5, 6, rep))
        a2 = gen.make("uniform", "f64", n2, gen.seed_for(5, 7, rep))
        src1.copy_(torch.from_numpy(a1))
        src2.copy_(torch.from_numpy(a2))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        i1, i2 = idx.tolist()
        for a, i, dst in ((a1, i1, dst1), (a2, i2, dst2)):
            want = a.copy()
            assert i == ref.partition(want)[0]
            assert _same_sides(_host(dst), want, i)
    assert torch.cuda.mem_get_info()[0] == free0
    assert ks.ksort_get_device_error(s) == 0
