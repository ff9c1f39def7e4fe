"""ksort_partition_exact: Steps 1-4 in the paper's own element order (the hole scheme of
Section 1.1), compared byte for byte with the oracle's literal partition: the same key
index and the same array, not only the same sides. Then the recursion of Steps 5-6
replayed call by call on the GPU against the oracle's per-call record, including the
worked example of Section 1.2."""
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
    """uint32 keys travel as int32 bit patterns (torch's uint32 support is partial)."""
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


def _exact(ks, a):
    import torch
    src = _dev(a)
    dst = torch.empty_like(src)
    dst.view(torch.uint8).fill_(0xAB)
    i = ks.partition_exact(src, dst, dtype={np.dtype(np.float32): "f32",
                                            np.dtype(np.float64): "f64",
                                            np.dtype(np.uint32): "u32"}[a.dtype])
    assert ks.ksort_get_device_error() == 0
    return i, dst.cpu().numpy().view(a.dtype)


def _oracle(ref, a):
    b = a.copy()
    i, flag, temp, _ = ref.partition(b)
    return i, b


def test_illustration_first_row(ref, ks):
    # Section 1.2: the first call (key 55) leaves 8 5 50 22 55 66 75 78 60 94
    for dt in (np.uint32, np.float32, np.float64):
        a = np.array(gen.ILLUSTRATION, dt)
        i, got = _exact(ks, a)
        assert i == 4
        assert got.tolist() == [8, 5, 50, 22, 55, 66, 75, 78, 60, 94]
        ri, want = _oracle(ref, a)
        assert (i, got.tobytes()) == (ri, want.tobytes())


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [1, 2, 3, 31, 1024, 1025, 1026, 2049, 4097, 100_003, 1_000_000])
def test_exact_matches_oracle(ref, ks, dtype, n):
    a = gen.make("uniform", dtype, n, gen.seed_for(7, n % 1013, 0))
    i, got = _exact(ks, a)
    if n == 1:
        assert i == 0 and got.tobytes() == a.tobytes()
        return
    ri, want = _oracle(ref, a)
    assert i == ri
    assert got.tobytes() == want.tobytes()


@pytest.mark.parametrize("dtype", ["f32", "u32"])
@pytest.mark.parametrize("pattern", ["sorted", "reverse", "distinct16", "organ_pipe"])
def test_exact_stress(ref, ks, dtype, pattern):
    for n in (20_000, 50_000):
        a = gen.make(pattern, dtype, n, gen.seed_for(7, 50, n))
        i, got = _exact(ks, a)
        ri, want = _oracle(ref, a)
        assert (i, got.tobytes()) == (ri, want.tobytes()), (pattern, n)


def test_small_words_exhaustive(ref, ks):
    # every {0,1,2}-word of length 2..7 (duplicates of the key included)
    import itertools
    for n in range(2, 8):
        for w in itertools.product((0, 1, 2), repeat=n):
            a = np.array(w, np.uint32)
            i, got = _exact(ks, a)
            ri, want = _oracle(ref, a)
            assert (i, got.tobytes()) == (ri, want.tobytes()), w


@pytest.mark.parametrize("n", [10, 3000])
def test_recursion_replayed_call_by_call(ref, ks, n):
    """Steps 5-6 driven by the oracle's call record (depth first, left before right): each
    GPU call on [left, right] must leave the whole array exactly as the oracle's call did.
    n = 10 is the worked example of Section 1.2."""
    import torch
    if n == 10:
        a = np.array(gen.ILLUSTRATION, np.uint32)
    else:
        a = gen.make("uniform", "u32", n, gen.seed_for(7, 99, 0))
    _, rows = ref.sort_traced(a.copy())
    cur = _dev(a)
    tmp = torch.empty_like(cur)
    idx = torch.empty(1, dtype=torch.int64, device="cuda")
    for r in rows:
        lo, hi = r["left"], r["right"] + 1
        seg = cur[lo:hi]
        ks.ksort_partition_exact(ks.U32, seg, tmp[lo:hi], hi - lo, idx)
        cur[lo:hi] = tmp[lo:hi]
        assert int(idx.item()) + lo == r["index"]
        assert cur.cpu().numpy().tobytes() == r["array"].tobytes()  # bytes: u32 as i32
    final = cur.cpu().numpy().view(np.uint32)
    assert (final[1:] >= final[:-1]).all()
    assert ks.ksort_get_device_error() == 0
