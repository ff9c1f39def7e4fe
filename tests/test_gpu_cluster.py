"""The cluster form of ksort_sort (tuning cluster_sort): one thread-block cluster holds
the whole array in shared memory and runs every level above the cutoff, all sub-arrays
of a level at once, then the finisher takes the small sides. Every sort must stay
bit-identical to the oracle for each key type, size (one level to the cluster's
capacity), cutoff and input class; NaN inputs must give a permutation with the other
keys in order; arrays beyond the cluster's reach must take the work queue; graph replay
and two clusters at once on two streams must work."""
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
def cluster(ks):
    """cluster_sort on for every dtype (tile shape 3); restored afterwards."""
    saved = {c: ks.ksort_get_tuning(c) for c in DTYPES.values()}
    for c in DTYPES.values():
        ks.ksort_set_tuning(c, cluster_sort=1)
    yield
    for c, t in saved.items():
        ks.ksort_set_tuning(c, cutoff=t["cutoff"], cluster_sort=t["cluster_sort"],
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


def test_shape(ks):
    for code in DTYPES.values():
        c, m = ks.ksort_cluster_shape(code)
        assert c in (8, 16)
        per = m // c
        assert m % c == 0 and per % 4 == 0 and per <= 32 * 1024
        assert m >= (100_000 if code != ks.F64 else 50_000)


@pytest.mark.parametrize("dtype", list(DTYPES))
def test_cluster_sizes(ref, ks, cluster, dtype):
    """From one level (cutoff + 1) up to the cluster's capacity, then just beyond it
    (the work queue), with ragged slices."""
    code = DTYPES[dtype]
    cut = ks.ksort_get_tuning(code)["cutoff"]
    _, cap = ks.ksort_cluster_shape(code)
    for n in (cut + 1, cut + 2, 5_001, 33_333, 100_003, cap - 3, cap, cap + 1):
        a = gen.make("uniform", dtype, n, gen.seed_for(14, 1, n % 1009))
        ks.ksort_sort(code, _dev(a[:2]), 2)  # the stats below belong to the next call
        assert _sort(ks, code, a).tobytes() == _oracle(ref, a).tobytes(), n
        st = ks.ksort_get_stats()
        assert st["launches"] == (2 if n <= cap else 3), n
        assert st["small_keys"] <= n and st["large_items"] >= 1


@pytest.mark.parametrize("cutoff", [64, 1024, 16384])
def test_cluster_cutoffs(ref, ks, cluster, cutoff):
    """Small cutoffs make many active sub-arrays per level (below 512 * (cutoff + 1)
    keys), large ones few; above that bound the work queue takes the array."""
    for dtype, code in DTYPES.items():
        c = min(cutoff, ks.ksort_max_cutoff(code))
        ks.ksort_set_tuning(code, cutoff=c)
        for n in (20_011, 150_001):
            a = gen.make("uniform", dtype, n, gen.seed_for(14, 2, c))
            assert _sort(ks, code, a).tobytes() == _oracle(ref, a).tobytes(), (dtype, c, n)


@pytest.mark.parametrize("pattern", ["sorted", "reverse", "distinct16", "organ_pipe",
                                     "quantized15"])
def test_cluster_stress(ref, ks, cluster, pattern):
    """Orders that make one-sided partitions (one level per key near the top) and runs of
    equal keys (which go right, Step 3)."""
    for dtype, code in DTYPES.items():
        n = 30_000 if pattern in ("sorted", "reverse", "organ_pipe", "distinct16") else 150_000
        a = gen.make(pattern, dtype, n, gen.seed_for(14, 3, n))
        assert _sort(ks, code, a).tobytes() == _oracle(ref, a).tobytes(), (dtype, pattern)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_cluster_specials(ref, ks, cluster, dtype):
    """Infinities, subnormals and both zeros: a permutation in ascending order; without
    NaN and -0 (every equal pair then has equal bits) it is the oracle's array."""
    dt = np.float32 if dtype == "f32" else np.float64
    code = DTYPES[dtype]
    rng = np.random.default_rng(3622)
    pool = np.array([np.inf, -np.inf, np.finfo(dt).tiny / 4, 1.0, -1.0, 0.0], dt)
    a = rng.standard_normal(120_001).astype(dt)
    pick = rng.random(a.size) < 0.2
    a[pick] = rng.choice(pool, int(pick.sum()))
    assert _sort(ks, code, a).tobytes() == _oracle(ref, a).tobytes()
    a[rng.random(a.size) < 0.05] = -0.0
    a[rng.random(a.size) < 0.01] = np.nan
    got = _sort(ks, code, a)
    bits = np.uint64 if dt == np.float64 else np.uint32
    assert np.sort(got.view(bits)).tobytes() == np.sort(a.view(bits)).tobytes()
    v = got[~np.isnan(got)]
    assert np.all(v[1:] >= v[:-1])


def test_cluster_graph_replay(ref, ks, cluster):
    import torch
    n = 200_003
    s = torch.cuda.Stream()
    keys = torch.empty(n, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(s):
        ks.ksort_reserve_workspace(ks.F32, n, 1, stream=s)
        keys.copy_(torch.from_numpy(gen.uniform_f32(2, n)))
        ks.ksort_sort(ks.F32, keys, n, stream=s)  # set-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ks.ksort_sort(ks.F32, keys, n, stream=s)
    for rep in range(3):
        a = gen.uniform_f32(gen.seed_for(14, 4, rep), n)
        keys.copy_(torch.from_numpy(a))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert ks.ksort_get_device_error(s) == 0
        assert keys.cpu().numpy().tobytes() == _oracle(ref, a).tobytes()


def test_cluster_two_streams_and_repeats(ref, ks, cluster):
    """Two clusters at once on two streams, four sorts each back to back."""
    import torch
    arrays = [gen.uniform_f32(gen.seed_for(14, 5, r), 180_001 + r) for r in range(2)]
    streams = [torch.cuda.Stream() for _ in arrays]
    bufs = [[_dev(a) for _ in range(4)] for a in arrays]
    for s, b in zip(streams, bufs):
        ks.ksort_reserve_workspace(ks.F32, b[0].numel(), 1, stream=s)
    torch.cuda.synchronize()
    for k in range(4):
        for s, b in zip(streams, bufs):
            ks.ksort_sort(ks.F32, b[k], b[k].numel(), stream=s)
    torch.cuda.synchronize()
    for s, b, a in zip(streams, bufs, arrays):
        assert ks.ksort_get_device_error(s) == 0
        want = _oracle(ref, a).tobytes()
        for t in b:
            assert t.cpu().numpy().tobytes() == want
