"""GPU parity of the one-pass ring partition (part_ring_kernel), the default form of
ksort_partition and ksort_partition_out, in every compiled configuration, against the C
oracle on the same seeded inputs: a first-level partition (Steps 1-4) must give the
oracle's key index and the same two multisets.

Sizes span one tile, several tiles per CTA with ragged tails and the array's last
partial tile; inputs cover the stress patterns (everything left, everything right, few
distinct values), special float values, misaligned starts, two partitions running at
once on two streams (more CTAs than fit the GPU together), CUDA-graph replay, and the
full 5e7-key size that bench.py times."""
import numpy as np
import pytest

import ksort_inputs as gen

pytestmark = pytest.mark.gpu

DTYPES = {"f32": 0, "f64": 1, "u32": 2}
FORMS = [1, 2, 3, 4, 5, 6]


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
        ks.ksort_set_tuning(c, partition_form=t["partition_form"], tile_shape=t["tile_shape"],
                            spin_limit_ms=t["spin_limit_ms"])


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def bits(v):
    """Multiset of bit patterns, sorted, as bytes (+0 and -0, NaN payloads kept apart)."""
    return np.sort(v.view(np.uint64 if v.dtype.itemsize == 8 else np.uint32)).tobytes()


def check_sides(got, i, want, ri, a0):
    assert i == ri
    assert got[i:i + 1].tobytes() == np.asarray([a0], dtype=got.dtype).tobytes()
    assert bits(got[:i]) == bits(want[:ri])
    assert bits(got[i + 1:]) == bits(want[ri + 1:])


def check_partition(ref, ks, a):
    """Out of place (input untouched) and in place, both against the oracle."""
    import torch
    want = a.copy()
    ri = ref.partition(want)[0] if len(a) > 1 else 0  # one key: index 0 (no step runs)
    src = to_dev(a)
    dst = torch.empty_like(src)
    i = int(ks.partition_out(src, dst).item())
    assert ks.ksort_get_device_error() == 0
    assert src.cpu().numpy().tobytes() == a.tobytes()
    check_sides(dst.cpu().numpy(), i, want, ri, a[0])
    t = to_dev(a)
    i2 = ks.partition_(t)
    assert ks.ksort_get_device_error() == 0
    check_sides(t.cpu().numpy(), i2, want, ri, a[0])


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("dtype", list(DTYPES))
def test_ring_sizes(ref, ks, restore, dtype, form):
    code = DTYPES[dtype]
    ks.ksort_set_tuning(code, partition_form=form)
    assert ks.ksort_get_tuning(code)["partition_form"] == form
    nt, tile, occ = ks.ksort_partition_shape(code, form)
    assert nt % 32 == 0 and tile % 512 == 0 and occ >= 1
    for n in (1, 2, 3, 33, tile - 1, tile, tile + 1, tile + 2, 5 * tile + 3, 1_000_003,
              3_000_017):
        a = gen.make("uniform", dtype, n, gen.seed_for(7, form, n % 1013))
        check_partition(ref, ks, a)


@pytest.mark.parametrize("dtype", ["f32", "u32"])
@pytest.mark.parametrize("pattern", ["sorted", "reverse", "distinct16", "organ_pipe"])
def test_ring_stress_patterns(ref, ks, restore, dtype, pattern):
    """Sorted input sends every key right of the first, reverse input every key left;
    16 distinct values put long runs equal to the key on the right side (Step 3)."""
    for form in (1, 4, 5):
        ks.ksort_set_tuning(DTYPES[dtype], partition_form=form)
        for n in (50_000, 2_000_003):
            a = gen.make(pattern, dtype, n, gen.seed_for(7, 20, n % 997))
            check_partition(ref, ks, a)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_ring_special_values(ref, ks, restore, dtype):
    """NaN elements go left (the compare key <= NaN is false), a NaN key sends every
    element left, +0 and -0 compare equal, infinities and subnormals compare as IEEE
    orders them."""
    dt = np.float32 if dtype == "f32" else np.float64
    rng = np.random.default_rng(1107)
    specials = np.array([np.nan, -np.nan, 0.0, -0.0, np.inf, -np.inf,
                         np.finfo(dt).tiny / 4, -np.finfo(dt).tiny / 4, 1.0, 0.5], dt)
    for form in FORMS:
        ks.ksort_set_tuning(DTYPES[dtype], partition_form=form)
        for key in (np.nan, 0.0, -0.0, 0.5, np.inf, -np.inf):
            a = rng.choice(specials, size=300_001).astype(dt)
            a[0] = key
            check_partition(ref, ks, a)


@pytest.mark.parametrize("dtype", list(DTYPES))
def test_ring_misaligned_starts(ref, ks, restore, dtype):
    """Views that start 1..3 keys past a 16-byte boundary: tiles are anchored at the
    boundary below the first classified key, and the keys before the view stay put."""
    import torch
    base = gen.make("uniform", dtype, 700_003, gen.seed_for(7, 30, 1))
    for form in FORMS:
        ks.ksort_set_tuning(DTYPES[dtype], partition_form=form)
        for off in (1, 2, 3):
            a = base[off:]
            want = a.copy()
            ri, *_ = ref.partition(want)
            big = to_dev(base)
            out = torch.zeros_like(big)
            view = big[off:]
            i = int(ks.partition_out(view, out[off:]).item())
            assert ks.ksort_get_device_error() == 0
            got = out.cpu().numpy()
            assert not got[:off].any()
            check_sides(got[off:], i, want, ri, a[0])
            i2 = ks.partition_(view)
            check_sides(big.cpu().numpy()[off:], i2, want, ri, a[0])
            assert big.cpu().numpy()[:off].tobytes() == base[:off].tobytes()


def test_ring_two_streams_at_once(ref, ks, restore):
    """Two partitions on two streams overlap on the GPU, each with a grid that fills
    it alone. A CTA waits only for tiles that running CTAs have claimed, so both finish,
    and both results match the oracle."""
    import torch
    for form in FORMS:
        # every wait here lasts microseconds; a short limit turns a stall into an error
        ks.ksort_set_tuning(0, partition_form=form, spin_limit_ms=200)
        arrays = [gen.make("uniform", "f32", 4_000_037, gen.seed_for(7, 40 + form, r))
                  for r in range(2)]
        streams = [torch.cuda.Stream() for _ in arrays]
        srcs = [to_dev(a) for a in arrays]
        dsts = [torch.empty_like(s) for s in srcs]
        idx = [torch.empty(1, dtype=torch.int64, device="cuda") for _ in arrays]
        torch.cuda.synchronize()
        for rep in range(4):
            for s, src, dst, ix in zip(streams, srcs, dsts, idx):
                ks.ksort_partition_out(0, src, dst, src.numel(), ix, stream=s)
        torch.cuda.synchronize()
        for s in streams:
            assert ks.ksort_get_device_error(s) == 0
        for a, dst, ix in zip(arrays, dsts, idx):
            want = a.copy()
            ri, *_ = ref.partition(want)
            check_sides(dst.cpu().numpy(), int(ix.item()), want, ri, a[0])


def test_ring_graph_replay(ref, ks, restore):
    """Captured once in a CUDA graph (workspace reserved first) and replayed: every
    replay partitions the current input afresh."""
    import torch
    ks.ksort_set_tuning(0, partition_form=5)
    n = 2_500_001
    s = torch.cuda.Stream()
    src = torch.empty(n, dtype=torch.float32, device="cuda")
    dst = torch.empty_like(src)
    ix = torch.empty(1, dtype=torch.int64, device="cuda")
    with torch.cuda.stream(s):
        ks.ksort_reserve_workspace(0, n, 1, stream=s)
        ks.ksort_partition_out(0, src, dst, n, ix, stream=s)  # set-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ks.ksort_partition_out(0, src, dst, n, ix, stream=s)
    for rep in range(3):
        a = gen.make("uniform", "f32", n, gen.seed_for(7, 50, rep))
        src.copy_(torch.from_numpy(a))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert ks.ksort_get_device_error(s) == 0
        want = a.copy()
        ri, *_ = ref.partition(want)
        check_sides(dst.cpu().numpy(), int(ix.item()), want, ri, a[0])


def test_ring_full_size(ref, ks, restore):
    """The 5e7-key float32 partition that bench.py times, in the configuration the
    library defaults to (5) and in configuration 1, against the oracle's own partition
    of the same array."""
    import torch
    n = 50_000_000
    a = gen.uniform_f32(gen.seed_for(1, 6, 500), n)
    want = a.copy()
    ri, *_ = ref.partition(want)
    src = to_dev(a)
    for form in (5, 1):
        ks.ksort_set_tuning(0, partition_form=form)
        dst = torch.empty_like(src)
        i = int(ks.partition_out(src, dst).item())
        assert ks.ksort_get_device_error() == 0
        check_sides(dst.cpu().numpy(), i, want, ri, a[0])
        del dst


def test_legacy_forms_still_selectable(ref, ks, restore):
    """partition_form -1 hands single partitions back to the form of the tile shape
    (part_kernel, or the split partition of the wave form)."""
    ks.ksort_set_tuning(0, partition_form=-1)
    assert ks.ksort_get_tuning(0)["partition_form"] == -1
    for shape in (1, 10):
        ks.ksort_set_tuning(0, tile_shape=shape)
        a = gen.make("uniform", "f32", 1_000_003, gen.seed_for(7, 60, shape))
        check_partition(ref, ks, a)
