"""The C ABI library loads and exports what include/*.h declares (no GPU needed).
Also the host-side argument checks that return before any CUDA call."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"KSORT_API\s+[\w\s\*]*?\b(ksort_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    import paper_1107_3622_gb300 as ks
    return ks.load()


def test_header_declares_entry_points():
    names = _declared()
    for must in ("ksort_partition", "ksort_partition_out", "ksort_sort", "ksort_sort_batched",
                 "ksort_get_device_error", "ksort_reserve_workspace", "ksort_status_string"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_library_is_in_tree(lib):
    import paper_1107_3622_gb300 as ks
    assert os.path.commonpath([ks.library_path(), ROOT]) == ROOT


def test_status_strings(lib):
    import paper_1107_3622_gb300 as ks
    for code in range(10):
        assert ks.ksort_status_string(code) and "unknown" not in ks.ksort_status_string(code)
    assert "unknown" in ks.ksort_status_string(99)


def test_host_side_rejections_need_no_gpu(lib):
    # These return before any CUDA runtime call.
    assert lib.ksort_sort(0, None, -1, None) == 1          # negative n
    assert lib.ksort_sort(7, None, 10, None) == 2          # unknown dtype
    assert lib.ksort_sort(0, None, 1, None) == 0           # n <= 1 is a no-op
    assert lib.ksort_sort_batched(0, None, None, 3, 10, None) == 1  # offsets missing
    assert lib.ksort_partition(0, None, 0, None, None) == 1         # n == 0
    assert lib.ksort_partition(5, None, 4, None, None) == 2
    assert lib.ksort_selftest_wait_timeout(0, None) == 1
    assert lib.ksort_partition_out_noalloc(0, None, None, (1 << 24) + 1, None, None) == 9
    assert lib.ksort_partition_out_noalloc(0, None, None, 0, None, None) == 1
    assert lib.ksort_get_phase_times(None, 1, None, None) == 1  # no output buffers
    assert lib.ksort_get_phase_times(None, -1, None, None) == 1
    assert lib.ksort_set_phase_timing(0) == 0


def test_tuning_validation(lib):
    import paper_1107_3622_gb300 as ks
    for code in (ks.F32, ks.F64, ks.U32):
        assert ks.ksort_max_cutoff(code) >= 1024
        assert ks.ksort_tile_keys(code) >= 1024
        before = ks.ksort_get_tuning(code)
        with pytest.raises(ks.KSortError):
            ks.ksort_set_tuning(code, cutoff=ks.ksort_max_cutoff(code) + 1)
        with pytest.raises(ks.KSortError):
            ks.ksort_set_tuning(code, cutoff=1)
        assert ks.ksort_get_tuning(code) == before


def test_oracle_and_library_share_no_code():
    """The oracle and the CUDA path are independent: neither includes nor imports the
    other, and the package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_1107_3622_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if os.path.isfile(path) and path.endswith((".py", ".cu", ".cuh", ".h")):
            text = open(path).read()
            assert "oracle" not in re.findall(r"^\s*(?:import|from)\s+(\w+)", text, re.M), path
            assert "ksort_ref" not in text, path
    for path in glob.glob(os.path.join(ROOT, "oracle", "*")):
        if os.path.isfile(path) and path.endswith((".py", ".c", ".h")):
            text = open(path).read()
            assert "paper_1107_3622_gb300" not in text and "ksort.h" not in text, path


def test_tile_shapes_and_tuning_fields(lib):
    import paper_1107_3622_gb300 as ks
    for code in (ks.F32, ks.F64, ks.U32):
        shapes = [ks.ksort_tile_shape(code, s) for s in range(1, 13)]
        vec = 2 if code == ks.F64 else 4
        for nt, ipt, _ in shapes:
            assert nt % 32 == 0 and ipt % vec == 0 and ipt <= 32
        assert len(set(shapes)) == 12
        assert [fm for _, _, fm in shapes] == [0] * 3 + [1] * 3 + [2] * 3 + [3] * 3
        # forms 0, 2 and 3 share their CTA shapes; form 1 (the ring) has its own: a
        # producer warp, a reservation warp and data warps
        assert [s[:2] for s in shapes[:3]] == [s[:2] for s in shapes[6:9]] == \
            [s[:2] for s in shapes[9:]]
        for nt, ipt, _ in shapes[3:6]:
            assert (nt - 64) % 256 == 0
        with pytest.raises(ks.KSortError):
            ks.ksort_tile_shape(code, 0)
        with pytest.raises(ks.KSortError):
            ks.ksort_tile_shape(code, 13)
        before = ks.ksort_get_tuning(code)
        assert before["tile_shape"] in range(1, 13)
        assert before["wave_levels"] == -1 or before["wave_levels"] in range(1, 65)
        with pytest.raises(ks.KSortError):
            ks.ksort_set_tuning(code, tile_shape=13)
        with pytest.raises(ks.KSortError):
            ks.ksort_set_tuning(code, ctas_per_sm=-2)
        for bad in (-2, 65):
            with pytest.raises(ks.KSortError):
                ks.ksort_set_tuning(code, wave_levels=bad)
        assert before["medium_tiles"] == -1 or before["medium_tiles"] in range(1, 17)
        for bad in (-2, 17):
            with pytest.raises(ks.KSortError):
                ks.ksort_set_tuning(code, medium_tiles=bad)
        ks.ksort_set_tuning(code, medium_tiles=5)
        assert ks.ksort_get_tuning(code)["medium_tiles"] == 5
        ks.ksort_set_tuning(code, medium_tiles=before["medium_tiles"])
        ks.ksort_set_tuning(code, tile_shape=2)
        nt, ipt, _ = shapes[1]
        assert ks.ksort_tile_keys(code) == nt * ipt
        ks.ksort_set_tuning(code, tile_shape=11, wave_levels=7)
        assert ks.ksort_tile_keys(code) == nt * ipt  # the wave form keeps the CTA shape's tile
        assert ks.ksort_get_tuning(code)["wave_levels"] == 7
        ks.ksort_set_tuning(code, tile_shape=before["tile_shape"], wave_levels=-1)
        assert ks.ksort_get_tuning(code) == before
    for code in (ks.F32, ks.F64, ks.U32):
        before = ks.ksort_get_tuning(code)
        assert before["partition_form"] in (-1, 1, 2, 3, 4, 5, 6)
        for bad in (-2, 7):
            with pytest.raises(ks.KSortError):
                ks.ksort_set_tuning(code, partition_form=bad)
        ks.ksort_set_tuning(code, partition_form=-1)
        assert ks.ksort_get_tuning(code)["partition_form"] == -1
        ks.ksort_set_tuning(code, partition_form=3)
        assert ks.ksort_get_tuning(code)["partition_form"] == 3
        ks.ksort_set_tuning(code, partition_form=before["partition_form"])
        assert ks.ksort_get_tuning(code) == before
        assert before["sort_reserve"] in (-1, 1)
        for bad in (-2, 2):
            with pytest.raises(ks.KSortError):
                ks.ksort_set_tuning(code, sort_reserve=bad)
        ks.ksort_set_tuning(code, sort_reserve=-1)
        assert ks.ksort_get_tuning(code)["sort_reserve"] == -1
        ks.ksort_set_tuning(code, sort_reserve=before["sort_reserve"])
        assert ks.ksort_get_tuning(code) == before
        assert before["finish_in_tiles"] == -1 or 1 <= before["finish_in_tiles"] <= 4096
        for bad in (-2, 4097):
            with pytest.raises(ks.KSortError):
                ks.ksort_set_tuning(code, finish_in_tiles=bad)
        ks.ksort_set_tuning(code, finish_in_tiles=32)
        assert ks.ksort_get_tuning(code)["finish_in_tiles"] == 32
        ks.ksort_set_tuning(code, finish_in_tiles=-1)
        assert ks.ksort_get_tuning(code)["finish_in_tiles"] == -1
        ks.ksort_set_tuning(code, finish_in_tiles=before["finish_in_tiles"])
        assert ks.ksort_get_tuning(code) == before
        assert before["finisher_threads"] in (256, 512, 1024)
        for bad in (-1, 128, 300, 2048):
            with pytest.raises(ks.KSortError):
                ks.ksort_set_tuning(code, finisher_threads=bad)
        for nt in (512, 1024, 256):
            ks.ksort_set_tuning(code, finisher_threads=nt)
            assert ks.ksort_get_tuning(code)["finisher_threads"] == nt
        ks.ksort_set_tuning(code, finisher_threads=before["finisher_threads"])
        assert ks.ksort_get_tuning(code) == before
        assert before["cluster_sort"] in (-1, 1)
        for bad in (-2, 2):
            with pytest.raises(ks.KSortError):
                ks.ksort_set_tuning(code, cluster_sort=bad)
        for v in (1, -1):
            ks.ksort_set_tuning(code, cluster_sort=v)
            assert ks.ksort_get_tuning(code)["cluster_sort"] == v
        ks.ksort_set_tuning(code, cluster_sort=before["cluster_sort"])
        assert ks.ksort_get_tuning(code) == before
        # every ring configuration stages the same bytes per tile for 4- and 8-byte keys
        keyb = 8 if code == ks.F64 else 4
        for form in (1, 2, 3, 4, 5, 6):
            nt, tile, occ = ks.ksort_partition_shape(code, form)
            assert nt % 32 == 0 and nt >= 96 and occ >= 1
            assert tile * keyb == ks.ksort_partition_shape(ks.F32, form)[1] * 4
        for bad in (0, 7):
            with pytest.raises(ks.KSortError):
                ks.ksort_partition_shape(code, bad)
    # shared-memory staging of two cutoff-sized buffers must fit a CTA (227 KB)
    assert 2 * 8 * ks.ksort_max_cutoff(ks.F64) <= 227 * 1024
    assert 2 * 4 * ks.ksort_max_cutoff(ks.F32) <= 227 * 1024


def test_autotune_workload_keys():
    import numpy as np
    from paper_1107_3622_gb300 import autotune
    assert autotune.workload_key("sort", 0, n=7_000_000) == "sort:f32:2^23"
    assert autotune.workload_key("sort", 1, n=1_000_000) == "sort:f64:2^20"
    k = autotune.workload_key("batched", 2, lengths=np.array([100, 1000, 500_000]))
    assert k == "batched:u32:3x[100,500000]:2^19"
    assert len(autotune.library_hash()) == 16
    # a search limited to some tile shapes is cached under its own key; unknown shapes
    # are refused before any device work
    assert autotune.shapes_suffix(None) == ""
    assert autotune.shapes_suffix((1, 2, 3)) == "|shapes=1,2,3"
    import pytest
    with pytest.raises(ValueError):
        autotune.autotune("batched", 2, lengths=np.array([100, 1000]), shapes=(0, 13))


def _header_structs():
    """{typedef name: [(field, C type), ...]} of every plain struct in include/*.h."""
    out = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for body, name in re.findall(r"typedef\s+struct\s*\{(.*?)\}\s*(\w+)\s*;", text, flags=re.S):
            out[name] = re.findall(r"(\w+)\s+(\w+)\s*;", body)
    return out


def test_binding_structs_match_the_header():
    """The ctypes mirrors of the header's structs have the same fields, in the same order
    and of the same C types, so every call that passes one reads what the library wrote."""
    import paper_1107_3622_gb300 as ks
    ctype = {"int32_t": ctypes.c_int32, "uint64_t": ctypes.c_uint64, "int64_t": ctypes.c_int64}
    structs = _header_structs()
    for name, mirror in (("ksort_tuning_t", ks.Tuning), ("ksort_stats_t", ks.Stats)):
        fields = structs[name]
        assert [f for _, f in fields] == [n for n, _ in mirror._fields_], name
        assert [ctype[t] for t, _ in fields] == [c for _, c in mirror._fields_], name
        assert ctypes.sizeof(mirror) == sum(ctypes.sizeof(ctype[t]) for t, _ in fields)

