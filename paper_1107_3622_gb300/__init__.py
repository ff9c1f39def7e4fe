"""K-sort on GB300: Python binding of libksort (include/ksort.h).

K-sort (arxiv 1107.3622, Section 1.1) partitions a sub-array around its first element
(Steps 1-4: x goes right of the key when key <= x) and recurses on both sides
(Steps 5-6). Every step runs in the CUDA kernels of libksort.so; this module only
marshals arguments (torch tensors -> device pointers, the current torch stream) and
turns status codes into exceptions. PyTorch supplies device memory and streams.

The functions named ``ksort_*`` mirror the C entry points one to one. The short
helpers (``partition_``, ``sort_``, ``sort_batched_``) wrap them for tensors.
There is no CPU fallback: without the compiled library every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

__all__ = [
    "KSortError", "F32", "F64", "U32", "load", "library_path",
    "ksort_partition", "ksort_partition_out", "ksort_partition_out_noalloc",
    "ksort_partition_exact", "partition_exact", "ksort_sort", "ksort_sort_batched",
    "ksort_reserve_workspace", "ksort_release_workspace", "ksort_get_device_error",
    "ksort_get_stats", "ksort_set_phase_timing", "ksort_get_phase_times",
    "ksort_get_phase_history",
    "ksort_set_tuning", "ksort_get_tuning", "ksort_max_cutoff",
    "ksort_tile_keys", "ksort_tile_shape", "ksort_partition_shape", "ksort_cluster_shape",
    "ksort_status_string", "ksort_last_cuda_error",
    "ksort_selftest_wait_timeout", "ksort_selftest_noalloc_timeout", "ksort_debug_trace",
    "partition_", "partition_out", "sort_", "sort_batched_", "dtype_code",
]

F32, F64, U32 = 0, 1, 2
KSORT_ERR_TIMEOUT = 5
KSORT_ERR_TOO_LARGE = 9
KSORT_NOALLOC_MAX_KEYS = 1 << 24
_NAMES = {F32: "f32", F64: "f64", U32: "u32"}

_HERE = os.path.dirname(os.path.abspath(__file__))
# KSORT_LIBRARY may name another build of the same sources (used for tuning sweeps).
_LIB_PATH = os.environ.get("KSORT_LIBRARY") or os.path.join(_HERE, "_lib", "libksort.so")
_lock = threading.Lock()
_lib = None


class KSortError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = f"{where}: {ksort_status_string(status)} (status {status})"
        if status == 4:
            msg += f" [{ksort_last_cuda_error()}]"
        super().__init__(msg)


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "large_items", "large_keys", "tiles", "small_items", "small_keys",
        "smem_levels", "lookback_steps", "items_pushed", "launches")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class Tuning(ctypes.Structure):
    _fields_ = [("cutoff", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("spin_limit_ms", ctypes.c_int32), ("tile_shape", ctypes.c_int32),
                ("wave_levels", ctypes.c_int32), ("medium_tiles", ctypes.c_int32),
                ("partition_form", ctypes.c_int32), ("sort_reserve", ctypes.c_int32),
                ("finish_in_tiles", ctypes.c_int32), ("finisher_threads", ctypes.c_int32),
                ("cluster_sort", ctypes.c_int32)]


def library_path() -> str:
    return _LIB_PATH


def load():
    """Loads the in-tree libksort.so, building it first if it is missing or stale."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import _build
        if not os.environ.get("KSORT_LIBRARY") and not _build.up_to_date():
            try:
                _build.build()
            except Exception as e:  # no toolkit: fail loudly, never fall back
                if not os.path.exists(_LIB_PATH):
                    raise RuntimeError(
                        f"libksort.so is not built and could not be built: {e}") from e
        L = ctypes.CDLL(_LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        sig = {
            "ksort_partition": (i32, [i32, vp, i64, vp, vp]),
            "ksort_partition_out": (i32, [i32, vp, vp, i64, vp, vp]),
            "ksort_partition_out_noalloc": (i32, [i32, vp, vp, i64, vp, vp]),
            "ksort_partition_exact": (i32, [i32, vp, vp, i64, vp, vp]),
            "ksort_sort": (i32, [i32, vp, i64, vp]),
            "ksort_sort_batched": (i32, [i32, vp, vp, i64, i64, vp]),
            "ksort_reserve_workspace": (i32, [i32, i64, i64, vp]),
            "ksort_release_workspace": (i32, [vp]),
            "ksort_get_device_error": (i32, [vp]),
            "ksort_get_stats": (i32, [vp, ctypes.POINTER(Stats)]),
            "ksort_set_phase_timing": (i32, [i32]),
            "ksort_get_phase_times": (i32, [vp, i32, ctypes.POINTER(ctypes.c_float),
                                            ctypes.POINTER(ctypes.c_int32)]),
            "ksort_set_tuning": (i32, [i32, ctypes.POINTER(Tuning)]),
            "ksort_get_tuning": (i32, [i32, ctypes.POINTER(Tuning)]),
            "ksort_max_cutoff": (i32, [i32]),
            "ksort_tile_keys": (i32, [i32]),
            "ksort_tile_shape": (i32, [i32, i32, ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(ctypes.c_int32)]),
            "ksort_partition_shape": (i32, [i32, i32, ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int32)]),
            "ksort_cluster_shape": (i32, [i32, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int64)]),
            "ksort_status_string": (ctypes.c_char_p, [i32]),
            "ksort_last_cuda_error": (ctypes.c_char_p, []),
            "ksort_selftest_wait_timeout": (i32, [i32, vp]),
            "ksort_selftest_noalloc_timeout": (i32, [i32, vp, vp]),
            "ksort_debug_trace": (i32, [vp, i64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return _lib


# ----------------------------------------------------------------------------- helpers
def dtype_code(t, dtype=None) -> int:
    """Key type code of a tensor. int32 tensors are taken as uint32 bit patterns only
    when ``dtype='u32'`` is given."""
    import torch
    if dtype is not None:
        code = {"f32": F32, "f64": F64, "u32": U32}[dtype]
        want = {F32: (torch.float32,), F64: (torch.float64,),
                U32: (torch.uint32, torch.int32)}[code]
        if t.dtype not in want:
            raise TypeError(f"tensor dtype {t.dtype} does not hold {dtype} keys")
        return code
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.uint32:
        return U32
    raise TypeError(f"unsupported key dtype {t.dtype} (float32, float64, uint32)")


def _stream(stream):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _check(status: int, where: str):
    if status != 0:
        raise KSortError(status, where)


# ----------------------------------------------------------------------------- C names
def ksort_partition(dtype: int, keys, n: int, key_index, stream=None):
    _check(load().ksort_partition(dtype, _ptr(keys), n, _ptr(key_index), _stream(stream)),
           "ksort_partition")


def ksort_partition_out(dtype: int, src, dst, n: int, key_index, stream=None):
    _check(load().ksort_partition_out(dtype, _ptr(src), _ptr(dst), n, _ptr(key_index),
                                      _stream(stream)), "ksort_partition_out")


def ksort_partition_out_noalloc(dtype: int, src, dst, n: int, key_index, stream=None):
    """Same as ksort_partition_out, with the kernels' scratch in a fixed device array
    (n <= KSORT_NOALLOC_MAX_KEYS). A device-side error shows as a negative key index."""
    _check(load().ksort_partition_out_noalloc(dtype, _ptr(src), _ptr(dst), n, _ptr(key_index),
                                              _stream(stream)), "ksort_partition_out_noalloc")


def ksort_partition_exact(dtype: int, src, dst, n: int, key_index, stream=None):
    """Steps 1-4 into ``dst`` in the paper's own element order (the hole scheme's layout)."""
    _check(load().ksort_partition_exact(dtype, _ptr(src), _ptr(dst), n, _ptr(key_index),
                                        _stream(stream)), "ksort_partition_exact")


def ksort_sort(dtype: int, keys, n: int, stream=None):
    _check(load().ksort_sort(dtype, _ptr(keys), n, _stream(stream)), "ksort_sort")


def ksort_sort_batched(dtype: int, keys, offsets, num_arrays: int, total_keys: int, stream=None):
    _check(load().ksort_sort_batched(dtype, _ptr(keys), _ptr(offsets), num_arrays, total_keys,
                                     _stream(stream)), "ksort_sort_batched")


def ksort_reserve_workspace(dtype: int, max_total_keys: int, max_arrays: int = 1, stream=None):
    _check(load().ksort_reserve_workspace(dtype, max_total_keys, max_arrays, _stream(stream)),
           "ksort_reserve_workspace")


def ksort_release_workspace(stream=None):
    _check(load().ksort_release_workspace(_stream(stream)), "ksort_release_workspace")


def ksort_get_device_error(stream=None) -> int:
    """Synchronises the stream; returns (and clears) the device status code."""
    return int(load().ksort_get_device_error(_stream(stream)))


def ksort_get_stats(stream=None) -> dict:
    s = Stats()
    _check(load().ksort_get_stats(_stream(stream), ctypes.byref(s)), "ksort_get_stats")
    return s.as_dict()


def ksort_set_phase_timing(enable: bool):
    _check(load().ksort_set_phase_timing(1 if enable else 0), "ksort_set_phase_timing")


def ksort_get_phase_history(stream=None, max_calls: int = 64) -> list:
    """Phase durations (ms) of up to max_calls of the latest timed calls on the stream,
    oldest first: [seed, partition passes, finisher] per sort, [partition] per partition."""
    out = (ctypes.c_float * (3 * max(1, max_calls)))()
    calls = ctypes.c_int32(0)
    _check(load().ksort_get_phase_times(_stream(stream), max_calls, out, ctypes.byref(calls)),
           "ksort_get_phase_times")
    return [[float(v) for v in out[3 * c:3 * c + 3] if v >= 0.0] for c in range(calls.value)]


def ksort_get_phase_times(stream=None) -> list:
    """Phase durations (ms) of the last timed call on the stream ([] if none)."""
    h = ksort_get_phase_history(stream, 1)
    return h[0] if h else []


def ksort_set_tuning(dtype: int, cutoff: int = 0, ctas_per_sm: int = 0, spin_limit_ms: int = 0,
                     tile_shape: int = 0, wave_levels: int = 0, medium_tiles: int = 0,
                     partition_form: int = 0, sort_reserve: int = 0, finish_in_tiles: int = 0,
                     finisher_threads: int = 0, cluster_sort: int = 0):
    """Zero arguments keep their value; ctas_per_sm=-1 restores "as many as fit",
    wave_levels=-1 the automatic level count, medium_tiles=-1 turns whole-item CTAs off,
    partition_form=-1 makes single partitions follow tile_shape instead of the ring,
    sort_reserve=-1 makes sort tile passes take their offsets by look-back,
    finish_in_tiles=W (tile shape 3) lets the tile kernel finish small sub-arrays while
    W or more of its CTAs wait for future tiles; -1 gives the finisher its own launch;
    finisher_threads (256, 512, 1024) sets the finisher CTA's size; cluster_sort=1 runs
    the upper levels of arrays that fit one thread-block cluster inside it, -1 not."""
    t = Tuning(cutoff, ctas_per_sm, spin_limit_ms, tile_shape, wave_levels, medium_tiles,
               partition_form, sort_reserve, finish_in_tiles, finisher_threads, cluster_sort)
    _check(load().ksort_set_tuning(dtype, ctypes.byref(t)), "ksort_set_tuning")


def ksort_get_tuning(dtype: int) -> dict:
    t = Tuning()
    _check(load().ksort_get_tuning(dtype, ctypes.byref(t)), "ksort_get_tuning")
    return {"cutoff": t.cutoff, "ctas_per_sm": t.ctas_per_sm, "spin_limit_ms": t.spin_limit_ms,
            "tile_shape": t.tile_shape, "wave_levels": t.wave_levels,
            "medium_tiles": t.medium_tiles, "partition_form": t.partition_form,
            "sort_reserve": t.sort_reserve, "finish_in_tiles": t.finish_in_tiles,
            "finisher_threads": t.finisher_threads, "cluster_sort": t.cluster_sort}


def ksort_tile_shape(dtype: int, shape: int) -> tuple[int, int, int]:
    """(threads, keys per tile-holding thread, form) of partition-pass form `shape`
    (1-based); form 0 registers, 1 shared-memory tile ring, 2 warp roles, 3 level-synchronous
    upper levels."""
    nt, ipt, fm = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().ksort_tile_shape(dtype, shape, ctypes.byref(nt), ctypes.byref(ipt),
                                   ctypes.byref(fm)), "ksort_tile_shape")
    return int(nt.value), int(ipt.value), int(fm.value)


def ksort_partition_shape(dtype: int, form: int) -> tuple[int, int, int]:
    """(threads, tile keys, CTAs per SM) of ring-partition configuration `form` (1-6)."""
    nt, tk, occ = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().ksort_partition_shape(dtype, form, ctypes.byref(nt), ctypes.byref(tk),
                                        ctypes.byref(occ)), "ksort_partition_shape")
    return int(nt.value), int(tk.value), int(occ.value)


def ksort_cluster_shape(dtype: int) -> tuple[int, int]:
    """(CTAs of the cluster form's thread-block cluster, most keys it holds) on the
    current device; (0, 0) when no cluster can run."""
    c, m = ctypes.c_int32(), ctypes.c_int64()
    _check(load().ksort_cluster_shape(dtype, ctypes.byref(c), ctypes.byref(m)),
           "ksort_cluster_shape")
    return int(c.value), int(m.value)


def ksort_max_cutoff(dtype: int) -> int:
    return int(load().ksort_max_cutoff(dtype))


def ksort_tile_keys(dtype: int) -> int:
    return int(load().ksort_tile_keys(dtype))


def ksort_selftest_wait_timeout(limit_ms: int, stream=None):
    _check(load().ksort_selftest_wait_timeout(limit_ms, _stream(stream)),
           "ksort_selftest_wait_timeout")


def ksort_selftest_noalloc_timeout(limit_ms: int, key_index, stream=None):
    """key_index: a device int64 tensor of one element (receives -KSORT_ERR_TIMEOUT)."""
    _check(load().ksort_selftest_noalloc_timeout(limit_ms, _ptr(key_index), _stream(stream)),
           "ksort_selftest_noalloc_timeout")


def ksort_debug_trace(trace=None, tickets: int = 0):
    """Installs (or with None removes) a device uint64 buffer of 8 * tickets timestamps."""
    _check(load().ksort_debug_trace(_ptr(trace) if trace is not None else None,
                                    tickets if trace is not None else 0), "ksort_debug_trace")


def ksort_status_string(status: int) -> str:
    return load().ksort_status_string(status).decode()


def ksort_last_cuda_error() -> str:
    return load().ksort_last_cuda_error().decode()


# ----------------------------------------------------------------------------- tensors
def partition_(t, dtype=None, stream=None) -> int:
    """Steps 1-4 in place on a 1-D CUDA tensor; returns the key's final index."""
    import torch
    code = dtype_code(t, dtype)
    idx = torch.empty(1, dtype=torch.int64, device=t.device)
    ksort_partition(code, t, t.numel(), idx, stream)
    return int(idx.item())


def partition_out(src, dst, dtype=None, stream=None):
    """Steps 1-4 from ``src`` into ``dst``; returns the key index as a device tensor."""
    import torch
    code = dtype_code(src, dtype)
    if dst.dtype != src.dtype or dst.numel() != src.numel():
        raise ValueError("dst must match src in dtype and size")
    idx = torch.empty(1, dtype=torch.int64, device=src.device)
    ksort_partition_out(code, src, dst, src.numel(), idx, stream)
    return idx


def partition_exact(src, dst, dtype=None, stream=None) -> int:
    """Steps 1-4 from ``src`` into ``dst`` with the paper's element order; returns the
    key's final index."""
    import torch
    code = dtype_code(src, dtype)
    if dst.dtype != src.dtype or dst.numel() != src.numel():
        raise ValueError("dst must match src in dtype and size")
    idx = torch.empty(1, dtype=torch.int64, device=src.device)
    ksort_partition_exact(code, src, dst, src.numel(), idx, stream)
    return int(idx.item())


def sort_(t, dtype=None, stream=None):
    """Steps 1-6: sorts a 1-D CUDA tensor ascending, in place."""
    ksort_sort(dtype_code(t, dtype), t, t.numel(), stream)
    return t


def sort_batched_(flat, offsets, dtype=None, stream=None):
    """Sorts flat[offsets[r]:offsets[r+1]] for every r in one launch (int64 offsets
    on the device)."""
    import torch
    if offsets.dtype != torch.int64 or not offsets.is_cuda:
        raise ValueError("offsets must be a CUDA int64 tensor")
    ksort_sort_batched(dtype_code(flat, dtype), flat, offsets, offsets.numel() - 1,
                       flat.numel(), stream)
    return flat
