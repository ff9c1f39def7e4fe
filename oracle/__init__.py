"""ctypes front end for the K-sort C oracle (arxiv 1107.3622, Section 1.1, Steps 1-6).

TEST INFRASTRUCTURE ONLY. The test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only users. The GPU library never imports
this package and this package never imports the GPU library.

``build()`` compiles ``ksort_ref.c`` with gcc into ``oracle/_build/``; every other
function builds on first use when the shared object is missing or stale.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libksort_ref.so")
# A test may point the wrapper at another build of the same source (the mutation
# tests compile deliberately broken copies); nothing is built in that case.
_SO_OVERRIDE = os.environ.get("KSORT_ORACLE_SO")
_SOURCES = ("ksort_ref.c", "ksort_ref_body.h", "ksort_ref.h")
_lock = threading.Lock()
_lib = None

SUFFIX = {np.dtype(np.float32): "f32", np.dtype(np.float64): "f64", np.dtype(np.uint32): "u32"}
_CTYPE = {"f32": ctypes.c_float, "f64": ctypes.c_double, "u32": ctypes.c_uint32}


class Stats(ctypes.Structure):
    _fields_ = [("calls", ctypes.c_uint64), ("compares", ctypes.c_uint64),
                ("max_depth", ctypes.c_uint64)]


class Trace(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int64), ("count", ctypes.c_int64),
                ("left", ctypes.c_void_p), ("right", ctypes.c_void_p),
                ("index", ctypes.c_void_p), ("flag", ctypes.c_void_p),
                ("key", ctypes.c_void_p), ("temp", ctypes.c_void_p),
                ("snapshot", ctypes.c_void_p)]


def _stale() -> bool:
    if not os.path.exists(_SO):
        return True
    t = os.path.getmtime(_SO)
    return any(os.path.getmtime(os.path.join(_HERE, s)) > t for s in _SOURCES)


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2, C99, no target-specific flags)."""
    if _SO_OVERRIDE:
        return _SO_OVERRIDE
    with _lock:
        if force or _stale():
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _SO + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-Wall", "-Wextra",
                   os.path.join(_HERE, "ksort_ref.c"), "-o", tmp]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        for sfx, ct in _CTYPE.items():
            f = getattr(L, f"ksort_ref_partition_{sfx}")
            f.restype = ctypes.c_int64
            f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                          ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p,
                          ctypes.POINTER(ctypes.c_uint64)]
            f = getattr(L, f"ksort_ref_sort_{sfx}")
            f.restype = ctypes.c_int
            f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(Stats),
                          ctypes.POINTER(Trace)]
            f = getattr(L, f"ksort_ref_sort_batched_{sfx}")
            f.restype = ctypes.c_int
            f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                          ctypes.POINTER(Stats)]
        _lib = L
    return _lib


def _suffix(a: np.ndarray) -> str:
    try:
        return SUFFIX[a.dtype]
    except KeyError:
        raise TypeError(f"oracle supports float32, float64 and uint32, not {a.dtype}") from None


def _ptr(a: np.ndarray) -> int:
    if not a.flags["C_CONTIGUOUS"] or not a.flags["WRITEABLE"]:
        raise ValueError("oracle arrays must be C-contiguous and writeable")
    return a.ctypes.data


def partition(a: np.ndarray, left: int = 0, right: int | None = None):
    """Steps 1-4 on a[left..right] in place. Returns (i, flag, temp, compares)."""
    sfx = _suffix(a)
    if right is None:
        right = len(a) - 1
    if not (0 <= left < right < len(a)):
        raise ValueError("need 0 <= left < right < len(a)")
    flag = ctypes.c_int32(0)
    temp = _CTYPE[sfx]()
    cmp_ = ctypes.c_uint64(0)
    i = getattr(lib(), f"ksort_ref_partition_{sfx}")(
        _ptr(a), left, right, ctypes.byref(flag), ctypes.cast(ctypes.byref(temp), ctypes.c_void_p),
        ctypes.byref(cmp_))
    return int(i), int(flag.value), (temp.value if flag.value else None), int(cmp_.value)


def sort(a: np.ndarray) -> Stats:
    """Steps 1-6 on the whole array, in place. Returns the call/compare counters."""
    sfx = _suffix(a)
    st = Stats()
    rc = getattr(lib(), f"ksort_ref_sort_{sfx}")(_ptr(a), len(a), ctypes.byref(st), None)
    if rc != 0:
        raise MemoryError("oracle could not allocate its stack")
    return st


def sort_traced(a: np.ndarray, capacity: int | None = None, snapshots: bool = True):
    """Steps 1-6 with a per-call record. Returns (stats, rows); each row is a dict
    with left, right, index, flag, key, temp and (optionally) the array after the call."""
    sfx = _suffix(a)
    n = len(a)
    cap = capacity if capacity is not None else max(1, n)
    left = np.zeros(cap, np.int64); right = np.zeros(cap, np.int64)
    index = np.zeros(cap, np.int64); flag = np.zeros(cap, np.int32)
    key = np.zeros(cap, a.dtype); temp = np.zeros(cap, a.dtype)
    snap = np.zeros((cap, n), a.dtype) if snapshots else None
    tr = Trace(cap, 0, left.ctypes.data, right.ctypes.data, index.ctypes.data, flag.ctypes.data,
               key.ctypes.data, temp.ctypes.data, snap.ctypes.data if snapshots else None)
    st = Stats()
    rc = getattr(lib(), f"ksort_ref_sort_{sfx}")(_ptr(a), n, ctypes.byref(st), ctypes.byref(tr))
    if rc != 0:
        raise MemoryError("oracle could not allocate its stack")
    rows = []
    for c in range(min(tr.count, cap)):
        rows.append(dict(left=int(left[c]), right=int(right[c]), index=int(index[c]),
                         flag=int(flag[c]), key=key[c].item(),
                         temp=temp[c].item() if flag[c] else None,
                         array=snap[c].copy() if snapshots else None))
    return st, rows


def sort_batched(flat: np.ndarray, offsets: np.ndarray) -> Stats:
    """Sorts flat[offsets[r]:offsets[r+1]] for every r, in place."""
    sfx = _suffix(flat)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    st = Stats()
    rc = getattr(lib(), f"ksort_ref_sort_batched_{sfx}")(_ptr(flat), off.ctypes.data,
                                                         len(off) - 1, ctypes.byref(st))
    if rc != 0:
        raise ValueError("oracle: bad offsets or allocation failure")
    return st
