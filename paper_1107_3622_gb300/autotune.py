"""Autotuner of libksort: picks, for one key type and workload (a sort, a batch of sorts
or a single partition), the form of the partition passes (kernel kind and threads x
keys per thread), the number of level-synchronous levels when that form is the wave
form, the shared-memory cutoff below which sub-arrays are finished in SMEM, and the
finisher's CTAs per SM and threads per CTA, whether a single array that fits one
thread-block cluster runs its upper levels there, and for tile shape 3 whether the tile kernel finishes the small
sub-arrays itself (and its park threshold). For a single partition it picks the configuration of the ring
partition (tile size, slots, CTAs per SM), or the tile shape's own form if that wins.

Every candidate runs the real workload through the C ABI on the current device. The
input is restored from a pristine copy and L2 flushed before each timed run, and CUDA
events time the call alone. The median over `reps` runs decides. The search is
coordinate descent: tile shape, then wave levels (wave forms only), then the fused
finisher (tile shape 3 only), then cutoff, then finisher CTAs and their size, repeated while
something improves. The winner is checked for a sorted output, applied with
ksort_set_tuning, and stored in a JSON cache keyed by device, library sources, key
type and workload, so later processes can apply it without searching.
"""
from __future__ import annotations

import hashlib
import json
import math
import os
import statistics
import threading

import numpy as np

from . import F32, F64, U32, _HERE, ksort_get_device_error, ksort_get_tuning, \
    ksort_max_cutoff, ksort_partition_out, ksort_reserve_workspace, ksort_set_tuning, \
    ksort_sort, ksort_sort_batched

_NAMES = {F32: "f32", F64: "f64", U32: "u32"}
CUTOFFS = (1024, 2048, 4096, 8192, 16384)
SHAPES = tuple(range(1, 13))
WAVE_SHAPES = (10, 11, 12)
# -1: the library's automatic count; fixed counts around the depth of random inputs
WAVE_LEVELS = (-1, 6, 9, 12, 15, 18)
FINISHER_CTAS = (-1, 3, 2)
# single partitions: the ring partition's configurations, or -1 (the tile shape's form)
PARTITION_FORMS = (1, 2, 3, 4, 5, 6, -1)
# tile shape 3: -1 (a separate finisher launch) or the fused finisher's park threshold
FINISH_IN_TILES = (-1, 4, 16, 64)
FUSED_SHAPE = 3
FINISHER_THREADS = (256, 512, 1024)
CLUSTER_SORT = (-1, 1)
_L2_FLUSH_BYTES = 256 << 20
_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("KSORT_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "ksort_gb300", "autotune.json")


def library_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(_HERE, "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def device_key() -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|sm{p.major}{p.minor}|{p.multi_processor_count}"


def workload_key(kind: str, dtype: int, n: int = 0, lengths=None) -> str:
    """Sorts and partitions are bucketed by log2 n; batches by array count and keys."""
    if kind in ("sort", "partition"):
        return f"{kind}:{_NAMES[dtype]}:2^{round(math.log2(max(n, 2)))}"
    lengths = np.asarray(lengths)
    total = int(lengths.sum())
    return (f"batched:{_NAMES[dtype]}:{len(lengths)}x"
            f"[{int(lengths.min())},{int(lengths.max())}]:2^{round(math.log2(max(total, 2)))}")


def _load_cache() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key: str, entry: dict):
    with _lock:
        c = _load_cache()
        c[key] = entry
        path = cache_path()
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(c, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def shapes_suffix(shapes) -> str:
    """Cache-key suffix of a search limited to some tile shapes ('' when unlimited)."""
    return f"|shapes={','.join(str(x) for x in shapes)}" if shapes else ""


def _full_key(kind, dtype, n, lengths, shapes=None) -> str:
    k = f"{device_key()}|{library_hash()}|{workload_key(kind, dtype, n, lengths)}"
    return k + shapes_suffix(shapes)


def apply_cached(kind: str, dtype: int, n: int = 0, lengths=None, shapes=None) -> dict | None:
    """Applies a cached choice for this workload; returns it, or None if none is cached."""
    e = _load_cache().get(_full_key(kind, dtype, n, lengths, shapes))
    if not e:
        return None
    t = e["tuning"]
    ksort_set_tuning(dtype, cutoff=t["cutoff"], ctas_per_sm=t["ctas_per_sm"] or -1,
                     tile_shape=t["tile_shape"], wave_levels=t.get("wave_levels", -1),
                     partition_form=t.get("partition_form", 5),
                     finish_in_tiles=t.get("finish_in_tiles", -1),
                     finisher_threads=t.get("finisher_threads", 256),
                     cluster_sort=t.get("cluster_sort", -1))
    return e


class _Runner:
    """Holds the workload's pristine input and runs/times one call."""

    def __init__(self, kind, dtype, n, lengths, seed):
        import torch
        import ksort_inputs as gen
        self.kind, self.dtype = kind, dtype
        name = _NAMES[dtype]
        if kind in ("sort", "partition"):
            self.total, self.offsets, self.arrays = n, None, 1
        else:
            off = gen.offsets_from_lengths(np.asarray(lengths, np.int64))
            self.total, self.arrays = int(off[-1]), len(lengths)
            self.offsets = torch.from_numpy(off).cuda()
        self.pristine = gen.uniform_torch(name, seed, self.total, device="cuda")
        self.keys = torch.empty_like(self.pristine)
        self.index = torch.zeros(1, dtype=torch.int64, device="cuda")
        self.flush = torch.empty(_L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def call(self):
        if self.kind == "partition":  # out of place: the input stays pristine
            ksort_partition_out(self.dtype, self.pristine, self.keys, self.total, self.index)
        elif self.kind == "sort":
            ksort_sort(self.dtype, self.keys, self.total)
        else:
            ksort_sort_batched(self.dtype, self.keys, self.offsets, self.arrays, self.total)

    def time(self, reps: int) -> float:
        import torch
        ksort_reserve_workspace(self.dtype, self.total, self.arrays)
        self.keys.copy_(self.pristine)
        self.call()  # warm-up (also grows nothing later)
        ms = []
        for _ in range(reps):
            self.keys.copy_(self.pristine)
            self.flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            self.call()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        st = ksort_get_device_error()
        if st:
            raise RuntimeError(f"device error {st} while tuning")
        return statistics.median(ms)

    def check_sorted(self) -> bool:
        import torch
        self.keys.copy_(self.pristine)
        self.call()
        k = self.keys.view(torch.int32).to(torch.int64) & 0xFFFFFFFF \
            if self.dtype == U32 else self.keys
        if self.kind == "partition":
            i = int(self.index.item())
            src = self.pristine.view(torch.int32).to(torch.int64) & 0xFFFFFFFF \
                if self.dtype == U32 else self.pristine
            return bool(k[i] == src[0]) and bool((k[:i] < k[i]).all()) and \
                bool((k[i + 1:] >= k[i]).all())
        if self.kind == "sort":
            return bool((k[1:] >= k[:-1]).all())
        off = self.offsets
        ok = k[1:] >= k[:-1]
        # pairs that straddle two arrays may decrease
        starts = off[1:-1]
        starts = starts[(starts > 0) & (starts < self.total)] - 1
        ok[starts] = True
        return bool(ok.all())


def autotune(kind: str, dtype: int, n: int = 0, lengths=None, reps: int = 3,
             seed: int | None = None, use_cache: bool = True, max_rounds: int = 2,
             shapes=None) -> dict:
    """Searches and applies the best tuning for one workload; returns the cache entry.
    `shapes` limits the tile shapes searched (default: all)."""
    import ksort_inputs as gen
    if kind not in ("sort", "batched", "partition"):
        raise ValueError("kind is 'sort', 'partition' or 'batched'")
    if shapes is not None and not set(shapes) <= set(SHAPES):
        raise ValueError("unknown tile shape")
    if use_cache:
        e = apply_cached(kind, dtype, n, lengths, shapes)
        if e is not None:
            return dict(e, cached=True)
    if seed is None:
        seed = gen.seed_for(4, 0, 0)
    before = ksort_get_tuning(dtype)
    runner = _Runner(kind, dtype, n, lengths, seed)
    maxc = ksort_max_cutoff(dtype)
    cutoffs = [c for c in CUTOFFS if c <= maxc]
    best = {"tile_shape": before["tile_shape"], "cutoff": before["cutoff"],
            "ctas_per_sm": before["ctas_per_sm"] or -1,
            "wave_levels": before.get("wave_levels", -1),
            "partition_form": before.get("partition_form", 5),
            "finish_in_tiles": before.get("finish_in_tiles", -1),
            "finisher_threads": before.get("finisher_threads", 256),
            "cluster_sort": before.get("cluster_sort", -1)}
    if shapes and best["tile_shape"] not in shapes:
        best["tile_shape"] = shapes[0]
    tried = {}

    def measure(cfg) -> float:
        if cfg["tile_shape"] not in WAVE_SHAPES:
            cfg["wave_levels"] = -1  # no effect outside the wave form
        if cfg["tile_shape"] != FUSED_SHAPE:
            cfg["finish_in_tiles"] = -1  # only tile shape 3 has the fused finisher
        key = (cfg["tile_shape"], cfg["cutoff"], cfg["ctas_per_sm"], cfg["wave_levels"],
               cfg["partition_form"], cfg["finish_in_tiles"], cfg["finisher_threads"],
               cfg["cluster_sort"])
        if key not in tried:
            ksort_set_tuning(dtype, cutoff=cfg["cutoff"], ctas_per_sm=cfg["ctas_per_sm"],
                             tile_shape=cfg["tile_shape"], wave_levels=cfg["wave_levels"],
                             partition_form=cfg["partition_form"],
                             finish_in_tiles=cfg["finish_in_tiles"],
                             finisher_threads=cfg["finisher_threads"],
                             cluster_sort=cfg["cluster_sort"])
            tried[key] = runner.time(reps)
        return tried[key]

    best_ms = measure(best)
    axes = (("cluster_sort", CLUSTER_SORT if kind == "sort" else (-1,)),
            ("tile_shape", tuple(shapes) if shapes else SHAPES), ("wave_levels", WAVE_LEVELS),
            ("finish_in_tiles", FINISH_IN_TILES), ("cutoff", cutoffs),
            ("ctas_per_sm", FINISHER_CTAS), ("finisher_threads", FINISHER_THREADS))
    if kind == "partition":
        # the ring partition's configuration; the CTA shape only matters for the tile
        # shape's own forms (part_kernel or the split pair), under partition_form -1
        axes = (("partition_form", PARTITION_FORMS), ("tile_shape", SHAPES[:3] + WAVE_SHAPES))
    for _ in range(max_rounds):
        improved = False
        for name, values in axes:
            if name == "wave_levels" and best["tile_shape"] not in WAVE_SHAPES:
                continue
            if name == "finish_in_tiles" and best["tile_shape"] != FUSED_SHAPE:
                continue
            if kind == "partition" and name == "tile_shape" and best["partition_form"] != -1:
                continue
            for v in values:
                cfg = dict(best, **{name: v})
                ms = measure(cfg)
                if ms < best_ms * 0.995:
                    best, best_ms, improved = cfg, ms, True
        if not improved:
            break
    ksort_set_tuning(dtype, cutoff=best["cutoff"], ctas_per_sm=best["ctas_per_sm"],
                     tile_shape=best["tile_shape"], wave_levels=best["wave_levels"],
                     partition_form=best["partition_form"],
                     finish_in_tiles=best["finish_in_tiles"],
                     finisher_threads=best["finisher_threads"],
                     cluster_sort=best["cluster_sort"])
    if not runner.check_sorted():
        ksort_set_tuning(dtype, cutoff=before["cutoff"], ctas_per_sm=before["ctas_per_sm"] or -1,
                         tile_shape=before["tile_shape"], wave_levels=before.get("wave_levels", -1),
                         partition_form=before.get("partition_form", 5),
                         finish_in_tiles=before.get("finish_in_tiles", -1),
                         finisher_threads=before.get("finisher_threads", 256),
                         cluster_sort=before.get("cluster_sort", -1))
        raise RuntimeError("autotuned configuration produced an unsorted output")
    entry = {"workload": workload_key(kind, dtype, n, lengths), "device": device_key(),
             "library": library_hash(), "tuning": best, "ms": round(best_ms, 4),
             "keys": runner.total, "reps": reps,
             "candidates": [{"tile_shape": k[0], "cutoff": k[1], "ctas_per_sm": k[2],
                             "wave_levels": k[3], "partition_form": k[4],
                             "finish_in_tiles": k[5], "finisher_threads": k[6],
                             "cluster_sort": k[7], "ms": round(v, 4)}
                            for k, v in sorted(tried.items())]}
    if use_cache:
        _store(_full_key(kind, dtype, n, lengths, shapes), entry)
    return dict(entry, cached=False)


def reset(dtype: int):
    """Back to the library defaults (tile shape 1, default cutoff, all finisher CTAs,
    automatic wave levels, ring partition configuration 5, separate finisher launch of
    256-thread CTAs, no cluster form)."""
    default_cutoff = {F32: 4096, F64: 2048, U32: 4096}[dtype]
    ksort_set_tuning(dtype, cutoff=default_cutoff, ctas_per_sm=-1, tile_shape=1, wave_levels=-1,
                     partition_form=5, finish_in_tiles=-1, finisher_threads=256,
                     cluster_sort=-1)
