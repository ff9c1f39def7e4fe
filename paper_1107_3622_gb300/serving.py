"""Serving form of K-sort: a continuous-batching request loop over ksort_sort_batched,
with admission by free HBM.

Requests (a key type, a length, a seed) arrive over time with their keys in page-locked
host memory: one flat host pool per key type holds every request's keys in arrival
order, standing in for buffers handed over by clients. A request's sorted keys go back
to the same place in that pool.

The server holds two kinds of device memory, both allocated once at start-up:
  - `slots` stream slots, each with its own CUDA stream, a sort workspace reserved for
    `slot_keys` keys and `max_arrays` arrays (scratch + work queue), and an offsets
    buffer;
  - a key arena: one device buffer sized from the HBM left free after the slot
    workspaces (torch.cuda.mem_get_info, less a headroom, optionally capped), carved
    into batch buffers by a first-fit allocator and given back when a batch completes,
    never freed to the driver while the server runs.
When a slot is free the planner admits waiting requests into one batch:
  - a FIFO prefix of one key type's queue (the type whose oldest request has waited
    longest), so the batch is one contiguous range of that type's host pool;
  - no more than a slot holds (`slot_keys` keys, `max_arrays` arrays) and no more than
    the largest free block of the arena: admission is by free HBM. When even the oldest
    request does not fit, nothing is admitted until a running batch gives its buffer
    back (FIFO order, so a large request is never starved by smaller ones behind it).
An admitted batch runs on its slot's stream: the copy of its keys from the host pool
into its arena buffer, one ksort_sort_batched call (the persistent kernels), the copy of
the sorted keys back to the host pool, and a completion event. Batches on different
slots overlap on the device. A request's latency runs from its arrival to its batch's
completion event (host-to-device copy, sort and device-to-host copy included), on the
device clock aligned with the host clock at start.

Every step of the sort runs in libksort's kernels; this module schedules, allocates,
copies and reads events.
"""
from __future__ import annotations

import bisect
import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

import ksort_inputs as gen

from . import F32, U32, dtype_code, ksort_get_device_error, ksort_reserve_workspace, \
    ksort_sort, ksort_sort_batched

KEY_TYPES = ("f32", "u32")
KEY_BYTES = {"f32": 4, "u32": 4}
ARENA_ALIGN = 256


@dataclass
class Request:
    rid: int
    arrival_s: float     # seconds after the start of the run
    dtype: str           # "f32" or "u32"
    n: int
    seed: int
    pool_off: int = 0    # first key in its type's host pool
    batch: int = -1      # batch that served it
    admit_s: float = math.nan
    done_s: float = math.nan


def poisson_requests(count: int, rate_per_s: float, lo: int = 1_000, hi: int = 10_000_000,
                     seed: int | None = None) -> list[Request]:
    """`count` requests with exponential gaps (rate `rate_per_s`), lengths
    round(exp(U[ln lo, ln hi])), key type f32 or u32 with probability 1/2 each.
    Every draw is a SplitMix64 stream of its own."""
    if seed is None:
        seed = gen.seed_for(5, 0, 0)
    u_gap = gen.uniform_f64(seed ^ 0x1, count)
    u_len = gen.uniform_f64(seed ^ 0x2, count)
    u_typ = gen.uniform_f64(seed ^ 0x3, count)
    gaps = -np.log1p(-u_gap) / rate_per_s
    arrivals = np.cumsum(gaps) - gaps[0]
    lengths = np.rint(np.exp(math.log(lo) + u_len * (math.log(hi) - math.log(lo)))).astype(np.int64)
    reqs = []
    for i in range(count):
        reqs.append(Request(rid=i, arrival_s=float(arrivals[i]),
                            dtype="f32" if u_typ[i] < 0.5 else "u32",
                            n=int(lengths[i]), seed=gen.seed_for(5, 1, i)))
    return reqs


def mean_length(lo: int = 1_000, hi: int = 10_000_000) -> float:
    """E[round(exp(U[ln lo, ln hi]))] ~ (hi - lo) / ln(hi / lo)."""
    return (hi - lo) / math.log(hi / lo)


def align_up(nbytes: int, align: int = ARENA_ALIGN) -> int:
    return (nbytes + align - 1) // align * align


# ----------------------------------------------------------------------------- arena
class Arena:
    """First-fit allocator over the byte range [0, size) of one device buffer.

    Blocks are `align`-byte multiples at `align`-byte offsets; free blocks are kept
    sorted by offset and merged with their neighbours when a block comes back, so a
    drained arena is one free block again. Host-side bookkeeping only: the device
    buffer itself is allocated once by its owner."""

    def __init__(self, size: int, align: int = ARENA_ALIGN):
        if size < align:
            raise ValueError(f"arena of {size} bytes is smaller than one {align}-byte block")
        self.align = align
        self.size = size // align * align
        self._free_off = [0]           # sorted offsets of the free blocks
        self._free_len = [self.size]   # their lengths
        self._used = {}                # offset -> length of each allocated block
        self.in_use = 0
        self.peak_in_use = 0

    def largest_free(self) -> int:
        return max(self._free_len, default=0)

    def alloc(self, nbytes: int) -> int | None:
        """Offset of a new block of at least nbytes, or None when no free block holds it."""
        need = align_up(max(nbytes, 1), self.align)
        for i, ln in enumerate(self._free_len):
            if ln >= need:
                off = self._free_off[i]
                if ln == need:
                    del self._free_off[i], self._free_len[i]
                else:
                    self._free_off[i] += need
                    self._free_len[i] -= need
                self._used[off] = need
                self.in_use += need
                self.peak_in_use = max(self.peak_in_use, self.in_use)
                return off
        return None

    def free(self, off: int):
        need = self._used.pop(off)     # KeyError: not a block of this arena
        self.in_use -= need
        i = bisect.bisect_left(self._free_off, off)
        self._free_off.insert(i, off)
        self._free_len.insert(i, need)
        if i + 1 < len(self._free_off) and off + need == self._free_off[i + 1]:
            self._free_len[i] += self._free_len.pop(i + 1)
            self._free_off.pop(i + 1)
        if i > 0 and self._free_off[i - 1] + self._free_len[i - 1] == off:
            self._free_len[i - 1] += self._free_len.pop(i)
            self._free_off.pop(i)

    def blocks(self) -> int:
        return len(self._used)


# ----------------------------------------------------------------------------- planner
@dataclass
class Batch:
    bid: int
    dtype: str
    reqs: list
    base: int            # first key of the batch in its type's host pool
    total: int           # keys in the batch
    dev_off: int = -1    # byte offset of its buffer in the arena (-1: no arena)
    nbytes: int = 0
    slot: int = -1


class Planner:
    """Admission and batching policy, independent of the GPU (tested on CPU).

    With `budget_bytes` the planner owns an Arena of that size and admits a batch only
    into a free block of it; `complete` gives the block back."""

    def __init__(self, slot_keys: int, max_arrays: int, budget_bytes: int | None = None):
        if slot_keys < 1 or max_arrays < 1:
            raise ValueError("slot capacity must be positive")
        self.slot_keys = slot_keys
        self.max_arrays = max_arrays
        self.arena = Arena(budget_bytes) if budget_bytes is not None else None
        self.queues = {t: deque() for t in KEY_TYPES}
        self.refusals = 0    # next_batch calls that found requests waiting but no room
        self._next = 0

    def arrive(self, r: Request):
        if r.n > self.slot_keys:
            raise ValueError(f"request {r.rid} ({r.n} keys) exceeds a slot ({self.slot_keys})")
        if self.arena is not None and align_up(r.n * KEY_BYTES[r.dtype]) > self.arena.size:
            raise ValueError(f"request {r.rid} ({r.n} keys) exceeds the HBM budget "
                             f"({self.arena.size} bytes)")
        q = self.queues[r.dtype]
        if q and r.pool_off != q[-1].pool_off + q[-1].n:
            raise ValueError("requests of one key type must be contiguous in arrival order")
        q.append(r)

    def waiting(self) -> int:
        return sum(len(q) for q in self.queues.values())

    def next_batch(self) -> Batch | None:
        """The batch a free slot should run now, or None when nothing waits or the
        oldest waiting request does not fit the arena's largest free block."""
        heads = [(q[0].arrival_s, t) for t, q in self.queues.items() if q]
        if not heads:
            return None
        _, t = min(heads)
        q = self.queues[t]
        kb = KEY_BYTES[t]
        room = self.arena.largest_free() if self.arena is not None else None
        reqs, total = [], 0
        while q and len(reqs) < self.max_arrays and total + q[0].n <= self.slot_keys:
            if room is not None and align_up((total + q[0].n) * kb) > room:
                break
            r = q.popleft()
            reqs.append(r)
            total += r.n
        if not reqs:
            self.refusals += 1
            return None
        b = Batch(bid=self._next, dtype=t, reqs=reqs, base=reqs[0].pool_off, total=total,
                  nbytes=total * kb)
        if self.arena is not None:
            b.dev_off = self.arena.alloc(b.nbytes)
            assert b.dev_off is not None  # the largest free block holds it
        self._next += 1
        for r in reqs:
            r.batch = b.bid
        return b

    def complete(self, b: Batch):
        """The batch's device buffer is no longer read or written: give it back."""
        if self.arena is not None and b.dev_off >= 0:
            self.arena.free(b.dev_off)
            b.dev_off = -1


# ----------------------------------------------------------------------------- host pools
class HostPools:
    """One flat page-locked host array per key type holding every request's keys in
    arrival order (u32 keys as int32 bit patterns). Each array is ordinary host memory
    registered with the CUDA driver, so that copies between it and the device run
    asynchronously on a slot's stream; `close` unregisters it."""

    NP_TYPES = {"f32": np.float32, "u32": np.int32}

    def __init__(self, reqs: list[Request], fill: bool = True):
        import torch
        sizes = {t: 0 for t in KEY_TYPES}
        for r in reqs:
            r.pool_off = sizes[r.dtype]
            sizes[r.dtype] += r.n
        self.arrays, self.tensors, self._registered = {}, {}, []
        for t in KEY_TYPES:
            a = np.empty(max(sizes[t], 1), dtype=self.NP_TYPES[t])
            rc = torch.cuda.cudart().cudaHostRegister(a.ctypes.data, a.nbytes, 0)
            if int(rc) != 0:
                self.close()
                raise RuntimeError(f"cudaHostRegister of {a.nbytes} bytes failed ({int(rc)})")
            self._registered.append(a)
            self.arrays[t] = a
            self.tensors[t] = torch.from_numpy(a)
        if fill:
            for r in reqs:
                self.keys(r).copy_(request_keys(r, device="cuda"))
            torch.cuda.synchronize()

    def keys(self, r: Request):
        """The request's slice of its type's pool (a CPU tensor on page-locked memory)."""
        return self.tensors[r.dtype][r.pool_off:r.pool_off + r.n]

    def nbytes(self) -> int:
        return sum(a.nbytes for a in self._registered)

    def close(self):
        import torch
        while self._registered:
            a = self._registered.pop()
            torch.cuda.cudart().cudaHostUnregister(a.ctypes.data)
        self.tensors, self.arrays = {}, {}

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def build_pools(reqs: list[Request]) -> HostPools:
    """Host pools of every request's keys, page-locked, filled from each request's seed."""
    return HostPools(reqs)


def request_keys(r: Request, device="cuda"):
    """The request's original keys, regenerated from its seed."""
    return gen.uniform_torch(r.dtype, r.seed, r.n, device=device)


# ----------------------------------------------------------------------------- server
@dataclass
class Slot:
    stream: object
    offsets_dev: object
    offsets_host: object
    batch: Batch | None = None
    event: object = None


@dataclass
class RunResult:
    requests: list
    batches: list
    keys: int
    wall_s: float
    max_in_flight: int
    latencies_s: np.ndarray = field(default_factory=lambda: np.zeros(0))
    hbm: dict = field(default_factory=dict)

    def summary(self) -> dict:
        lat = self.latencies_s * 1e3
        wait = np.array([r.admit_s - r.arrival_s for r in self.requests]) * 1e3
        span = max(r.done_s for r in self.requests) - min(r.arrival_s for r in self.requests)
        out = {
            "requests": len(self.requests), "keys": int(self.keys),
            "batches": len(self.batches), "max_batches_in_flight": self.max_in_flight,
            "keys_per_s": round(self.keys / span, 1) if span > 0 else None,
            "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "mean_ms": round(float(lat.mean()), 3),
            "p50_admission_wait_ms": round(float(np.percentile(wait, 50)), 3),
            "p99_admission_wait_ms": round(float(np.percentile(wait, 99)), 3),
            "span_s": round(span, 4),
        }
        out.update(self.hbm)
        return out


class Server:
    """`slots` stream slots and a key arena sized from the HBM left free after their
    workspaces: free - `headroom_bytes`, capped at `budget_bytes` when given."""

    def __init__(self, slots: int = 4, slot_keys: int = 1 << 27, max_arrays: int = 4096,
                 budget_bytes: int | None = None, headroom_bytes: int = 4 << 30):
        import torch
        self.slots = []
        for _ in range(slots):
            s = torch.cuda.Stream()
            for t in KEY_TYPES:
                ksort_reserve_workspace(F32 if t == "f32" else U32, slot_keys, max_arrays, s)
            self.slots.append(Slot(
                stream=s,
                offsets_dev=torch.empty(max_arrays + 1, dtype=torch.int64, device="cuda"),
                offsets_host=torch.empty(max_arrays + 1, dtype=torch.int64).pin_memory()))
        torch.cuda.synchronize()
        free, total = torch.cuda.mem_get_info()
        budget = free - headroom_bytes
        if budget_bytes is not None:
            budget = min(budget, budget_bytes)
        budget = budget // ARENA_ALIGN * ARENA_ALIGN
        if budget < ARENA_ALIGN:
            raise RuntimeError(f"no HBM left for the key arena ({free} bytes free, "
                               f"{headroom_bytes} kept back)")
        self.arena_buf = torch.empty(budget, dtype=torch.uint8, device="cuda")
        self.planner = Planner(slot_keys, max_arrays, budget)
        self.hbm = {"device_bytes": int(total), "free_after_workspaces_bytes": int(free),
                    "headroom_bytes": int(headroom_bytes), "budget_bytes": int(budget)}

    def close(self):
        import torch
        torch.cuda.synchronize()
        self.arena_buf = None
        self.slots = []
        torch.cuda.empty_cache()

    def _launch(self, slot: Slot, b: Batch, pools: HostPools):
        import torch
        k = len(b.reqs)
        off = slot.offsets_host.numpy()
        off[0] = 0
        np.cumsum([r.n for r in b.reqs], out=off[1:k + 1])
        code = F32 if b.dtype == "f32" else U32
        dev = self.arena_buf[b.dev_off:b.dev_off + b.nbytes].view(
            torch.float32 if b.dtype == "f32" else torch.int32)
        host = pools.tensors[b.dtype][b.base:b.base + b.total]
        with torch.cuda.stream(slot.stream):
            dev.copy_(host, non_blocking=True)
            slot.offsets_dev[:k + 1].copy_(slot.offsets_host[:k + 1], non_blocking=True)
            ksort_sort_batched(code, dev, slot.offsets_dev, k, b.total, slot.stream)
            host.copy_(dev, non_blocking=True)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(slot.stream)
        slot.batch, slot.event = b, ev

    def run(self, reqs: list[Request], pools: HostPools, poll_sleep_s: float = 0.0) -> RunResult:
        """Serves `reqs` (sorted by arrival) in real time; returns when all are done."""
        import torch
        reqs = sorted(reqs, key=lambda r: r.arrival_s)
        torch.cuda.synchronize()
        start_ev = torch.cuda.Event(enable_timing=True)
        start_ev.record()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        i, done_batches, in_flight, max_in_flight = 0, [], 0, 0
        events = {}
        while True:
            now = time.perf_counter() - t0
            while i < len(reqs) and reqs[i].arrival_s <= now:
                self.planner.arrive(reqs[i])
                i += 1
            for slot in self.slots:
                if slot.batch is not None and slot.event.query():
                    self.planner.complete(slot.batch)
                    done_batches.append(slot.batch)
                    slot.batch = None
                    in_flight -= 1
            for si, slot in enumerate(self.slots):
                if slot.batch is not None or not self.planner.waiting():
                    continue
                b = self.planner.next_batch()
                if b is None:  # the oldest request waits for a buffer to come back
                    break
                b.slot = si
                now = time.perf_counter() - t0
                for r in b.reqs:
                    r.admit_s = now
                self._launch(slot, b, pools)
                events[b.bid] = slot.event
                in_flight += 1
            max_in_flight = max(max_in_flight, in_flight)
            if i == len(reqs) and in_flight == 0 and not self.planner.waiting():
                break
            if poll_sleep_s:
                time.sleep(poll_sleep_s)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        for s in self.slots:
            st = ksort_get_device_error(s.stream)
            if st:
                raise RuntimeError(f"device error {st} on a serving stream")
        keys = 0
        for b in done_batches:
            t_done = start_ev.elapsed_time(events[b.bid]) / 1e3
            for r in b.reqs:
                r.done_s = t_done
                keys += r.n
        lat = np.array([r.done_s - r.arrival_s for r in reqs])
        a = self.planner.arena
        hbm = dict(self.hbm, peak_bytes_in_use=int(a.peak_in_use), refusals=self.planner.refusals,
                   blocks_outstanding=a.blocks(),
                   h2d_bytes=int(sum(b.nbytes for b in done_batches)),
                   d2h_bytes=int(sum(b.nbytes for b in done_batches)))
        return RunResult(requests=reqs, batches=done_batches, keys=keys, wall_s=wall,
                         max_in_flight=max_in_flight, latencies_s=lat, hbm=hbm)


def sort_alone(r: Request):
    """The request's keys sorted by one ksort_sort call of their own (on the device)."""
    t = request_keys(r)
    ksort_sort(F32 if r.dtype == "f32" else U32, t, r.n)
    return t


def burst_capacity(server: "Server", count: int = 500, lo: int = 1_000, hi: int = 10_000_000,
                   seed: int | None = None) -> float:
    """Keys/s the server sustains on `count` requests of the mix that all arrive at once:
    its own throughput at saturation, copies, admission and slot overlap included."""
    if seed is None:
        seed = gen.seed_for(5, 4, 0)
    reqs = poisson_requests(count, 1e12, lo, hi, seed=seed)
    with build_pools(reqs) as pools:
        res = server.run(reqs, pools)
    span = max(r.done_s for r in reqs) - min(r.arrival_s for r in reqs)
    return res.keys / span


def measure_capacity(count: int = 256, lo: int = 1_000, hi: int = 10_000_000,
                     max_keys: int = 1 << 28) -> dict:
    """Keys/s of one ksort_sort_batched over a batch drawn from the serving size mix
    (float32 keys; u32 sorts take the same kernels at the same key size): the sort alone
    with the keys resident, and the same batch with its copy in from page-locked host
    memory and back, all on one stream (no overlap between the three)."""
    import torch
    reqs = poisson_requests(count, 1.0, lo, hi, seed=gen.seed_for(5, 2, 0))
    lens = [r.n for r in reqs]
    while sum(lens) > max_keys:
        lens.pop()
    off = torch.from_numpy(gen.offsets_from_lengths(np.array(lens, np.int64))).cuda()
    total = int(off[-1])
    src = gen.uniform_torch("f32", gen.seed_for(5, 3, 0), total, device="cuda")
    host = src.cpu().pin_memory()
    keys = src.clone()
    ksort_reserve_workspace(F32, total, len(lens))
    ksort_sort_batched(F32, keys, off, len(lens), total)  # warm-up
    best = {"sort_keys_per_s": math.inf, "with_copies_keys_per_s": math.inf}
    for copies in (False, True):
        name = "with_copies_keys_per_s" if copies else "sort_keys_per_s"
        for _ in range(3):
            keys.copy_(src)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            if copies:
                keys.copy_(host, non_blocking=True)
            ksort_sort_batched(F32, keys, off, len(lens), total)
            if copies:
                host.copy_(keys, non_blocking=True)
            e1.record()
            torch.cuda.synchronize()
            best[name] = min(best[name], e0.elapsed_time(e1) / 1e3)
            if copies:
                host.copy_(src)
    if ksort_get_device_error():
        raise RuntimeError("device error in the capacity batch")
    return {k: total / v for k, v in best.items()}


__all__ = ["Request", "Planner", "Arena", "Batch", "Server", "RunResult", "HostPools",
           "poisson_requests", "build_pools", "request_keys", "sort_alone",
           "measure_capacity", "burst_capacity", "mean_length", "dtype_code"]
