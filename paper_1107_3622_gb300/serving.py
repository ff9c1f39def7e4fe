"""Serving form of K-sort: a continuous-batching request loop over ksort_sort_batched.

Requests (a key type, a length, a seed) arrive over time. Their keys are already
resident in HBM: one flat device pool per key type holds every request's keys in
arrival order, standing in for data produced upstream on the GPU. The server sorts
each request in place, inside that pool.

The server owns a fixed HBM budget, split into `slots` stream slots. Each slot has
its own CUDA stream, a workspace reserved for `slot_keys` keys (scratch + work queue),
and an offsets buffer. When a slot is free, the planner admits waiting requests
into one batch:
  - a FIFO prefix of one key type's queue (the type whose oldest request has waited
    longest), so the batch is one contiguous range of that type's pool;
  - as many as fit the slot's reserved capacity (`slot_keys` keys, `max_arrays`
    arrays): admission is by the free HBM of the slot.
The batch runs as one ksort_sort_batched call (the persistent kernels) on the
slot's stream, followed by a completion event. Requests that arrive while batches
run are admitted as slots free up, and batches on different slots overlap on the
device. Latency is arrival -> the batch's completion event, on the device clock
aligned with the host clock at start.

Every step of the sort runs in libksort's kernels; this module schedules,
marshals offsets and reads events.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

import ksort_inputs as gen

from . import F32, U32, dtype_code, ksort_get_device_error, ksort_reserve_workspace, \
    ksort_sort, ksort_sort_batched

KEY_TYPES = ("f32", "u32")


@dataclass
class Request:
    rid: int
    arrival_s: float     # seconds after the start of the run
    dtype: str           # "f32" or "u32"
    n: int
    seed: int
    pool_off: int = 0    # first key in its type's pool
    batch: int = -1      # batch that served it
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


# ----------------------------------------------------------------------------- planner
@dataclass
class Batch:
    bid: int
    dtype: str
    reqs: list
    base: int            # first key of the batch in its type's pool
    total: int           # keys in the batch
    slot: int = -1


class Planner:
    """Admission and batching policy, independent of the GPU (tested on CPU)."""

    def __init__(self, slot_keys: int, max_arrays: int):
        if slot_keys < 1 or max_arrays < 1:
            raise ValueError("slot capacity must be positive")
        self.slot_keys = slot_keys
        self.max_arrays = max_arrays
        self.queues = {t: deque() for t in KEY_TYPES}
        self._next = 0

    def arrive(self, r: Request):
        if r.n > self.slot_keys:
            raise ValueError(f"request {r.rid} ({r.n} keys) exceeds a slot ({self.slot_keys})")
        q = self.queues[r.dtype]
        if q and r.pool_off != q[-1].pool_off + q[-1].n:
            raise ValueError("requests of one key type must be contiguous in arrival order")
        q.append(r)

    def waiting(self) -> int:
        return sum(len(q) for q in self.queues.values())

    def next_batch(self) -> Batch | None:
        """The batch a free slot should run now, or None when nothing waits."""
        heads = [(q[0].arrival_s, t) for t, q in self.queues.items() if q]
        if not heads:
            return None
        _, t = min(heads)
        q = self.queues[t]
        reqs, total = [], 0
        while q and len(reqs) < self.max_arrays and total + q[0].n <= self.slot_keys:
            r = q.popleft()
            reqs.append(r)
            total += r.n
        b = Batch(bid=self._next, dtype=t, reqs=reqs, base=reqs[0].pool_off, total=total)
        self._next += 1
        for r in reqs:
            r.batch = b.bid
        return b


# ----------------------------------------------------------------------------- pools
def build_pools(reqs: list[Request], device="cuda"):
    """One flat device pool per key type with every request's keys (arrival order)."""
    import torch
    sizes = {t: 0 for t in KEY_TYPES}
    for r in reqs:
        r.pool_off = sizes[r.dtype]
        sizes[r.dtype] += r.n
    pools = {"f32": torch.empty(max(sizes["f32"], 1), dtype=torch.float32, device=device),
             "u32": torch.empty(max(sizes["u32"], 1), dtype=torch.int32, device=device)}
    for r in reqs:
        fill_request(pools[r.dtype], r)
    torch.cuda.synchronize()
    return pools


def fill_request(pool, r: Request):
    keys = gen.uniform_torch(r.dtype, r.seed, r.n, device=pool.device)
    pool[r.pool_off:r.pool_off + r.n].copy_(keys)


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

    def summary(self) -> dict:
        lat = self.latencies_s * 1e3
        span = max(r.done_s for r in self.requests) - min(r.arrival_s for r in self.requests)
        return {
            "requests": len(self.requests), "keys": int(self.keys),
            "batches": len(self.batches), "max_batches_in_flight": self.max_in_flight,
            "keys_per_s": round(self.keys / span, 1) if span > 0 else None,
            "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "mean_ms": round(float(lat.mean()), 3),
            "span_s": round(span, 4),
        }


class Server:
    def __init__(self, slots: int = 4, slot_keys: int = 1 << 27, max_arrays: int = 4096):
        import torch
        self.planner = Planner(slot_keys, max_arrays)
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

    def _launch(self, slot: Slot, b: Batch, pools):
        import torch
        k = len(b.reqs)
        off = slot.offsets_host.numpy()
        off[0] = 0
        np.cumsum([r.n for r in b.reqs], out=off[1:k + 1])
        pool = pools[b.dtype]
        code = F32 if b.dtype == "f32" else U32
        with torch.cuda.stream(slot.stream):
            slot.offsets_dev[:k + 1].copy_(slot.offsets_host[:k + 1], non_blocking=True)
            ksort_sort_batched(code, pool[b.base:b.base + b.total], slot.offsets_dev, k, b.total,
                               slot.stream)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(slot.stream)
        slot.batch, slot.event = b, ev

    def run(self, reqs: list[Request], pools, poll_sleep_s: float = 0.0) -> RunResult:
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
                    done_batches.append(slot.batch)
                    slot.batch = None
                    in_flight -= 1
            for si, slot in enumerate(self.slots):
                if slot.batch is None and self.planner.waiting():
                    b = self.planner.next_batch()
                    b.slot = si
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
        return RunResult(requests=reqs, batches=done_batches, keys=keys, wall_s=wall,
                         max_in_flight=max_in_flight, latencies_s=lat)


def sort_alone(r: Request):
    """The request's keys sorted by one ksort_sort call of their own."""
    t = request_keys(r)
    ksort_sort(F32 if r.dtype == "f32" else U32, t, r.n)
    return t


def measure_capacity(count: int = 256, lo: int = 1_000, hi: int = 10_000_000,
                     max_keys: int = 1 << 28) -> float:
    """Keys/s of one ksort_sort_batched over a batch drawn from the serving size mix
    (float32 keys; u32 sorts take the same kernels at the same key size)."""
    import torch
    reqs = poisson_requests(count, 1.0, lo, hi, seed=gen.seed_for(5, 2, 0))
    lens = [r.n for r in reqs]
    while sum(lens) > max_keys:
        lens.pop()
    off = torch.from_numpy(gen.offsets_from_lengths(np.array(lens, np.int64))).cuda()
    total = int(off[-1])
    src = gen.uniform_torch("f32", gen.seed_for(5, 3, 0), total, device="cuda")
    keys = src.clone()
    ksort_reserve_workspace(F32, total, len(lens))
    ksort_sort_batched(F32, keys, off, len(lens), total)  # warm-up
    best = math.inf
    for _ in range(3):
        keys.copy_(src)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ksort_sort_batched(F32, keys, off, len(lens), total)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    if ksort_get_device_error():
        raise RuntimeError("device error in the capacity batch")
    return total / best


__all__ = ["Request", "Planner", "Batch", "Server", "RunResult", "poisson_requests",
           "build_pools", "request_keys", "sort_alone", "measure_capacity", "mean_length",
           "dtype_code"]
