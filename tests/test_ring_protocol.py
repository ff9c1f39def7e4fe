"""A model of the ring partition's barrier protocol (part_ring_kernel, one CTA), checked
under random interleavings on the CPU. The actors are the producer (slot reuse after the
slot's `empty` phase, at most DEPTH tiles loading or awaiting compaction, the end mark),
NLB role warps taking the tiles in turn (their waits on `counted`, the end seen by
polling) or, without role warps, the last data warp of each tile taking its ranges, the
data warps (waits on `full` and `ready`, write-out in tile order, the opportunistic
write-out by test), and the bulk copies, which land in any order. Every
mbarrier keeps a count of completed phases; a parity wait passes when the parity of that
count differs from the parity of the phase it waits for, as `mbarrier.try_wait.parity`
does. The checks: a wait never passes before the phase it means has completed (no
parity aliasing), every CTA finishes, and every data warp writes every tile once.

It also keeps the fault that this model found: waking the role warp of the index after
the end mark by completing that index's phase of `counted` lets a parity wait alias."""
import random

import pytest


class _Bar:
    def __init__(self, name, count):
        self.name, self.count, self.pending, self.done, self.tx = name, count, count, 0, 0

    def arrive(self, n=1):
        self.pending -= n
        assert self.pending >= 0, f"over-arrival on {self.name}"
        self._complete()

    def expect_tx(self):
        self.tx += 1
        self.arrive()

    def land(self):
        self.tx -= 1
        self._complete()

    def _complete(self):
        if self.pending == 0 and self.tx == 0:
            self.done += 1
            self.pending = self.count


class Fault(Exception):
    pass


def _run(S, DEPTH, NLB, NDW, T, seed, end_wake=False):
    rnd = random.Random(seed)
    R = S + 1
    full = [_Bar(f"full{s}", 1) for s in range(S)]
    empty = [_Bar(f"empty{s}", NDW) for s in range(S)]
    counted = [_Bar(f"counted{s}", NDW) for s in range(S)]
    ready = [_Bar(f"ready{s}", 1) for s in range(S)]
    tix = [None] * R
    acc = [0] * S
    state = {"end_at": None, "copies": [], "written": []}

    def passes(bar, k):
        if bar.done % 2 != k % 2:
            if bar.done != k + 1:
                raise Fault(f"{bar.name}: a wait for phase {k} passed with {bar.done} done")
            return True
        return False

    def wait(bar, k):
        while not passes(bar, k):
            yield

    def producer():
        for i in range(T + 1):
            s = i % S
            if i >= S:
                yield from wait(empty[s], i // S - 1)
            if i >= DEPTH:
                j = i - DEPTH
                yield from wait(counted[j % S] if NLB else ready[j % S], j // S)
            if i == T:  # no tiles left: the end mark
                tix[i % R] = -1
                state["end_at"] = i
                full[s].arrive()
                if end_wake and NLB == 2:
                    tix[(i + 1) % R] = -1
                    counted[(i + 1) % S].arrive(NDW)
                return
            tix[i % R] = i
            full[s].expect_tx()
            state["copies"].append(s)
            yield

    def role(w):
        i = w
        while True:
            yield
            if state["end_at"] is not None and i >= state["end_at"]:
                return
            while not passes(counted[i % S], i // S):
                if state["end_at"] is not None and i >= state["end_at"]:
                    return
                yield
            t = tix[i % R]
            if t != i and t != -1:
                raise Fault(f"role warp {w} read tile {t} for index {i}")
            if t == -1:
                return
            yield  # the reservation's atomic
            ready[i % S].arrive()
            i += NLB

    def data(dw):
        wnext, i = 0, 0

        def write():
            nonlocal wnext
            state["written"].append((dw, wnext))
            empty[wnext % S].arrive()
            wnext += 1

        while True:
            while wnext <= i - S:
                yield from wait(ready[wnext % S], wnext // S)
                write()
            yield from wait(full[i % S], i // S)
            t = tix[i % R]
            if t != i and t != -1:
                raise Fault(f"data warp {dw} read tile {t} for index {i}")
            if t == -1:
                counted[i % S].arrive()
                break
            yield  # compaction
            if NLB:
                counted[i % S].arrive()
            else:  # the last data warp of the tile takes its ranges
                acc[i % S] += 1
                if acc[i % S] == NDW:
                    acc[i % S] = 0
                    yield  # the reservation's atomic
                    ready[i % S].arrive()
            while wnext <= i and passes(ready[wnext % S], wnext // S):
                write()
                yield
            i += 1
        while wnext < i:
            yield from wait(ready[wnext % S], wnext // S)
            write()

    actors = [producer()] + [role(w) for w in range(NLB)] + [data(d) for d in range(NDW)]
    alive = list(range(len(actors)))
    for _ in range(100_000):
        if not alive:
            break
        if state["copies"] and rnd.random() < 0.3:
            full[state["copies"].pop(rnd.randrange(len(state["copies"])))].land()
            continue
        k = rnd.choice(alive)
        try:
            next(actors[k])
        except StopIteration:
            alive.remove(k)
    else:
        raise Fault("no progress")
    if sorted(state["written"]) != sorted((d, j) for d in range(NDW) for j in range(T)):
        raise Fault("a tile was not written by every data warp")


# the library's shapes (slots, DEPTH, role warps), and more around them
SHAPES = [(6, 3, 2), (6, 4, 2), (6, 3, 0), (8, 3, 0), (4, 3, 2), (4, 2, 2), (8, 3, 2),
          (6, 3, 1), (3, 2, 1), (2, 1, 2)]


@pytest.mark.parametrize("S,DEPTH,NLB", SHAPES)
def test_protocol_never_aliases_and_always_finishes(S, DEPTH, NLB):
    for T in (0, 1, 2, 3, 5, 6, 7, 13):
        for seed in range(25):
            _run(S, DEPTH, NLB, 3, T, seed)


def test_the_removed_end_wake_aliases():
    faults = 0
    for T in (5, 7, 11):
        for seed in range(25):
            try:
                _run(4, 3, 2, 3, T, seed, end_wake=True)
            except Fault:
                faults += 1
    assert faults > 0
