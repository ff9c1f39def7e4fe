"""Seeded synthetic inputs for K-sort (arxiv 1107.3622), shared by the oracle tests,
the GPU parity tests and the benchmark.

This module only draws numbers: it holds none of the sorting arithmetic. The paper
fills its arrays with i.i.d. continuous U[0,1] variates (Section 2, Monte Carlo
experiment) but names no generator, so every stream here is SplitMix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):

    state_i = seed + (i + 1) * 0x9E3779B97F4A7C15          (mod 2**64)
    z = (state_i ^ (state_i >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    x_i = z ^ (z >> 31)

Value maps (all exact, no rounding):
    float32 U[0,1)  = (x >> 40) * 2**-24      (24-bit grid, never -0, never NaN)
    float64 U[0,1)  = (x >> 11) * 2**-53
    uint32 uniform  = x >> 32
    16 distinct     = x >> 60                 (values 0..15, as uint32 or float32)
    15-bit U[0,1)   = (x >> 49) * 2**-15      (32768 levels: a duplicate-heavy U[0,1])

Seeds: ``seed_for(config, size_idx, rep) = 0x11073622 ^ (config << 48) ^ (size_idx << 32) ^ rep``.

Two implementations of the same stream are given: numpy (host) and torch int64
(host or device, two's-complement wrap-around with masked logical shifts). They are
checked against each other in the CPU tests.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB
BASE_SEED = 0x11073622
MASK64 = (1 << 64) - 1

# The paper's own ten-element example (Section 1.2, "Illustration").
ILLUSTRATION = (55, 66, 60, 78, 22, 50, 75, 5, 8, 94)

# Table 1 sizes (Section 2).
TABLE1_SIZES = (100_000, 500_000, 1_000_000, 2_500_000, 5_000_000, 6_000_000,
                7_000_000, 7_100_000, 7_500_000, 10_000_000)


def seed_for(config: int, size_idx: int = 0, rep: int = 0) -> int:
    return (BASE_SEED ^ (config << 48) ^ (size_idx << 32) ^ rep) & MASK64


# ----------------------------------------------------------------------------- numpy
def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """x_start .. x_{start+n-1} of the SplitMix64 stream for ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        s = np.uint64(seed & MASK64) + i * np.uint64(GOLDEN)
        z = (s ^ (s >> np.uint64(30))) * np.uint64(MIX1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
        return z ^ (z >> np.uint64(31))


def uniform_f32(seed: int, n: int) -> np.ndarray:
    x = splitmix64(seed, n)
    return ((x >> np.uint64(40)).astype(np.float32) * np.float32(2.0 ** -24)).astype(np.float32)


def uniform_f64(seed: int, n: int) -> np.ndarray:
    x = splitmix64(seed, n)
    return (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_u32(seed: int, n: int) -> np.ndarray:
    return (splitmix64(seed, n) >> np.uint64(32)).astype(np.uint32)


def distinct16_u32(seed: int, n: int) -> np.ndarray:
    return (splitmix64(seed, n) >> np.uint64(60)).astype(np.uint32)


def distinct16_f32(seed: int, n: int) -> np.ndarray:
    return distinct16_u32(seed, n).astype(np.float32)


def quantized15(dtype: str, seed: int, n: int) -> np.ndarray:
    """U[0,1) on a grid of 2**15 levels, (x >> 49) * 2**-15: each value repeats about
    n / 32768 times (uint32: the level index itself)."""
    q = splitmix64(seed, n) >> np.uint64(49)
    if dtype == "u32":
        return q.astype(np.uint32)
    return (q.astype(np.float64) * (2.0 ** -15)).astype(NP_DTYPE[dtype])


def organ_pipe(n: int, dtype) -> np.ndarray:
    """a[i] = min(i, n-1-i): rises then falls (exact in float32 for n < 2**25)."""
    i = np.arange(n, dtype=np.int64)
    return np.minimum(i, n - 1 - i).astype(dtype)


_UNIFORM = {"f32": uniform_f32, "f64": uniform_f64, "u32": uniform_u32}
NP_DTYPE = {"f32": np.float32, "f64": np.float64, "u32": np.uint32}


def make(pattern: str, dtype: str, n: int, seed: int) -> np.ndarray:
    """One input array. ``pattern`` in {uniform, sorted, reverse, distinct16, organ_pipe,
    quantized15}.

    ``sorted``/``reverse`` are the uniform draw sorted ascending / descending, as the
    stress configuration describes (already-sorted and reverse-sorted inputs).
    """
    if pattern == "uniform":
        return _UNIFORM[dtype](seed, n)
    if pattern == "sorted":
        return np.sort(_UNIFORM[dtype](seed, n), kind="stable")
    if pattern == "reverse":
        return np.sort(_UNIFORM[dtype](seed, n), kind="stable")[::-1].copy()
    if pattern == "distinct16":
        return distinct16_u32(seed, n).astype(NP_DTYPE[dtype])
    if pattern == "organ_pipe":
        return organ_pipe(n, NP_DTYPE[dtype])
    if pattern == "quantized15":
        return quantized15(dtype, seed, n)
    raise ValueError(f"unknown pattern {pattern!r}")


def batched_lengths(num_arrays: int = 4096, lo: int = 100, hi: int = 1_000_000,
                    seed: int | None = None) -> np.ndarray:
    """Array lengths round(exp(U[ln lo, ln hi])) for the mixed-size batch (int64)."""
    if seed is None:
        seed = seed_for(3, 0, 0xA11)
    u = uniform_f64(seed, num_arrays)
    return np.rint(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)


def offsets_from_lengths(lengths: np.ndarray) -> np.ndarray:
    off = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=off[1:])
    return off


# ----------------------------------------------------------------------------- torch
def _torch_mix(s):
    import torch

    def lsr(v, k):  # logical shift right on int64 bit patterns
        return (v >> k) & ((1 << (64 - k)) - 1)

    z = (s ^ lsr(s, 30)) * torch.tensor(MIX1 - (1 << 64), dtype=torch.int64, device=s.device)
    z = (z ^ lsr(z, 27)) * torch.tensor(MIX2 - (1 << 64), dtype=torch.int64, device=s.device)
    return z ^ lsr(z, 31)


def splitmix64_torch(seed: int, n: int, device="cpu", start: int = 0):
    """Same stream as :func:`splitmix64`, as int64 bit patterns in a torch tensor."""
    import torch

    seed_s = seed - (1 << 64) if seed >= (1 << 63) else seed
    g = torch.tensor(GOLDEN - (1 << 64), dtype=torch.int64, device=device)
    i = torch.arange(start + 1, start + n + 1, dtype=torch.int64, device=device)
    return _torch_mix(seed_s + i * g)


def uniform_torch(dtype: str, seed: int, n: int, device="cpu", chunk: int = 1 << 26):
    """Uniform draw of ``dtype`` in {f32, f64, u32} built in chunks on ``device``.

    u32 values come back as torch.int32 holding the uint32 bit pattern (torch has no
    full uint32 arithmetic); reinterpret with ``.view(torch.uint32)`` if wanted.
    """
    import torch

    out_dt = {"f32": torch.float32, "f64": torch.float64, "u32": torch.int32}[dtype]
    out = torch.empty(n, dtype=out_dt, device=device)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        x = splitmix64_torch(seed, m, device=device, start=s)
        if dtype == "f32":
            out[s:s + m] = ((x >> 40) & ((1 << 24) - 1)).to(torch.float32) * (2.0 ** -24)
        elif dtype == "f64":
            out[s:s + m] = ((x >> 11) & ((1 << 53) - 1)).to(torch.float64) * (2.0 ** -53)
        else:
            hi = (x >> 32) & 0xFFFFFFFF
            out[s:s + m] = (hi - ((hi >> 31) << 32)).to(torch.int32)
    return out
