"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the method: it only draws matrices.  The
generator is counter-based (SplitMix64, Steele, Lea and Flood, OOPSLA 2014)
so that any entry can be produced independently on any device with the same
torch code, giving bit-identical matrices on the host and on the GPU:

    z(i, l) = splitmix64(splitmix64(seed) XOR (i·k + l))
    A[i][l] = ((z >> 32) · p) >> 32                   (uniform in [0, p))

Matrices are returned as torch.int32 tensors holding the uint32 bit pattern
(every value here is < 2^31, so it reads the same either way).
"""
from __future__ import annotations

import math

import torch

_M64 = (1 << 64) - 1


def _s64(x: int) -> int:
    """A 64-bit constant as the signed int64 torch stores."""
    x &= _M64
    return x - (1 << 64) if x >= (1 << 63) else x


_GOLDEN = _s64(0x9E3779B97F4A7C15)
_MIX1 = _s64(0xBF58476D1CE4E5B9)
_MIX2 = _s64(0x94D049BB133111EB)


def _srl(z: torch.Tensor, s: int) -> torch.Tensor:
    """Logical right shift of int64 lanes."""
    return (z >> s) & ((1 << (64 - s)) - 1)


def splitmix64(z: torch.Tensor) -> torch.Tensor:
    z = z + _GOLDEN
    z = (z ^ _srl(z, 30)) * _MIX1
    z = (z ^ _srl(z, 27)) * _MIX2
    return z ^ _srl(z, 31)


def splitmix64_int(x: int) -> int:
    """Scalar SplitMix64 on Python integers (for seeds and counters)."""
    z = (int(x) + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def uniform_residues(n: int, k: int, p: int, seed: int, device="cpu",
                     row_block: int = 2048) -> torch.Tensor:
    """n×k matrix of residues uniform in [0, p) (int32 tensor, row-major)."""
    if p >= (1 << 31):
        raise ValueError("p must be below 2^31")
    base = _s64(splitmix64_int(seed))
    out = torch.empty((n, k), dtype=torch.int32, device=device)
    if n == 0 or k == 0:
        return out
    cols = torch.arange(k, dtype=torch.int64, device=device)
    for r0 in range(0, n, row_block):
        r1 = min(n, r0 + row_block)
        rows = torch.arange(r0, r1, dtype=torch.int64, device=device)
        ctr = rows[:, None] * k + cols[None, :]
        z = splitmix64(ctr ^ base)
        u = _srl(z, 32)
        out[r0:r1] = ((u * p) >> 32).to(torch.int32)
    return out


def arbitrary_u32(n: int, k: int, seed: int, device="cpu") -> torch.Tensor:
    """n×k matrix of arbitrary uint32 bit patterns (int32 tensor), for inputs ≥ p."""
    base = _s64(splitmix64_int(seed ^ 0x5EED))
    out = torch.empty((n, k), dtype=torch.int32, device=device)
    if n == 0 or k == 0:
        return out
    ctr = torch.arange(n * k, dtype=torch.int64, device=device).reshape(n, k)
    z = _srl(splitmix64(ctr ^ base), 32)
    out.copy_(torch.where(z >= (1 << 31), z - (1 << 32), z).to(torch.int32))
    return out


def batch_shapes(count: int, lo: int, hi: int, seed: int) -> list[tuple[int, int]]:
    """``count`` (n, k) pairs, each log-uniform in [lo, hi] (seeded)."""
    shapes = []
    base = splitmix64_int(seed)
    span = math.log(hi) - math.log(lo)
    for t in range(count):
        un = (splitmix64_int(base ^ (2 * t)) >> 11) / float(1 << 53)
        uk = (splitmix64_int(base ^ (2 * t + 1)) >> 11) / float(1 << 53)
        n = int(min(hi, max(lo, math.floor(math.exp(math.log(lo) + un * span)))))
        k = int(min(hi, max(lo, math.floor(math.exp(math.log(lo) + uk * span)))))
        shapes.append((n, k))
    return shapes
