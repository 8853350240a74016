"""Order-independent digest of a pair set, accumulated with torch.

Used by the full-size tests to reduce up to 1e10 result pairs to what the
oracle's digest stores: the member count, the per-point degree array (how
many pairs (i, j) each i has) and the pair hash sum of mix64(i << 32 | j)
mod 2^64, where mix64 is the splitmix64 finaliser.  The arithmetic is plain
torch int64 (wrapping multiplication, masked shifts for the logical right
shift); it runs on whatever device the pairs are on.  A CPU test pins it to
the oracle's own hash.
"""
from __future__ import annotations

import hashlib

import numpy as np

_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def _s64(x: int) -> int:
    """A 64-bit pattern as a signed int64 value."""
    return x - (1 << 64) if x >= (1 << 63) else x


def _shr(z, s: int):
    """Logical right shift of int64 values."""
    return (z >> s) & ((1 << (64 - s)) - 1)


def mix64(z):
    z = (z ^ _shr(z, 30)) * _s64(_M1)
    z = (z ^ _shr(z, 27)) * _s64(_M2)
    return z ^ _shr(z, 31)


class Digest:
    """Running (count, degree, hash) of the pairs passed to add()."""

    def __init__(self, n: int, device):
        import torch
        self.torch = torch
        self.n = n
        self.count = 0
        self.hash = 0
        self.degree = torch.zeros(n, dtype=torch.int64, device=device)

    def add(self, pairs, block: int = 1 << 27) -> None:
        """pairs: (k, 2) int32 / uint32-as-int32 tensor of (i, j)."""
        torch = self.torch
        for k0 in range(0, pairs.shape[0], block):
            p = pairs[k0:k0 + block]
            i = p[:, 0].to(torch.int64) & 0xFFFFFFFF
            j = p[:, 1].to(torch.int64) & 0xFFFFFFFF
            z = mix64((i << 32) | j)
            lo = int((z & 0xFFFFFFFF).sum().item())
            hi = int(_shr(z, 32).sum().item())
            self.hash = (self.hash + lo + (hi << 32)) % (1 << 64)
            self.count += int(p.shape[0])
            self.degree += torch.bincount(i, minlength=self.n)

    def degree_sha256(self) -> str:
        d = self.degree.cpu().numpy()
        assert d.max() < (1 << 32)
        return hashlib.sha256(d.astype("<u4").tobytes()).hexdigest()


def sha256(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()
