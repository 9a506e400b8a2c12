"""Seeded synthetic inputs for the AES-CTR offload workloads.

This module only draws random bytes, keys, IVs and request lengths; it holds
none of the cipher's arithmetic.  Both the CUDA path's tests/benchmark and the
oracle's tests take their inputs from here, so the two sides see identical
data.  Everything is drawn from numpy's PCG64 with an explicit seed, in a
fixed order documented per generator.

The paper measures its GPU AES offload on uniform buffers from 4 KiB to
8 MiB (App. A, Table 2; Sec. 6 setup) and publishes no dataset, so these
uniform random payloads stand in for its inputs.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

#: Seed of workload k is SEED_BASE + k.
SEED_BASE = 2607026300

#: Request payloads of a batch are placed at offsets aligned to this many bytes.
ARENA_ALIGN = 256


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_bytes(g: np.random.Generator, n: int) -> np.ndarray:
    return np.frombuffer(g.bytes(n), dtype=np.uint8).copy() if n else np.zeros(0, np.uint8)


@dataclass
class SingleBuffer:
    """One payload under one key (the 1 MiB single-call case and the size sweep)."""

    payload: np.ndarray
    key: np.ndarray
    bits: int
    iv: np.ndarray


def single_buffer(nbytes: int, bits: int = 128, seed: int = SEED_BASE + 1,
                  low32: int | None = None) -> SingleBuffer:
    """Draw payload, then key, then IV from one PCG64 stream.

    ``low32`` overrides the IV's last four bytes (big-endian) -- e.g.
    0xFFFFFFF8 makes the counter carry out of its low 32-bit word after eight
    blocks.
    """
    g = rng(seed)
    payload = random_bytes(g, nbytes)
    key = random_bytes(g, bits // 8)
    iv = random_bytes(g, 16)
    if low32 is not None:
        iv[12:16] = np.frombuffer(int(low32).to_bytes(4, "big"), np.uint8)
    return SingleBuffer(payload, key, bits, iv)


@dataclass
class BatchWorkload:
    """Many requests with their own key, IV and length, packed in one arena."""

    lengths: np.ndarray          # int64 [n]
    offsets: np.ndarray          # int64 [n], ARENA_ALIGN-aligned offsets into the arena
    bits: np.ndarray             # int32 [n], 128 or 256
    keys: np.ndarray             # uint8 [n, 32]; the first bits/8 bytes are the key
    ivs: np.ndarray              # uint8 [n, 16]
    arena_bytes: int
    seed: int
    payload: np.ndarray | None = field(default=None, repr=False)  # uint8 [arena_bytes]

    @property
    def n(self) -> int:
        return int(self.lengths.size)

    @property
    def total_bytes(self) -> int:
        return int(self.lengths.sum())

    def key_of(self, i: int) -> np.ndarray:
        return self.keys[i, : int(self.bits[i]) // 8]


def batch_varlen(n: int = 4096, min_len: int = 1024, max_len: int = 8 << 20,
                 tail_frac: float = 0.25, frac_256: float = 0.5,
                 seed: int = SEED_BASE + 3, with_payload: bool = True) -> BatchWorkload:
    """The batched varlen workload: lengths log-uniform on [min_len, max_len].

    Draw order from one PCG64 stream: log-lengths (n), tail coin flips (n),
    tail sizes (n), key-size coin flips (n), keys (n*32 bytes), IVs (n*16
    bytes), then the arena payload.  A request with a tail gets
    len - len % 16 + r with r uniform on 1..15 (clamped to max_len); the others
    are rounded down to a multiple of 16 (never below min_len).
    """
    g = rng(seed)
    loglen = g.uniform(np.log(min_len), np.log(max_len), size=n)
    lengths = np.floor(np.exp(loglen)).astype(np.int64)
    has_tail = g.random(n) < tail_frac
    tail = g.integers(1, 16, size=n)
    is256 = g.random(n) < frac_256
    keys = random_bytes(g, n * 32).reshape(n, 32)
    ivs = random_bytes(g, n * 16).reshape(n, 16)
    base = lengths - lengths % 16
    base = np.maximum(base, min_len - min_len % 16)
    lengths = np.where(has_tail, np.minimum(base + tail, max_len), base)
    bits = np.where(is256, 256, 128).astype(np.int32)
    padded = (lengths + ARENA_ALIGN - 1) // ARENA_ALIGN * ARENA_ALIGN
    offsets = np.concatenate([[0], np.cumsum(padded)[:-1]]).astype(np.int64)
    arena = int(padded.sum())
    payload = random_bytes(g, arena) if with_payload else None
    return BatchWorkload(lengths, offsets, bits, keys, ivs, arena, seed, payload)


def served_sizes(n: int, seed: int = SEED_BASE + 4) -> np.ndarray:
    """Request sizes of the open-loop served mix: 70% 1 MiB, 10% 8 MiB,
    20% log-uniform on [4 KiB, 64 KiB] (rounded down to 16 bytes)."""
    g = rng(seed)
    u = g.random(n)
    small = np.floor(np.exp(g.uniform(np.log(4096), np.log(65536), size=n))).astype(np.int64)
    small -= small % 16
    return np.where(u < 0.7, 1 << 20, np.where(u < 0.8, 8 << 20, small)).astype(np.int64)


def poisson_arrivals(n: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson process of the given rate."""
    g = rng(seed)
    return np.cumsum(g.exponential(1.0 / rate_per_s, size=n))


def key_set(n_keys: int, frac_256: float = 0.5, seed: int = SEED_BASE + 5):
    """n_keys random keys; returns (bits int32[n], keys uint8[n, 32])."""
    g = rng(seed)
    is256 = g.random(n_keys) < frac_256
    keys = random_bytes(g, n_keys * 32).reshape(n_keys, 32)
    return np.where(is256, 256, 128).astype(np.int32), keys
