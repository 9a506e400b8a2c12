"""The seeded input recipes (paper_2607_02630_gb300/workloads.py) have the
shapes the benchmark and the parity tests rely on: the batched varlen
workload's length law, tail share, key-size mix and arena layout; the served
mix's size classes; Poisson arrivals; reproducibility from the seed.  The
paper publishes no dataset (App. A measures uniform buffers of 4 KiB to
8 MiB), so these recipes are the stand-in inputs and are pinned here."""
import math

import numpy as np

from paper_2607_02630_gb300 import workloads as W


def binomial_ok(k, n, p, sigmas=5.0):
    return abs(k - n * p) <= sigmas * math.sqrt(n * p * (1 - p))


def test_batch_varlen_recipe():
    w = W.batch_varlen(with_payload=False)
    n = w.n
    assert n == 4096
    L = w.lengths
    assert L.min() >= 1024 - 1024 % 16 and L.max() <= 8 << 20
    tails = (L % 16) != 0
    assert binomial_ok(int(tails.sum()), n, 0.25)
    assert ((L[~tails] % 16) == 0).all()
    assert binomial_ok(int((w.bits == 256).sum()), n, 0.5)
    assert set(np.unique(w.bits)) == {128, 256}
    # log-uniform on [1 KiB, 8 MiB]: log-lengths spread evenly (median near the midpoint)
    lg = np.log(L.astype(np.float64))
    mid = (math.log(1024) + math.log(8 << 20)) / 2
    assert abs(float(np.median(lg)) - mid) < 0.25
    q = np.quantile(lg, [0.25, 0.75])
    span = math.log(8 << 20) - math.log(1024)
    assert abs(q[0] - (math.log(1024) + span / 4)) < 0.3 and abs(q[1] - (math.log(1024) + 3 * span / 4)) < 0.3
    # arena: aligned, in order, no overlap, everything inside
    off = w.offsets
    assert (off % W.ARENA_ALIGN == 0).all()
    assert (off[1:] >= off[:-1] + L[:-1]).all()
    assert off[-1] + L[-1] <= w.arena_bytes
    # the size the benchmark reports for the default seed
    assert w.total_bytes == 3662162935


def test_batch_varlen_is_reproducible_and_seed_dependent():
    a = W.batch_varlen(n=64, seed=11)
    b = W.batch_varlen(n=64, seed=11)
    c = W.batch_varlen(n=64, seed=12)
    assert np.array_equal(a.lengths, b.lengths) and np.array_equal(a.payload, b.payload)
    assert np.array_equal(a.keys, b.keys) and np.array_equal(a.ivs, b.ivs)
    assert not np.array_equal(a.lengths, c.lengths)
    for i in range(a.n):
        assert a.key_of(i).size == a.bits[i] // 8


def test_served_mix_sizes():
    n = 20000
    s = W.served_sizes(n)
    one, eight = s == (1 << 20), s == (8 << 20)
    small = ~(one | eight)
    assert binomial_ok(int(one.sum()), n, 0.7) and binomial_ok(int(eight.sum()), n, 0.1)
    assert ((s[small] >= 4096 - 16) & (s[small] <= 65536) & (s[small] % 16 == 0)).all()
    # mean of the mix: 0.7 MiB + 0.8 MiB + the small class (~ 12.6 KiB mean) * 0.2
    assert abs(float(s.mean()) / 1e6 - 1.58) < 0.06


def test_poisson_arrivals():
    rate = 50_000.0
    t = W.poisson_arrivals(20000, rate, seed=5)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    assert abs(float(gaps.mean()) * rate - 1.0) < 0.03
    # exponential gaps: coefficient of variation 1
    assert abs(float(gaps.std() / gaps.mean()) - 1.0) < 0.05


def test_single_buffer_and_counter_override():
    a = W.single_buffer(1 << 12, 256, seed=7)
    assert a.payload.size == 4096 and a.key.size == 32 and a.iv.size == 16 and a.bits == 256
    b = W.single_buffer(1 << 12, 256, seed=7, low32=0xFFFFFFF8)
    assert np.array_equal(a.payload, b.payload) and np.array_equal(a.key, b.key)
    assert np.array_equal(a.iv[:12], b.iv[:12]) and bytes(b.iv[12:]) == bytes.fromhex("fffffff8")


def test_key_set():
    bits, keys = W.key_set(64)
    assert keys.shape == (64, 32) and set(np.unique(bits)) <= {128, 256}
    assert 10 < int((bits == 256).sum()) < 54
