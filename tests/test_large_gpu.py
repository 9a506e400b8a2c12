"""Buffers past 4 GiB on every path: byte offsets beyond 2^32 and block
indices beyond 2^28, checked against the oracle on sampled windows (the
oracle starts a window at T_1 + offset/16)."""
import numpy as np
import pytest

import oracle
from paper_2607_02630_gb300 import workloads as W

from gpu_util import iv_with_low

pytestmark = pytest.mark.gpu

N = (4 << 30) + (64 << 10) + 7  # past 4 GiB, ending in a 7-byte tail


def windows(n):
    return [(0, 4096), ((1 << 32) - 2048, (1 << 32) + 2048), (n - 4096 - 7, n)]


def iv_at(iv, byte_offset):
    v = (int.from_bytes(bytes(iv), "big") + byte_offset // 16) % (1 << 128)
    return np.frombuffer(v.to_bytes(16, "big"), np.uint8)


@pytest.fixture(scope="module")
def big(cuda):
    gen = cuda.Generator(device="cuda").manual_seed(W.SEED_BASE + 13)
    src = cuda.randint(0, 256, (N + 9,), dtype=cuda.uint8, device="cuda", generator=gen)
    dst = cuda.empty(N + 16 + 9, dtype=cuda.uint8, device="cuda")
    yield src, dst
    del src, dst
    cuda.cuda.empty_cache()


def check(cuda, src, dst, key, bits, iv, ncpu):
    cuda.cuda.synchronize()
    for a, b in windows(N):
        assert a % 16 == 0
        got = dst[a:b].cpu().numpy()
        want = oracle.ctr_mt(key, bits, iv_at(iv, a), src[a:b].cpu().numpy(), ncpu)
        np.testing.assert_array_equal(got, want, err_msg=f"window [{a}, {b})")
    assert (dst[N:N + 16].cpu().numpy() == 0xA5).all(), "bytes past len were written"


def test_single_buffer_past_4gib(cuda, aes, ncpu, big):
    src, dst = big
    g = W.rng(70)
    key = W.random_bytes(g, 32)
    iv = iv_with_low(g, "low64")
    ctx = aes.Context(key.tobytes(), 256)
    dst.fill_(0xA5)
    aes.ctr(ctx, iv.tobytes(), src, dst, N)
    check(cuda, src, dst, key, 256, iv, ncpu)


def test_batch_request_past_4gib(cuda, aes, ncpu, big):
    src, dst = big
    g = W.rng(71)
    key = W.random_bytes(g, 16)
    iv = W.random_bytes(g, 16)
    ctx = aes.Context(key.tobytes(), 128)
    dst.fill_(0xA5)
    aes.batch([(ctx, iv.tobytes(), src.data_ptr(), dst.data_ptr(), N)])
    check(cuda, src, dst, key, 128, iv, ncpu)


def test_served_request_past_4gib(cuda, aes, ncpu, big):
    src, dst = big
    g = W.rng(72)
    key = W.random_bytes(g, 16)
    iv = W.random_bytes(g, 16)
    srv = aes.Server(slots=4, max_keys=1, idle_timeout_us=2_000_000)
    try:
        ks = srv.key_register(key.tobytes(), 128)
        dst.fill_(0xA5)
        cuda.cuda.synchronize()  # the fill runs on torch's stream, the served kernel on its own
        t = srv.submit(ks, iv.tobytes(), src.data_ptr(), dst.data_ptr(), N)
        assert srv.wait(t, 30_000_000) == aes.AES_OK
        check(cuda, src, dst, key, 128, iv, ncpu)
    finally:
        assert srv.close() == aes.AES_OK
