"""Single-buffer AES-CTR on the GPU, bit-exact against the CPU oracle.

AES-CTR is deterministic: exactly one output is correct, so every comparison
here is byte-for-byte (tolerance 0).  Inputs come from the seeded generators
in paper_2607_02630_gb300.workloads; expected values only from oracle/.
"""
import re
import zlib

import numpy as np
import pytest

import oracle
from paper_2607_02630_gb300 import workloads as W

from gpu_util import iv_plus, iv_with_low, to_dev, to_host

pytestmark = pytest.mark.gpu

SHAPES = [
    dict(variant=1, threads=256, blocks_per_thread=1),
    dict(variant=1, threads=512, blocks_per_thread=1),
    dict(variant=1, threads=1024, blocks_per_thread=1),
    dict(variant=1, threads=512, blocks_per_thread=2),
    dict(variant=1, threads=1024, blocks_per_thread=2),
    dict(variant=1, threads=1024, blocks_per_thread=4),
    dict(variant=1, threads=256, blocks_per_thread=4, ctas=3),
    dict(variant=2, threads=128),
    dict(variant=2, threads=128, ctas=2),
    dict(),  # tuned
]


def gpu_ctr(torch, aes, ctx, iv, data, pad=64, **shape):
    src = to_dev(torch, data)
    dst = to_dev(torch, np.zeros(0, np.uint8), pad=data.size + pad)
    aes.ctr(ctx, iv.tobytes(), src, dst, data.size, **shape)
    torch.cuda.synchronize()
    out = to_host(dst)
    assert (out[data.size:] == 0xA5).all(), "bytes past len were written"
    return out[: data.size]


@pytest.mark.parametrize("bits", [128, 192, 256])
def test_key_expansion_matches_oracle(aes, bits):
    g = W.rng(10 + bits)
    for _ in range(8):
        key = W.random_bytes(g, bits // 8)
        ctx = aes.Context(key.tobytes(), bits)
        assert ctx.round_keys() == oracle.key_expansion(key, bits).tobytes()
        ctx.close()


def test_one_mib_aes128_config(cuda, aes, ncpu):
    """One 1 MiB buffer, AES-128 key and IV drawn from the same seed."""
    w = W.single_buffer(1 << 20, 128, seed=W.SEED_BASE + 1)
    ctx = aes.Context(w.key.tobytes(), 128)
    got = gpu_ctr(cuda, aes, ctx, w.iv, w.payload)
    np.testing.assert_array_equal(got, oracle.ctr_mt(w.key, 128, w.iv, w.payload, ncpu))


@pytest.mark.parametrize("bits", [128, 256])
def test_every_length_0_to_64(cuda, aes, bits):
    g = W.rng(20 + bits)
    key = W.random_bytes(g, bits // 8)
    ctx = aes.Context(key.tobytes(), bits)
    for n in range(65):
        iv = W.random_bytes(g, 16)
        data = W.random_bytes(g, n)
        got = gpu_ctr(cuda, aes, ctx, iv, data)
        np.testing.assert_array_equal(got, oracle.ctr(key, bits, iv, data), err_msg=f"len={n}")


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "-".join(f"{k}{v}" for k, v in s.items()) or "auto")
@pytest.mark.parametrize("kind", ["random", "low32", "low64", "wrap128"])
def test_shapes_tails_and_carries(cuda, aes, ncpu, shape, kind):
    g = W.rng(zlib.crc32(repr((kind, sorted(shape.items()))).encode()))
    for bits in (128, 192, 256):
        key = W.random_bytes(g, bits // 8)
        ctx = aes.Context(key.tobytes(), bits)
        for n in (1, 15, 16, 17, 4096 + 5, 3 * 65536 + 13, (1 << 20) + 7):
            iv = iv_with_low(g, kind)
            data = W.random_bytes(g, n)
            got = gpu_ctr(cuda, aes, ctx, iv, data, **shape)
            np.testing.assert_array_equal(got, oracle.ctr_mt(key, bits, iv, data, ncpu),
                                          err_msg=f"bits={bits} n={n}")


@pytest.mark.parametrize("bits", [128, 256])
def test_size_sweep_with_low_word_carry(cuda, aes, ncpu, bits):
    """Sizes 4 KiB .. 64 MiB in powers of 4, counter low word starting at
    2^32 - 8 so the carry into byte 11 happens at block 8; tuned shape and
    both kernel variants."""
    for e in range(12, 27, 2):
        n = 1 << e
        w = W.single_buffer(n, bits, seed=W.SEED_BASE + 2 + e, low32=0xFFFFFFF8)
        ctx = aes.Context(w.key.tobytes(), bits)
        want = oracle.ctr_mt(w.key, bits, w.iv, w.payload, ncpu)
        for shape in ({}, dict(variant=1, threads=1024, blocks_per_thread=2), dict(variant=2, threads=128)):
            got = gpu_ctr(cuda, aes, ctx, w.iv, w.payload, **shape)
            np.testing.assert_array_equal(got, want, err_msg=f"n={n} shape={shape}")


@pytest.mark.parametrize("variant", [1, 2])
def test_256mib_sampled_windows(cuda, aes, variant):
    """The largest sweep size: 4 KiB windows spread over the buffer, each
    checked against the oracle started at T_1 + offset/16."""
    n = 256 << 20
    w = W.single_buffer(n, 256, seed=W.SEED_BASE + 2, low32=0xFFFFFFF8)
    ctx = aes.Context(w.key.tobytes(), 256)
    src = to_dev(cuda, w.payload)
    dst = cuda.empty(n, dtype=cuda.uint8, device="cuda")
    aes.ctr(ctx, w.iv.tobytes(), src, dst, n, variant=variant, threads=1024 if variant == 1 else 128,
            blocks_per_thread=2 if variant == 1 else 0)
    cuda.cuda.synchronize()
    g = W.rng(99)
    offs = sorted({0, n - 4096} | {int(x) * 16 for x in g.integers(0, (n - 4096) // 16, 30)})
    for off in offs:
        got = to_host(dst[off: off + 4096])
        want = oracle.ctr(w.key, 256, iv_plus(w.iv, off // 16), w.payload[off: off + 4096])
        np.testing.assert_array_equal(got, want, err_msg=f"offset {off}")


def test_in_place(cuda, aes, ncpu):
    g = W.rng(31)
    key = W.random_bytes(g, 32)
    ctx = aes.Context(key.tobytes(), 256)
    for shape in SHAPES:
        data = W.random_bytes(g, 300_001)
        iv = W.random_bytes(g, 16)
        buf = to_dev(cuda, data)
        aes.ctr(ctx, iv.tobytes(), buf, buf, data.size, **shape)
        cuda.cuda.synchronize()
        np.testing.assert_array_equal(to_host(buf), oracle.ctr_mt(key, 256, iv, data, ncpu))


def test_decrypt_is_encrypt_and_blocks_are_independent(cuda, aes):
    g = W.rng(32)
    key = W.random_bytes(g, 16)
    ctx = aes.Context(key.tobytes(), 128)
    iv = iv_with_low(g, "low32")
    data = W.random_bytes(g, 1 << 18)
    c = gpu_ctr(cuda, aes, ctx, iv, data)
    np.testing.assert_array_equal(gpu_ctr(cuda, aes, ctx, iv, c), data)
    for a, b in [(0, 1), (7, 9), (8, 4096), (100, 16384)]:
        part = gpu_ctr(cuda, aes, ctx, iv_plus(iv, a), data[16 * a: 16 * b])
        np.testing.assert_array_equal(part, c[16 * a: 16 * b])


def test_pinned_host_buffers(cuda, aes, ncpu):
    """in/out in pinned host memory: the kernel reads and writes them through
    their device aliases (zero-copy)."""
    g = W.rng(33)
    key = W.random_bytes(g, 16)
    ctx = aes.Context(key.tobytes(), 128)
    data = W.random_bytes(g, (1 << 20) + 9)
    iv = W.random_bytes(g, 16)
    src = cuda.from_numpy(data).pin_memory()
    dst = cuda.zeros(data.size, dtype=cuda.uint8).pin_memory()
    aes.ctr(ctx, iv.tobytes(), src, dst, data.size)
    cuda.cuda.synchronize()
    np.testing.assert_array_equal(dst.numpy(), oracle.ctr_mt(key, 128, iv, data, ncpu))


def test_argument_errors(cuda, aes):
    ctx = aes.Context(bytes(16), 128)
    buf = cuda.zeros(4096, dtype=cuda.uint8, device="cuda")
    iv = bytes(16)
    p = buf.data_ptr()
    assert aes.ctr_status(ctx, iv, p + 1, p + 2048, 64) == aes.AES_EALIGN
    assert aes.ctr_status(ctx, iv, p, p + 8, 64) == aes.AES_EALIGN
    assert aes.ctr_status(ctx, iv, p, p + 16, 64) == aes.AES_EOVERLAP
    assert aes.ctr_status(ctx, iv, p + 16, p, 64) == aes.AES_EOVERLAP
    assert aes.ctr_status(ctx, iv, p, p + 64, 64) == aes.AES_OK
    assert aes.ctr_status(ctx, iv, 0, p, 64) == aes.AES_EINVAL
    assert aes.ctr_status(ctx, iv, 0, 0, 0) == aes.AES_OK  # len 0: no-op
    pageable = np.zeros(4096, np.uint8)
    assert aes.ctr_status(ctx, iv, pageable.ctypes.data, p, 64) == aes.AES_EPTR
    assert aes.ctr_status(ctx, iv, p, p + 1024, 64, variant=1, threads=100) == aes.AES_EINVAL
    assert aes.ctr_status(ctx, iv, p, p + 1024, 64, variant=1, threads=256, blocks_per_thread=3) == aes.AES_EINVAL
    assert aes.ctr_status(ctx, iv, p, p + 1024, 64, variant=2, threads=256) == aes.AES_EINVAL
    assert aes.ctr_status(ctx, iv, p, p + 1024, 64, variant=7) == aes.AES_EINVAL
    cuda.cuda.synchronize()


def test_autotune_then_auto_shapes_stay_exact(cuda, aes, ncpu, tmp_path):
    path = str(tmp_path / "tune.json")
    aes.autotune(path)
    aes.autotune_load(path)
    for n in (4096, 1 << 20, 8 << 20):
        for bits in (128, 256):
            s = aes.tuned_shape(n, bits)
            assert s["variant"] in (1, 2) and s["ctas"] >= 1
    g = W.rng(34)
    for n in (5000, (1 << 20) + 3, (8 << 20) + 1):
        key = W.random_bytes(g, 32)
        ctx = aes.Context(key.tobytes(), 256)
        iv = W.random_bytes(g, 16)
        data = W.random_bytes(g, n)
        np.testing.assert_array_equal(gpu_ctr(cuda, aes, ctx, iv, data),
                                      oracle.ctr_mt(key, 256, iv, data, ncpu))
    # the batch shape was tuned too, and the tuned default stays exact
    text = open(path).read()
    m = re.search(r'"batch": \[(\d+), (\d+), (\d+), (\d+)\]', text)
    assert m and (int(m.group(1)), int(m.group(2))) in [(1, 256), (1, 512), (1, 1024), (2, 128)], text
    assert int(m.group(3)) in (1024, 2048, 4096) and int(m.group(4)) in (1, 2, 4)
    lengths = [1, 4096 + 7, 1 << 20, (3 << 20) + 5]
    total = sum((n + 255) // 256 * 256 for n in lengths)
    payload = W.random_bytes(g, total)
    src, dst = to_dev(cuda, payload), to_dev(cuda, np.zeros(0, np.uint8), pad=total)
    reqs, meta, o = [], [], 0
    for i, n in enumerate(lengths):
        bits = (128, 256)[i % 2]
        key = W.random_bytes(g, bits // 8)
        iv = W.random_bytes(g, 16)
        reqs.append((aes.Context(key.tobytes(), bits), iv.tobytes(), src.data_ptr() + o, dst.data_ptr() + o, n))
        meta.append((key, bits, iv, o, n))
        o += (n + 255) // 256 * 256
    aes.batch(reqs)
    out = to_host(dst)
    for key, bits, iv, o, n in meta:
        np.testing.assert_array_equal(out[o: o + n], oracle.ctr_mt(key, bits, iv, payload[o: o + n], ncpu))


def test_ctr_sync_blocks_until_done(cuda, aes, ncpu):
    """aes_ctr_sync returns only once the output is complete: read it without
    any device synchronisation."""
    g = W.rng(34)
    key = W.random_bytes(g, 32)
    ctx = aes.Context(key.tobytes(), 256)
    data = W.random_bytes(g, (1 << 20) + 5)
    iv = W.random_bytes(g, 16)
    src = cuda.from_numpy(data).pin_memory()
    dst = cuda.zeros(data.size, dtype=cuda.uint8).pin_memory()
    s = cuda.cuda.Stream()
    for _ in range(3):
        dst.zero_()
        aes.ctr_sync(ctx, iv.tobytes(), src, dst, data.size, stream=s)
        np.testing.assert_array_equal(dst.numpy(), oracle.ctr_mt(key, 256, iv, data, ncpu))
    assert aes.lib().aes_ctr_sync(None, iv.tobytes(), src.data_ptr(), dst.data_ptr(), 16, 0) == aes.AES_EINVAL
