"""Batched varlen AES-CTR (one persistent launch, work-stealing tiles) and its
CUDA-graph plans, bit-exact against the CPU oracle request by request."""
import numpy as np
import pytest

import oracle
from paper_2607_02630_gb300 import workloads as W

from gpu_util import iv_plus, iv_with_low, set_batch_shape, to_dev, to_host

pytestmark = pytest.mark.gpu


def make_requests(torch, aes, g, lengths, bits_list, kinds=None):
    """Requests packed into one device arena at 256-byte aligned offsets."""
    pad = [(n + 255) // 256 * 256 + 256 for n in lengths]
    offs = np.concatenate([[0], np.cumsum(pad)[:-1]]).astype(np.int64)
    total = int(sum(pad))
    payload = W.random_bytes(g, total)
    src = to_dev(torch, payload)
    dst = to_dev(torch, np.zeros(0, np.uint8), pad=total)
    reqs, meta = [], []
    for i, (n, bits) in enumerate(zip(lengths, bits_list)):
        key = W.random_bytes(g, bits // 8)
        iv = iv_with_low(g, kinds[i] if kinds else "random")
        ctx = aes.Context(key.tobytes(), bits)
        o = int(offs[i])
        reqs.append((ctx, iv.tobytes(), src.data_ptr() + o, dst.data_ptr() + o, int(n)))
        meta.append((key, bits, iv, o, int(n)))
    return reqs, meta, payload, src, dst


def check_all(torch, meta, payload, dst, ncpu):
    torch.cuda.synchronize()
    out = to_host(dst)
    for key, bits, iv, o, n in meta:
        want = oracle.ctr_mt(key, bits, iv, payload[o: o + n], ncpu)
        np.testing.assert_array_equal(out[o: o + n], want, err_msg=f"request at {o} len {n}")
        assert (out[o + n: o + n + 16] == 0xA5).all(), "bytes past len were written"


def mixed_lengths(g, k):
    fixed = [0, 1, 15, 16, 17, 31, 33, 4095, 4096, 4097]
    rand = [int(x) for x in np.exp(g.uniform(np.log(1024), np.log(3 << 20), k - len(fixed)))]
    return fixed + rand


# Every shape the batch autotuner can pick (variant, CTA size, blocks per lane
# in flight, tile size), plus odd CTA sizes and the defaults.
SHAPES = [(1, th, tb, nb) for tb in (1024, 2048, 4096) for th in (256, 512, 1024) for nb in (1, 2, 4)] + \
    [(2, 128, tb, 0) for tb in (1024, 2048, 4096)] + \
    [(1, 1024, 8192, 2), (1, 256, 512, 1), (1, 544, 1024, 2), (2, 128, 256, 0), (0, 0, 2048, 0), (0, 0, 0, 0)]


@pytest.mark.parametrize("variant,threads,tile_blocks,nb", SHAPES,
                         ids=[f"v{v}_t{th}_tile{tb}_nb{nb}" for v, th, tb, nb in SHAPES])
def test_mixed_batch_matches_oracle(cuda, aes, ncpu, variant, threads, tile_blocks, nb):
    g = W.rng(40 + tile_blocks + threads + nb)
    lengths = mixed_lengths(g, 48)
    bits = [(128, 192, 256)[i % 3] for i in range(len(lengths))]
    kinds = [("random", "low32", "low64", "wrap128")[i % 4] for i in range(len(lengths))]
    reqs, meta, payload, src, dst = make_requests(cuda, aes, g, lengths, bits, kinds)
    aes.batch(reqs, variant=variant, tile_blocks=tile_blocks, threads=threads, blocks_per_thread=nb)
    check_all(cuda, meta, payload, dst, ncpu)


def test_batch_autotune_picks_a_shape_that_stays_exact(cuda, aes, ncpu, tmp_path):
    """aes_batch_autotune times every candidate shape on the caller's own
    requests (overwriting their outputs with the correct ciphertext), makes
    the fastest the device's batch shape, and batches that then use it (plans
    and one-shot calls) still give the oracle's bytes."""
    g = W.rng(47)
    lengths = mixed_lengths(g, 40)
    bits = [(128, 256)[i % 2] for i in range(len(lengths))]
    reqs, meta, payload, src, dst = make_requests(cuda, aes, g, lengths, bits)
    d = aes.batch_tuned_shape()
    default = (d["variant"], d["threads"], d["tile_blocks"], d["blocks_per_thread"])
    try:
        best = aes.batch_autotune(reqs)
        assert best == aes.batch_tuned_shape()
        assert best["variant"] in (1, 2) and best["tile_blocks"] in (1024, 2048, 4096)
        check_all(cuda, meta, payload, dst, ncpu)  # the candidates' own launches
        dst.fill_(0xA5)
        plan = aes.BatchPlan(reqs)
        plan.launch()
        check_all(cuda, meta, payload, dst, ncpu)
        plan.close()
        dst.fill_(0xA5)
        aes.batch(reqs)
        check_all(cuda, meta, payload, dst, ncpu)
    finally:
        set_batch_shape(cuda, aes, tmp_path / "shape.json", default)  # for the tests that follow


@pytest.mark.parametrize("seed", [1, 7, 12345])
def test_scrambled_tile_order_gives_same_result(cuda, aes, ncpu, seed):
    g = W.rng(50)
    lengths = mixed_lengths(g, 40)
    bits = [128 if i % 2 else 256 for i in range(len(lengths))]
    reqs, meta, payload, src, dst = make_requests(cuda, aes, g, lengths, bits)
    aes.batch(reqs, tile_blocks=1024, tile_order_seed=seed)
    check_all(cuda, meta, payload, dst, ncpu)


def test_batch_equals_per_request_calls(cuda, aes):
    g = W.rng(51)
    lengths = mixed_lengths(g, 32)
    bits = [128 if i % 2 else 256 for i in range(len(lengths))]
    reqs, meta, payload, src, dst = make_requests(cuda, aes, g, lengths, bits)
    aes.batch(reqs)
    cuda.cuda.synchronize()
    batched = to_host(dst).copy()
    dst.fill_(0xA5)
    for r in reqs:
        aes.ctr(*r)
    cuda.cuda.synchronize()
    np.testing.assert_array_equal(to_host(dst), batched)


def test_plan_graph_replays(cuda, aes, ncpu):
    g = W.rng(52)
    lengths = mixed_lengths(g, 24)
    bits = [(128, 256)[i % 2] for i in range(len(lengths))]
    reqs, meta, payload, src, dst = make_requests(cuda, aes, g, lengths, bits)
    plan = aes.BatchPlan(reqs)
    assert plan.nbytes == sum(lengths)
    plan.launch()
    check_all(cuda, meta, payload, dst, ncpu)
    # same layout, new payload bytes: the replay encrypts the new contents
    payload2 = W.random_bytes(g, payload.size)
    src.copy_(cuda.from_numpy(payload2))
    dst.fill_(0xA5)
    plan.launch()
    plan.launch()  # idempotent: out depends only on in
    check_all(cuda, meta, payload2, dst, ncpu)
    plan.close()


def test_batch_argument_errors(cuda, aes):
    ctx = aes.Context(bytes(16), 128)
    buf = cuda.zeros(1 << 16, dtype=cuda.uint8, device="cuda")
    p = buf.data_ptr()
    ok = (ctx, bytes(16), p, p + 4096, 1024)
    assert aes.batch_status([ok]) == aes.AES_OK
    assert aes.batch_status([ok, (ctx, bytes(16), p + 8, p + 8192, 64)]) == aes.AES_EALIGN
    assert aes.batch_status([ok, (ctx, bytes(16), p, p + 16, 64)]) == aes.AES_EOVERLAP
    assert aes.batch_status([ok], tile_blocks=100) == aes.AES_EINVAL
    assert aes.batch_status([ok], threads=1000) == aes.AES_EINVAL
    assert aes.batch_status([(ctx, bytes(16), 0, 0, 0)]) == aes.AES_OK  # all empty
    cuda.cuda.synchronize()


def test_full_size_batch_workload_matches_oracle(cuda, aes, ncpu):
    """The 4096-request workload at full size (~3.7 GB), launched as the
    benchmark launches it (a graph plan with the device's batch shape), and
    every byte of every request compared with the oracle (about 80 s of
    oracle time on 16 host cores), as is every byte past each request up to
    the next 256-byte boundary (untouched)."""
    import concurrent.futures as cf

    w = W.batch_varlen(seed=W.SEED_BASE + 3)
    src = to_dev(cuda, w.payload)
    dst = cuda.full((w.arena_bytes,), 0xA5, dtype=cuda.uint8, device="cuda")
    ctxs = [aes.Context(w.key_of(i).tobytes(), int(w.bits[i])) for i in range(w.n)]
    reqs = [(ctxs[i], w.ivs[i].tobytes(), src.data_ptr() + int(w.offsets[i]),
             dst.data_ptr() + int(w.offsets[i]), int(w.lengths[i])) for i in range(w.n)]
    plan = aes.BatchPlan(reqs)
    assert plan.nbytes == w.total_bytes
    plan.launch()
    cuda.cuda.synchronize()
    plan.close()
    out = to_host(dst)
    del src, dst

    def check(i):
        o, n = int(w.offsets[i]), int(w.lengths[i])
        want = oracle.ctr_mt(w.key_of(i), int(w.bits[i]), w.ivs[i], w.payload[o: o + n],
                             ncpu if n >= (8 << 20) // 4 else 1)
        if not np.array_equal(out[o: o + n], want):
            bad = int(np.flatnonzero(out[o: o + n] != want)[0])
            return f"request {i} (len {n}) differs from byte {bad}"
        pad_end = (o + n + 255) // 256 * 256
        if not (out[o + n: pad_end] == 0xA5).all():
            return f"request {i}: bytes past len were written"
        return None

    # large requests use every core each; the many small ones run side by side
    order = sorted(range(w.n), key=lambda i: -int(w.lengths[i]))
    big = [i for i in order if w.lengths[i] >= (8 << 20) // 4]
    small = [i for i in order if w.lengths[i] < (8 << 20) // 4]
    errors = [e for e in map(check, big) if e]
    with cf.ThreadPoolExecutor(ncpu) as ex:
        errors += [e for e in ex.map(check, small) if e]
    assert not errors, errors[:5]
    cuda.cuda.empty_cache()


def test_batch_pinned_host_buffers(cuda, aes, ncpu):
    """Batch requests whose payloads live in pinned host memory (the kernel
    reads and writes them over NVLink-C2C through their device aliases), mixed
    with device-resident ones in the same launch."""
    g = W.rng(48)
    lengths = [1, 17, 4096 + 5, 1 << 20, (1 << 20) + 9, 3 << 16]
    pad = [(n + 255) // 256 * 256 + 256 for n in lengths]
    offs = np.concatenate([[0], np.cumsum(pad)[:-1]]).astype(np.int64)
    total = int(sum(pad))
    payload = W.random_bytes(g, total)
    hsrc = cuda.from_numpy(payload.copy()).pin_memory()
    hdst = cuda.full((total,), 0xA5, dtype=cuda.uint8).pin_memory()
    dsrc = to_dev(cuda, payload)
    ddst = to_dev(cuda, np.zeros(0, np.uint8), pad=total)
    reqs, meta = [], []
    for i, n in enumerate(lengths):
        bits = (128, 256)[i % 2]
        key = W.random_bytes(g, bits // 8)
        iv = iv_with_low(g, ("random", "low32")[i % 2])
        ctx = aes.Context(key.tobytes(), bits)
        o = int(offs[i])
        src, dst = (hsrc, hdst) if i % 3 != 2 else (dsrc, ddst)
        reqs.append((ctx, iv.tobytes(), src.data_ptr() + o, dst.data_ptr() + o, n))
        meta.append((key, bits, iv, o, n, i % 3 != 2))
    aes.batch(reqs)
    cuda.cuda.synchronize()
    hout, dout = hdst.numpy(), to_host(ddst)
    for key, bits, iv, o, n, on_host in meta:
        out = hout if on_host else dout
        want = oracle.ctr_mt(key, bits, iv, payload[o: o + n], ncpu)
        np.testing.assert_array_equal(out[o: o + n], want, err_msg=f"request at {o} len {n}")
        assert (out[o + n: o + n + 16] == 0xA5).all(), "bytes past len were written"


def test_in_place_batch_matches_oracle(cuda, aes, ncpu):
    """Every other request of the batch encrypts in place (in == out); the
    rest write to a second buffer.  All match the oracle."""
    g = W.rng(52)
    lengths = mixed_lengths(g, 24)
    bits = [(128, 256)[i % 2] for i in range(len(lengths))]
    reqs, meta, payload, src, dst = make_requests(cuda, aes, g, lengths, bits)
    reqs = [(c, iv, i_, i_ if k % 2 == 0 else o_, n) for k, (c, iv, i_, o_, n) in enumerate(reqs)]
    aes.batch(reqs, tile_blocks=1024)
    cuda.cuda.synchronize()
    out_src, out_dst = to_host(src), to_host(dst)
    for k, (key, b, iv, o, n) in enumerate(meta):
        got = out_src[o: o + n] if k % 2 == 0 else out_dst[o: o + n]
        np.testing.assert_array_equal(got, oracle.ctr_mt(key, b, iv, payload[o: o + n], ncpu),
                                      err_msg=f"request {k} len {n}")


@pytest.mark.parametrize("bits", [128, 256])
def test_batch_every_length_0_to_64(cuda, aes, ncpu, bits):
    """One batch of 65 requests, of every length from 0 to 64 bytes (each
    tail u = 1..15 of a partial final block several times over)."""
    g = W.rng(53 + bits)
    lengths = list(range(65))
    reqs, meta, payload, src, dst = make_requests(cuda, aes, g, lengths, [bits] * len(lengths))
    aes.batch(reqs, tile_blocks=1024)
    check_all(cuda, meta, payload, dst, ncpu)
