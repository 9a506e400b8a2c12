"""aes_ctr_batch_noalloc: the batched launch for callers that cannot allocate.

Callers whose device memory is already fully reserved by another pool, or
that must not pay for cudaMalloc/cudaFree on a latency-critical path, use
this entry point: it keeps its scratch in a static device array instead of
allocating.  Every request's output must equal the CPU oracle's bytes
(tolerance 0: AES-CTR has one correct output) and the bytes aes_ctr_batch
gives for the same requests, on calls in a row that reuse the same scratch
array -- including a call with the maximum of 1024 requests, and calls under
other tuned shapes (one block per lane in flight; 1024-thread CTAs holding
round keys in shared memory).  This file is collected last on purpose and
also passes when run alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2607_02630_gb300 import workloads as W

from gpu_util import set_batch_shape

pytestmark = pytest.mark.gpu

MAX_REQUESTS = 1024  # AES_NOALLOC_MAX_REQUESTS


def _requests(torch, aes, g, n, max_len):
    lens = [0, 1, 15, 16, 17, 4096 + 3] + [int(x) for x in np.exp(g.uniform(np.log(512), np.log(max_len), n - 6))]
    pad = [(k + 255) // 256 * 256 + 256 for k in lens]
    offs = np.concatenate([[0], np.cumsum(pad)[:-1]]).astype(np.int64)
    total = int(sum(pad))
    payload = W.random_bytes(g, total)
    src = torch.from_numpy(payload).cuda()
    dst_ref = torch.full((total,), 0xA5, dtype=torch.uint8, device="cuda")
    dst_new = torch.full((total,), 0x5A, dtype=torch.uint8, device="cuda")
    keys, ctxs, ivs = [], [], []
    for i in range(len(lens)):
        bits = (128, 192, 256)[i % 3]
        key = W.random_bytes(g, bits // 8)
        keys.append((key, bits))
        ctxs.append(aes.Context(key.tobytes(), bits))
        ivs.append(W.random_bytes(g, 16))

    def reqs(dst):
        return [(ctxs[i], ivs[i].tobytes(), src.data_ptr() + int(offs[i]), dst.data_ptr() + int(offs[i]), lens[i])
                for i in range(len(lens))]

    return reqs, dst_ref, dst_new, lens, offs, payload, keys, ivs, ctxs


def _noalloc(aes, lib, reqs, stream):
    arr = aes._descs(reqs)
    return lib.aes_ctr_batch_noalloc(arr, len(reqs), stream)


def _check_against_oracle_and_batch(cuda, aes, lib, stream, g, n, max_len, ncpu, label):
    reqs, dst_ref, dst_new, lens, offs, payload, keys, ivs, ctxs = _requests(cuda, aes, g, n, max_len)
    aes.batch(reqs(dst_ref), stream=stream)
    rc = _noalloc(aes, lib, reqs(dst_new), stream)
    assert rc == aes.AES_OK, aes.strerror(rc)
    cuda.cuda.synchronize()
    ref, new = dst_ref.cpu().numpy(), dst_new.cpu().numpy()
    for i, k in enumerate(lens):
        o = int(offs[i])
        key, bits = keys[i]
        want = oracle.ctr_mt(key, bits, ivs[i], payload[o: o + k], ncpu)
        np.testing.assert_array_equal(new[o: o + k], want, err_msg=f"{label}: request {i} vs the oracle")
        np.testing.assert_array_equal(new[o: o + k], ref[o: o + k], err_msg=f"{label}: request {i} vs aes_ctr_batch")
        assert (new[o + k: o + k + 16] == 0x5A).all(), f"{label}: bytes past len were written (request {i})"


@pytest.fixture()
def noalloc_lib(aes):
    lib = aes.lib()
    lib.aes_ctr_batch_noalloc.restype = ctypes.c_int
    lib.aes_ctr_batch_noalloc.argtypes = [ctypes.POINTER(aes.Desc), ctypes.c_int, ctypes.c_void_p]
    return lib


def test_no_alloc_batch_matches_oracle_and_batch_on_calls_in_a_row(cuda, aes, noalloc_lib, ncpu):
    stream = int(cuda.cuda.current_stream().cuda_stream)
    g = W.rng(77)
    # calls in a row: a large batch, a smaller one that leaves the first
    # call's descriptors behind in the shared scratch array, then the most
    # requests the array holds
    for n, max_len in ((300, 3 << 20), (37, 1 << 20), (MAX_REQUESTS, 64 << 10)):
        _check_against_oracle_and_batch(cuda, aes, noalloc_lib, stream, g, n, max_len, ncpu, f"n={n}")


@pytest.mark.parametrize("shape", [(1, 256, 1024, 1), (1, 1024, 4096, 4)], ids=["nb1_t256", "nb4_t1024_smem_keys"])
def test_no_alloc_batch_under_other_shapes(cuda, aes, noalloc_lib, ncpu, tmp_path, shape):
    stream = int(cuda.cuda.current_stream().cuda_stream)
    default = set_batch_shape(cuda, aes, tmp_path / "shape.json", shape)
    try:
        g = W.rng(78 + shape[1])
        for n, max_len in ((64, 2 << 20), (9, 256 << 10)):
            _check_against_oracle_and_batch(cuda, aes, noalloc_lib, stream, g, n, max_len, ncpu,
                                            f"shape={shape} n={n}")
    finally:
        set_batch_shape(cuda, aes, tmp_path / "shape.json", default)


def test_no_alloc_batch_rejects_too_many_requests(cuda, aes, noalloc_lib):
    ctx = aes.Context(bytes(16), 128)
    buf = cuda.zeros(1 << 12, dtype=cuda.uint8, device="cuda")
    n = MAX_REQUESTS + 1
    arr = aes._descs([(ctx, bytes(16), buf.data_ptr(), buf.data_ptr(), 16)] * n)
    assert noalloc_lib.aes_ctr_batch_noalloc(arr, n, None) == aes.AES_ETOOBIG
    assert noalloc_lib.aes_ctr_batch_noalloc(arr, 0, None) == aes.AES_OK
    assert noalloc_lib.aes_ctr_batch_noalloc(arr, -1, None) == aes.AES_EINVAL
