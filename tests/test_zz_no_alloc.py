"""aes_ctr_batch_noalloc: the batched launch for callers that cannot allocate.

Callers whose device memory is already fully reserved by another pool, or
that must not pay for cudaMalloc/cudaFree on a latency-critical path, use
this entry point: it keeps its scratch in a static device array instead of
allocating.  It must give exactly the bytes aes_ctr_batch gives (tolerance
0: AES-CTR has one correct output), on two calls in a row that reuse the
same scratch array.  This file is collected last on purpose and also passes
when run alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2607_02630_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _requests(torch, aes, g, n, max_len):
    lens = [0, 1, 15, 16, 17, 4096 + 3] + [int(x) for x in np.exp(g.uniform(np.log(512), np.log(max_len), n - 6))]
    pad = [(k + 255) // 256 * 256 + 256 for k in lens]
    offs = np.concatenate([[0], np.cumsum(pad)[:-1]]).astype(np.int64)
    total = int(sum(pad))
    src = torch.from_numpy(W.random_bytes(g, total)).cuda()
    dst_ref = torch.full((total,), 0xA5, dtype=torch.uint8, device="cuda")
    dst_new = torch.full((total,), 0x5A, dtype=torch.uint8, device="cuda")
    ctxs, ivs = [], []
    for i in range(len(lens)):
        bits = (128, 192, 256)[i % 3]
        ctxs.append(aes.Context(W.random_bytes(g, bits // 8).tobytes(), bits))
        ivs.append(W.random_bytes(g, 16).tobytes())

    def reqs(dst):
        return [(ctxs[i], ivs[i], src.data_ptr() + int(offs[i]), dst.data_ptr() + int(offs[i]), lens[i])
                for i in range(len(lens))]

    return reqs, dst_ref, dst_new, lens, offs, ctxs


def test_no_alloc_batch_matches_existing_batch_on_two_calls(cuda, aes):
    lib = aes.lib()
    lib.aes_ctr_batch_noalloc.restype = ctypes.c_int
    lib.aes_ctr_batch_noalloc.argtypes = [ctypes.POINTER(aes.Desc), ctypes.c_int, ctypes.c_void_p]
    stream = int(cuda.cuda.current_stream().cuda_stream)
    g = W.rng(77)
    # two calls in a row: a large batch, then a smaller one that leaves the
    # first call's descriptors behind in the shared scratch array
    for n, max_len in ((300, 3 << 20), (37, 1 << 20)):
        reqs, dst_ref, dst_new, lens, offs, ctxs = _requests(cuda, aes, g, n, max_len)
        aes.batch(reqs(dst_ref), stream=stream)
        arr = aes._descs(reqs(dst_new))
        rc = lib.aes_ctr_batch_noalloc(arr, len(lens), stream)
        assert rc == aes.AES_OK, aes.strerror(rc)
        cuda.cuda.synchronize()
        ref, new = dst_ref.cpu().numpy(), dst_new.cpu().numpy()
        for i, k in enumerate(lens):
            o = int(offs[i])
            np.testing.assert_array_equal(new[o: o + k], ref[o: o + k], err_msg=f"request {i} (n={n})")
            assert (new[o + k: o + k + 16] == 0x5A).all(), "bytes past len were written"


def test_no_alloc_batch_rejects_too_many_requests(cuda, aes):
    lib = aes.lib()
    lib.aes_ctr_batch_noalloc.restype = ctypes.c_int
    lib.aes_ctr_batch_noalloc.argtypes = [ctypes.POINTER(aes.Desc), ctypes.c_int, ctypes.c_void_p]
    ctx = aes.Context(bytes(16), 128)
    buf = cuda.zeros(1 << 12, dtype=cuda.uint8, device="cuda")
    n = 1025  # AES_NOALLOC_MAX_REQUESTS + 1
    arr = aes._descs([(ctx, bytes(16), buf.data_ptr(), buf.data_ptr(), 16)] * n)
    assert lib.aes_ctr_batch_noalloc(arr, n, None) == aes.AES_ETOOBIG
    assert lib.aes_ctr_batch_noalloc(arr, 0, None) == aes.AES_OK
    assert lib.aes_ctr_batch_noalloc(arr, -1, None) == aes.AES_EINVAL
