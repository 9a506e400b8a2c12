"""The reroute harness on the GPU: one block size through the sync, executor
and served modes, every mode's ciphertext identical and equal to the oracle."""
import numpy as np
import pytest

import oracle
from paper_2607_02630_gb300 import reroute as RR

pytestmark = pytest.mark.gpu


def test_run_point_modes_agree_and_match_oracle(cuda, aes, ncpu):
    srv = aes.Server(slots=64, max_keys=4, ctas=32, idle_timeout_us=500_000)
    try:
        key = bytes(range(16))
        n = 65536 + 16
        row = RR.run_point(aes, cuda, cuda.device("cuda", 0), n, srv, key, nclients=8, seconds=0.3, warmup=0.1,
                           executor_threads=4, seed=5)
        assert row["modes_agree"]
        for mode in ("sync", "executor", "served"):
            assert row[f"{mode}_rps"] > 0
        assert row["single_op_us"] > 0
        src, outs, ivs = row["_outputs"]
        for c in (0, 7):
            data = src[c].cpu().numpy()
            want = oracle.ctr_mt(key, 128, np.frombuffer(ivs[c], np.uint8), data, ncpu)
            np.testing.assert_array_equal(outs["served"][c].cpu().numpy(), want)
    finally:
        assert srv.close() == aes.AES_OK
