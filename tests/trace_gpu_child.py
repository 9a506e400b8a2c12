"""Child process of test_server_gpu.py::test_trace_build_stamps: loads the
trace build (the library must be chosen before it is first loaded), runs
served requests one at a time and checks their stamps."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2607_02630_gb300 import aesoffload as A  # noqa: E402


def main():
    import torch

    A.use_trace_build()
    torch.cuda.set_device(0)
    buf = torch.zeros(2 << 20, dtype=torch.uint8, device="cuda")
    out = torch.zeros_like(buf)
    torch.cuda.synchronize()
    srv = A.Server(slots=8, max_keys=1, idle_timeout_us=500_000, trace_requests=64)
    try:
        slot = srv.key_register(bytes(range(16)), 128)
        n = 40
        for i in range(n):
            t = srv.submit(slot, bytes(16), buf, out, 1 << 20)
            assert srv.wait(t, 10_000_000) == A.AES_OK
        tr = srv.trace()
    finally:
        srv.close()
    rows = tr[1: n + 1].astype(np.int64)  # requests 1..n
    assert (rows > 0).all(), rows
    steps = np.diff(rows, axis=1)
    assert (steps >= 0).all(), steps
    med = np.median(rows - rows[:, :1], axis=0)
    print("OK " + " ".join(f"{k}={v / 1000:.1f}us" for k, v in zip(A.Server.TRACE_POINTS, med)))


if __name__ == "__main__":
    main()
