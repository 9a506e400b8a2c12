"""Where one-in-flight latency goes on the served path (trace build).

Loads libaesoffload_trace.so -- the served kernel with a %globaltimer stamp
at each step of the request protocol -- so it must run in a process that has
not loaded the normal library yet:

    python -m paper_2607_02630_gb300.served_trace [--requests N] [--bytes B]

Submits N requests of B bytes one at a time (the next only after the last
completed), reads the stamps back, checks they are in protocol order, and
prints one JSON line: the median and p99 time of each step from the
request's dispatch, and the median time between consecutive steps.
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np

from . import aesoffload as A


def run(requests: int = 200, nbytes: int = 1 << 20, bits: int = 128, claim_mode: int = 0) -> dict:
    import torch

    A.use_trace_build()
    torch.cuda.set_device(0)
    buf = torch.randint(0, 256, (nbytes + 256,), dtype=torch.uint8, device="cuda")
    out = torch.zeros_like(buf)
    torch.cuda.synchronize()
    cap = 1
    while cap < requests + 2:
        cap <<= 1
    srv = A.Server(slots=8, max_keys=1, idle_timeout_us=2_000_000, trace_requests=cap, claim_mode=claim_mode)
    try:
        slot = srv.key_register(bytes(range(bits // 8)), bits)
        for _ in range(requests):
            t = srv.submit(slot, bytes(16), buf, out, nbytes)
            rc = srv.wait(t, 10_000_000)
            if rc != A.AES_OK:
                raise A.AesError(rc, "offload_wait")
        stamps = srv.trace()
    finally:
        srv.close()
    rows = stamps[1: requests + 1].astype(np.int64)  # sequence numbers 1..requests
    ordered = bool((rows > 0).all() and (np.diff(rows, axis=1) >= 0).all())
    rel = (rows - rows[:, :1]) / 1000.0  # us from dispatch
    steps = np.diff(rows, axis=1) / 1000.0
    names = A.Server.TRACE_POINTS
    return {
        "metric": "served one-in-flight latency breakdown (us from dispatch)",
        "requests": requests, "bytes": nbytes, "bits": bits, "claim_mode": claim_mode,
        "ordered": ordered,
        "median_us": {k: round(float(v), 2) for k, v in zip(names, np.median(rel, axis=0))},
        "p99_us": {k: round(float(v), 2) for k, v in zip(names, np.percentile(rel, 99, axis=0))},
        "median_step_us": {f"{a}->{b}": round(float(v), 2)
                           for a, b, v in zip(names[:-1], names[1:], np.median(steps, axis=0))},
        "how": "trace build (per-request %globaltimer stamps), one request in flight, default tiles",
    }


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--bytes", type=int, default=1 << 20)
    ap.add_argument("--bits", type=int, default=128, choices=[128, 192, 256])
    ap.add_argument("--claim-mode", type=int, default=0, choices=[0, 1])
    a = ap.parse_args(argv)
    res = run(a.requests, a.bytes, a.bits, a.claim_mode)
    print(json.dumps(res), flush=True)
    return 0 if res["ordered"] else 1


if __name__ == "__main__":
    sys.exit(main())
