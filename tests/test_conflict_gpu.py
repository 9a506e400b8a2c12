"""The conflict detector with a real GPU offload: handlers park at served
requests (emulated offloads, and real AES-CTR requests) while the detector
guards the shared counters."""
import numpy as np
import pytest

import oracle
from paper_2607_02630_gb300 import aesoffload as A

pytestmark = pytest.mark.gpu


EMULATE = pytest.mark.parametrize("emulate", [True, False], ids=["emulated_stores", "unprotect"])


@EMULATE
def test_enforce_with_served_emulated_offload(cuda, aes, emulate):
    srv = aes.Server(slots=64, max_keys=1, ctas=16, idle_timeout_us=500_000)
    try:
        un = aes.conflict_run(aes.CDET_UNPROTECTED, handlers=16, requests=2000, counters=16, offload_ns=20_000,
                              server=srv)
        enf = aes.conflict_run(aes.CDET_ENFORCE, handlers=16, requests=2000, counters=16, offload_ns=20_000,
                               server=srv, emulate_stores=emulate)
        assert un["lost_updates"] > 0
        assert enf["lost_updates"] == 0 and enf["final_count"] == 2000 and enf["conflicts"] > 0
    finally:
        assert srv.close() == aes.AES_OK


@EMULATE
def test_enforce_with_real_aes_offload(cuda, aes, ncpu, emulate):
    srv = aes.Server(slots=64, max_keys=1, ctas=32, idle_timeout_us=500_000)
    try:
        key = bytes(range(16))
        ks = srv.key_register(key, 128)
        handlers, nbytes = 8, 64 << 10
        src = cuda.randint(0, 256, (handlers * nbytes,), dtype=cuda.uint8, device="cuda")
        dst = cuda.zeros_like(src)
        cuda.cuda.synchronize()  # the served kernel runs on its own stream
        r = aes.conflict_run(aes.CDET_ENFORCE, handlers=handlers, requests=800, counters=8, server=srv,
                             key_slot=ks, buf_in=src, buf_out=dst, nbytes=nbytes, emulate_stores=emulate)
        assert r["lost_updates"] == 0 and r["final_count"] == 800
        # Request q encrypts under IV q (little-endian in bytes 0..3): find the
        # request whose keystream handler 0's block carries, then check the
        # whole block against the oracle.
        cuda.cuda.synchronize()
        data = src[:nbytes].cpu().numpy()
        out = dst[:nbytes].cpu().numpy()
        ks0 = out[:16] ^ data[:16]
        zero = np.zeros(16, np.uint8)
        ivs = [np.frombuffer(int(q).to_bytes(4, "little") + bytes(12), np.uint8) for q in range(800)]
        hits = [iv for iv in ivs if np.array_equal(oracle.ctr(key, 128, iv, zero), ks0)]
        assert len(hits) == 1
        np.testing.assert_array_equal(out, oracle.ctr_mt(key, 128, hits[0], data, ncpu))
    finally:
        assert srv.close() == aes.AES_OK


@pytest.mark.parametrize("pattern", [A.CDET_PATTERN_READONLY, A.CDET_PATTERN_PER_CONN, A.CDET_PATTERN_LOCKED],
                         ids=["read_only", "per_connection", "lock_protected"])
def test_safe_patterns_with_served_emulated_offload(cuda, aes, pattern):
    """Over a served (emulated) offload, the shared-state patterns the paper
    finds safe raise no conflict and lose nothing under detection."""
    srv = aes.Server(slots=64, max_keys=1, ctas=16, idle_timeout_us=500_000)
    try:
        r = aes.conflict_run(aes.CDET_DETECT, handlers=16, requests=1000, counters=16, offload_ns=20_000,
                             server=srv, pattern=pattern)
        assert r["conflicts"] == 0 and r["lost_updates"] == 0 and r["final_count"] == 1000, r
    finally:
        assert srv.close() == aes.AES_OK


def test_more_handlers_than_server_slots(cuda, aes):
    """16 handlers on a server with 4 request slots: a handler that finds
    every slot held reaps the parked handlers' completions itself (the event
    loop cannot run meanwhile), so the run completes; enforcement still loses
    nothing."""
    srv = aes.Server(slots=4, max_keys=1, ctas=16, idle_timeout_us=500_000)
    try:
        r = aes.conflict_run(aes.CDET_ENFORCE, handlers=16, requests=1000, counters=16, offload_ns=20_000,
                             server=srv)
        assert r["lost_updates"] == 0 and r["final_count"] == 1000, r
    finally:
        assert srv.close() == aes.AES_OK


# ---- the detector's host-only parts, on the host the GPU is attached to ----
# The store emulation decodes the faulting store instruction, so it depends
# on the CPU architecture: x86-64 where the CPU tests run, AArch64 (Grace) on
# GB300 machines.  These re-run the CPU suite's store-emulation checks there.

def test_store_emulation_selftest_on_the_gpu_host(aes):
    import platform

    import test_conflict_cpu as cpu

    r = aes.store_selftest(6000)
    print(f"store self-test on {platform.machine()}: {r}")
    cpu.test_store_emulation_selftest()


@pytest.mark.parametrize("mode", [A.CDET_DETECT, A.CDET_ENFORCE], ids=["detect", "enforce"])
def test_emulated_stores_on_the_gpu_host(aes, mode):
    import test_conflict_cpu as cpu

    cpu.test_emulated_stores_keep_the_detectors_results(mode)
    cpu.test_protection_changes_per_guarded_write()


def test_detector_under_ubsan_on_the_gpu_host(aes, tmp_path):
    import test_conflict_cpu as cpu

    cpu.test_detector_under_undefined_behaviour_sanitizer(tmp_path, "-O2")
