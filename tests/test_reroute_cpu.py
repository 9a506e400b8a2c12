"""The reroute harness (single-event-loop server, 50 clients, sync vs
executor vs served) with stand-in offloads of fixed duration, on the CPU.

The stand-ins take 2 ms each.  A server that waits for the offload on its
event loop completes at most one request per 2 ms whatever the number of
clients; rerouting through an executor or a submit/poll offload lets the
loop keep serving, so throughput grows with the requests in flight (the
paper's Sec. 3 claim, measured by its App. A sweep).
"""
import threading
import time

from paper_2607_02630_gb300 import reroute as RR

OFFLOAD_S = 0.002


class FakeBlocking:
    def __init__(self):
        self.calls = 0
        self.lock = threading.Lock()

    def run_blocking(self, conn, nbytes):
        time.sleep(OFFLOAD_S)
        with self.lock:
            self.calls += 1


class FakeServed:
    """submit() returns a future that a timer thread resolves later."""

    def __init__(self):
        self.calls = 0

    def submit(self, loop, conn, nbytes):
        fut = loop.create_future()
        self.calls += 1
        t = threading.Timer(OFFLOAD_S, lambda: loop.call_soon_threadsafe(RR._resolve, fut, None))
        t.daemon = True
        t.start()
        return fut


def run(mode, off, clients=50, threads=32):
    srv = RR.RerouteServer(mode, off, 4096, executor_threads=threads)
    try:
        return RR.drive(srv, nclients=clients, seconds=0.6, warmup=0.2), srv
    finally:
        srv.close()


def test_sync_is_bounded_by_the_offload():
    off = FakeBlocking()
    rps, srv = run("sync", off)
    assert 0 < rps <= 1.1 / OFFLOAD_S
    assert srv.served == off.calls and srv.conns == 50


def test_reroute_overlaps_offloads():
    sync_rps, _ = run("sync", FakeBlocking())
    exe_rps, _ = run("executor", FakeBlocking(), threads=32)
    srv_rps, _ = run("served", FakeServed())
    assert exe_rps > 4 * sync_rps
    assert srv_rps > 4 * sync_rps


def test_executor_capacity_caps_overlap():
    """With 4 executor threads at most 4 offloads overlap."""
    rps, _ = run("executor", FakeBlocking(), threads=4)
    assert rps <= 4 * 1.1 / OFFLOAD_S


def test_bad_mode_rejected():
    import pytest

    with pytest.raises(ValueError):
        RR.RerouteServer("threads", FakeBlocking(), 16)
