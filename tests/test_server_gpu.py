"""Served mode: resident kernel polling mapped descriptors (offload_*).

Checks bit-exact results against the oracle, that every request gives the
same bytes alone and in a concurrent mix, admission (slots, HBM budget),
tickets, idle exit + relaunch and the stop path.  Every device wait in the
resident kernel is bounded, so none of these can hang the GPU; host waits
use offload_wait with a timeout.
"""
import ctypes
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2607_02630_gb300 import workloads as W

from gpu_util import iv_plus, iv_with_low, to_dev, to_host

pytestmark = pytest.mark.gpu

WAIT_US = 10_000_000


@pytest.fixture(autouse=True, params=[0, 1], ids=["cursor", "per_request"])
def claim_mode(request, monkeypatch, aes):
    """Every test of this module runs under both tile-claim protocols of the
    served kernel: the global cursor (claim_mode 0) and per-request claim
    words (claim_mode 1).  Servers created without an explicit claim_mode
    get the parametrised one."""
    base = aes.Server

    class ModeServer(base):
        def __init__(self, *args, **kw):
            kw.setdefault("claim_mode", request.param)
            super().__init__(*args, **kw)

    monkeypatch.setattr(aes, "Server", ModeServer)
    return request.param


@pytest.fixture()
def server(aes, claim_mode):
    srv = aes.Server(slots=64, max_keys=16, ctas=32, tile_blocks=2048, idle_timeout_us=500_000)
    yield srv
    assert srv.close() == aes.AES_OK


def arena(torch, g, sizes):
    """Payloads at 256-byte aligned offsets in one device buffer, and an
    output buffer of 0xA5.  The fills run on torch's stream and the served
    kernel on the server's own, so wait for them before submitting."""
    pad = [(n + 255) // 256 * 256 + 256 for n in sizes]
    offs = np.concatenate([[0], np.cumsum(pad)[:-1]]).astype(np.int64)
    payload = W.random_bytes(g, int(sum(pad)))
    src, dst = to_dev(torch, payload), to_dev(torch, np.zeros(0, np.uint8), pad=int(sum(pad)))
    torch.cuda.synchronize()
    return payload, offs, src, dst


def test_served_results_match_oracle(cuda, aes, server, ncpu):
    g = W.rng(60)
    keys = [(W.random_bytes(g, b // 8), b) for b in (128, 256, 192, 128)]
    slots = [server.key_register(k.tobytes(), b) for k, b in keys]
    sizes = [0, 1, 15, 16, 17, 4096, 65536 + 3, 1 << 20, (1 << 20) + 9, 3 << 20, 8 << 20] + \
        [int(x) for x in W.served_sizes(20, seed=61) if x <= (1 << 20)]
    payload, offs, src, dst = arena(cuda, g, sizes)
    tickets = []
    for i, n in enumerate(sizes):
        iv = W.random_bytes(g, 16)
        k = i % len(keys)
        o = int(offs[i])
        t = server.submit(slots[k], iv.tobytes(), src.data_ptr() + o, dst.data_ptr() + o, n)
        tickets.append((t, k, iv, o, n))
    for t, k, iv, o, n in tickets:
        assert server.wait(t, WAIT_US) == aes.AES_OK
    out = to_host(dst)
    for t, k, iv, o, n in tickets:
        key, bits = keys[k]
        np.testing.assert_array_equal(out[o: o + n], oracle.ctr_mt(key, bits, iv, payload[o: o + n], ncpu))
        assert (out[o + n: o + n + 16] == 0xA5).all()
    st = server.stats()
    assert st["completed"] == len(sizes) and st["device_errors"] == 0


def test_keys_registered_while_resident(cuda, aes, ncpu):
    """Keys registered while the resident kernel runs: each new slot's first
    round key shares a cache line with the slot before it, which the kernel
    has just read.  Every request must use the key as registered."""
    srv = aes.Server(slots=16, max_keys=8, ctas=8, tile_blocks=1024, idle_timeout_us=5_000_000)
    try:
        g = W.rng(67)
        size = 256 << 10
        keys = [(W.random_bytes(g, b // 8), b) for b in (128, 256, 192, 128, 256, 192, 128, 256)]
        payload, offs, src, dst = arena(cuda, g, [size] * (2 * len(keys)))
        ivs = [W.random_bytes(g, 16) for _ in range(2 * len(keys))]
        relaunches = None
        for k, (key, bits) in enumerate(keys):
            slot = srv.key_register(key.tobytes(), bits)
            assert slot == k
            for i in (2 * k, 2 * k + 1):  # 16 tiles each: every CTA reads this slot
                o = int(offs[i])
                t = srv.submit(slot, ivs[i].tobytes(), src.data_ptr() + o, dst.data_ptr() + o, size)
                assert srv.wait(t, WAIT_US) == aes.AES_OK
            st = srv.stats()
            if relaunches is None:
                relaunches = st["relaunches"]
            assert st["running"] == 1 and st["relaunches"] == relaunches, st  # still the same launch
        out = to_host(dst)
        for i in range(2 * len(keys)):
            key, bits = keys[i // 2]
            o = int(offs[i])
            np.testing.assert_array_equal(out[o: o + size], oracle.ctr_mt(key, bits, ivs[i], payload[o: o + size], ncpu))
    finally:
        assert srv.close() == aes.AES_OK


def test_same_result_alone_and_in_the_mix(cuda, aes, server):
    """Each request's bytes do not depend on what else is on the GPU."""
    g = W.rng(62)
    keys = [(W.random_bytes(g, b // 8), b) for b in (128, 256)]
    slots = [server.key_register(k.tobytes(), b) for k, b in keys]
    sizes = [int(x) for x in W.served_sizes(48, seed=63)]
    sizes = [min(n, 2 << 20) for n in sizes]
    payload, offs, src, dst = arena(cuda, g, sizes)
    ivs = [W.random_bytes(g, 16).tobytes() for _ in sizes]
    # alone: one request in flight at a time
    alone = []
    for i, n in enumerate(sizes):
        o = int(offs[i])
        t = server.submit(slots[i % 2], ivs[i], src.data_ptr() + o, dst.data_ptr() + o, n)
        assert server.wait(t, WAIT_US) == aes.AES_OK
        alone.append(to_host(dst[o: o + n]).copy())
    # in the mix: all submitted back to back, completing out of order
    dst.fill_(0xA5)
    cuda.cuda.synchronize()  # the served kernel runs on its own stream
    order = list(g.permutation(len(sizes)))
    tickets = []
    for i in order:
        o = int(offs[i])
        tickets.append((i, server.submit(slots[i % 2], ivs[i], src.data_ptr() + o, dst.data_ptr() + o,
                                         sizes[i])))
    for i, t in tickets:
        assert server.wait(t, WAIT_US) == aes.AES_OK
    for i, n in enumerate(sizes):
        o = int(offs[i])
        np.testing.assert_array_equal(to_host(dst[o: o + n]), alone[i], err_msg=f"request {i}")


def test_poll_right_after_submit_and_ticket_rules(cuda, aes, server):
    slot = server.key_register(bytes(16), 128)
    buf = cuda.zeros(1 << 20, dtype=cuda.uint8, device="cuda")
    t = server.submit(slot, bytes(16), buf.data_ptr(), buf.data_ptr(), 1 << 20)
    assert server.poll(t) in (aes.AES_PENDING, aes.AES_OK)  # never unknown
    assert server.wait(t, WAIT_US) in (aes.AES_OK, aes.AES_EINVAL)
    assert server.poll(t) == aes.AES_EINVAL  # released
    assert server.poll(0) == aes.AES_EINVAL
    assert server.poll(t ^ (1 << 40)) == aes.AES_EINVAL


def test_submit_argument_errors(cuda, aes, server):
    slot = server.key_register(bytes(32), 256)
    buf = cuda.zeros(1 << 16, dtype=cuda.uint8, device="cuda")
    p = buf.data_ptr()
    assert server.submit_status(slot + 5, bytes(16), p, p, 64)[0] == aes.AES_EINVAL  # unregistered
    assert server.submit_status(-1, bytes(16), p, p, 64)[0] == aes.AES_EINVAL
    assert server.submit_status(slot, bytes(16), p + 4, p + 4096, 64)[0] == aes.AES_EALIGN
    assert server.submit_status(slot, bytes(16), p, p + 16, 64)[0] == aes.AES_EOVERLAP
    assert server.submit_status(slot, bytes(16), p, p, 1 << 50)[0] == aes.AES_ETOOBIG
    rc, t = server.submit_status(slot, bytes(16), 0, 0, 0)  # empty request completes
    assert rc == aes.AES_OK and server.wait(t, WAIT_US) == aes.AES_OK


def test_slots_exhausted_gives_eagain(cuda, aes):
    srv = aes.Server(slots=4, max_keys=2, ctas=2, idle_timeout_us=500_000)
    slot = srv.key_register(bytes(16), 128)
    buf = cuda.zeros(64 << 20, dtype=cuda.uint8, device="cuda")
    p = buf.data_ptr()
    n = 8 << 20
    tickets = []
    saw_again = False
    for i in range(6):
        rc, t = srv.submit_status(slot, bytes(16), p + i * n, p + i * n, n)
        if rc == aes.AES_EAGAIN:
            saw_again = True
        else:
            assert rc == aes.AES_OK
            tickets.append(t)
    assert len(tickets) <= 4 and saw_again  # ~0.3 ms per 8 MiB request on 2 CTAs
    for t in tickets:
        assert srv.wait(t, WAIT_US) == aes.AES_OK
    rc, t = srv.submit_status(slot, bytes(16), p, p, n)  # slots free again
    assert rc == aes.AES_OK and srv.wait(t, WAIT_US) == aes.AES_OK
    assert srv.close() == aes.AES_OK


def test_hbm_budget_back_pressure(cuda, aes):
    n = 8 << 20
    budget = 3 * n  # three in-place 8 MiB requests
    srv = aes.Server(slots=64, max_keys=2, ctas=4, hbm_budget=budget, idle_timeout_us=500_000)
    slot = srv.key_register(bytes(16), 128)
    buf = cuda.zeros(12 * n, dtype=cuda.uint8, device="cuda")
    p = buf.data_ptr()
    # out-of-place counts in + out: 2 * 2n > budget can never be admitted
    assert srv.submit_status(slot, bytes(16), p, p + 4 * n, 2 * n)[0] == aes.AES_ETOOBIG
    accepted, rejected = [], 0
    for i in range(12):
        rc, t = srv.submit_status(slot, bytes(16), p + i * n, p + i * n, n)
        if rc == aes.AES_EAGAIN:
            rejected += 1
        else:
            assert rc == aes.AES_OK
            accepted.append(t)
    assert rejected > 0 and len(accepted) >= 3
    for t in accepted:
        assert srv.wait(t, WAIT_US) == aes.AES_OK
    st = srv.stats()
    assert st["rejected_eagain"] == rejected
    rc, t = srv.submit_status(slot, bytes(16), p, p, n)
    assert rc == aes.AES_OK and srv.wait(t, WAIT_US) == aes.AES_OK
    assert srv.close() == aes.AES_OK


def test_idle_exit_then_relaunch(cuda, aes, ncpu):
    srv = aes.Server(slots=8, max_keys=2, ctas=8, idle_timeout_us=20_000)
    key = np.arange(16, dtype=np.uint8)
    slot = srv.key_register(key.tobytes(), 128)
    g = W.rng(64)
    data = W.random_bytes(g, 1 << 20)
    src = to_dev(cuda, data)
    dst = to_dev(cuda, np.zeros(0, np.uint8), pad=data.size)
    cuda.cuda.synchronize()
    iv = W.random_bytes(g, 16)
    t = srv.submit(slot, iv.tobytes(), src, dst, data.size)
    assert srv.wait(t, WAIT_US) == aes.AES_OK
    deadline = time.time() + 5
    while srv.stats()["running"] and time.time() < deadline:
        time.sleep(0.01)
    st = srv.stats()
    assert st["running"] == 0 and (st["kernel_status"] & 2), st  # exited on idle timeout
    dst.fill_(0)
    cuda.cuda.synchronize()
    t = srv.submit(slot, iv.tobytes(), src, dst, data.size)
    assert srv.wait(t, WAIT_US) == aes.AES_OK
    assert srv.stats()["relaunches"] >= 1
    np.testing.assert_array_equal(to_host(dst), oracle.ctr_mt(key, 128, iv, data, ncpu))
    assert srv.close() == aes.AES_OK


def test_light_load_keeps_every_cta_resident(cuda, aes, ncpu):
    """Requests of a few tiles, one every 10 ms: each is claimed by one or
    two of the 32 CTAs, so most CTAs go far longer than the idle timeout
    without a tile of their own.  Idle means no new request anywhere, so no
    CTA may exit while requests keep coming (kernel_status stays 0)."""
    srv = aes.Server(slots=8, max_keys=1, ctas=32, tile_blocks=64, idle_timeout_us=150_000)
    try:
        g = W.rng(68)
        key = W.random_bytes(g, 16)
        slot = srv.key_register(key.tobytes(), 128)
        n, size = 60, 1024
        payload, offs, src, dst = arena(cuda, g, [size] * n)
        ivs = [W.random_bytes(g, 16) for _ in range(n)]
        # Start from a launch whose CTAs are all resident: if the setup above
        # outlasted the idle timeout, let that launch end and relaunch it.
        t = srv.submit(slot, ivs[0].tobytes(), src.data_ptr() + int(offs[0]), dst.data_ptr() + int(offs[0]), size)
        assert srv.wait(t, WAIT_US) == aes.AES_OK
        if srv.stats()["kernel_status"] != 0:
            deadline = time.time() + 5
            while srv.stats()["running"] and time.time() < deadline:
                time.sleep(0.01)
            t = srv.submit(slot, ivs[0].tobytes(), src.data_ptr() + int(offs[0]), dst.data_ptr() + int(offs[0]),
                           size)
            assert srv.wait(t, WAIT_US) == aes.AES_OK
        base = srv.stats()["relaunches"]
        t_start = time.time()
        for i in range(n):
            o = int(offs[i])
            t = srv.submit(slot, ivs[i].tobytes(), src.data_ptr() + o, dst.data_ptr() + o, size)
            assert srv.wait(t, WAIT_US) == aes.AES_OK
            time.sleep(0.01)
        elapsed = time.time() - t_start
        st = srv.stats()
        assert elapsed >= 0.55  # several idle timeouts of light load
        assert st["running"] == 1 and st["relaunches"] == base and st["kernel_status"] == 0, st
        out = to_host(dst)
        for i in range(n):
            o = int(offs[i])
            np.testing.assert_array_equal(out[o: o + size], oracle.ctr(key, 128, ivs[i], payload[o: o + size]))
    finally:
        assert srv.close() == aes.AES_OK


def test_stop_with_work_in_flight(cuda, aes):
    srv = aes.Server(slots=32, max_keys=2, ctas=16, idle_timeout_us=2_000_000)
    slot = srv.key_register(bytes(16), 128)
    buf = cuda.zeros(256 << 20, dtype=cuda.uint8, device="cuda")
    p = buf.data_ptr()
    for i in range(32):
        srv.submit_status(slot, bytes(16), p + i * (8 << 20), p + i * (8 << 20), 8 << 20)
    t0 = time.time()
    assert srv.close() == aes.AES_OK
    assert time.time() - t0 < 5


def test_eight_submitter_threads(cuda, aes, ncpu):
    srv = aes.Server(slots=128, max_keys=8, ctas=64, tile_blocks=2048, idle_timeout_us=1_000_000)
    g = W.rng(65)
    keys = [(W.random_bytes(g, b // 8), b) for b in (128, 256) * 4]
    slots = [srv.key_register(k.tobytes(), b) for k, b in keys]
    per_thread = 24
    sizes = [int(min(x, 1 << 20)) for x in W.served_sizes(8 * per_thread, seed=66)]
    payload, offs, src, dst = arena(cuda, g, sizes)
    ivs = [W.random_bytes(g, 16).tobytes() for _ in sizes]
    errors = []

    def worker(tid):
        try:
            mine = []
            for j in range(per_thread):
                i = tid * per_thread + j
                o = int(offs[i])
                while True:
                    rc, t = srv.submit_status(slots[i % 8], ivs[i], src.data_ptr() + o, dst.data_ptr() + o,
                                              sizes[i])
                    if rc != aes.AES_EAGAIN:
                        break
                assert rc == aes.AES_OK, rc
                mine.append(t)
            for t in mine:
                assert srv.wait(t, WAIT_US) == aes.AES_OK
        except Exception as e:  # surfaced below
            errors.append(e)

    th = [threading.Thread(target=worker, args=(k,)) for k in range(8)]
    for x in th:
        x.start()
    for x in th:
        x.join(60)
    assert not errors, errors
    out = to_host(dst)
    for i, n in enumerate(sizes):
        o = int(offs[i])
        key, bits = keys[i % 8]
        want = oracle.ctr(key, bits, np.frombuffer(ivs[i], np.uint8), payload[o: o + n])
        np.testing.assert_array_equal(out[o: o + n], want, err_msg=f"request {i}")
    assert srv.close() == aes.AES_OK


@pytest.mark.parametrize("path", ["served", "per_call"])
def test_open_loop_drivers_match_oracle(cuda, aes, path):
    """offload_drive / aes_ctr_drive: Poisson arrivals over 8 submitter
    threads; every output equals the oracle's and every latency is measured
    from the scheduled arrival."""
    g = W.rng(70)
    n = 160
    sizes = [int(x) for x in W.served_sizes(n, seed=71)]
    sizes = [min(s, 1 << 20) for s in sizes]
    payload, offs, src, dst = arena(cuda, g, sizes)
    keys = [(W.random_bytes(g, b // 8), b) for b in (128, 256, 128, 256)]
    ivs = W.random_bytes(g, 16 * n).reshape(n, 16)
    reqs = np.zeros(n, dtype=aes.drive_dtype())
    reqs["iv"] = ivs
    reqs["inp"] = src.data_ptr() + offs
    reqs["out"] = dst.data_ptr() + offs
    reqs["len"] = sizes
    reqs["arrival_s"] = W.poisson_arrivals(n, 20_000.0, seed=72)
    kidx = np.arange(n) % 4
    if path == "served":
        srv = aes.Server(slots=64, max_keys=4, ctas=32, idle_timeout_us=1_000_000)
        reqs["key_slot"] = np.array([srv.key_register(k.tobytes(), b) for k, b in keys])[kidx]
        lat, res = aes.drive_served(srv, reqs, 8)
        assert srv.close() == aes.AES_OK
    else:
        ctxs = [aes.Context(k.tobytes(), b) for k, b in keys]
        reqs["key_slot"] = kidx
        lat, res = aes.drive_per_call(ctxs, reqs, 8)
    assert res["errors"] == 0 and res["bytes"] == sum(sizes)
    assert (lat > 0).all()
    out = to_host(dst)
    for i, n_i in enumerate(sizes):
        key, bits = keys[kidx[i]]
        o = int(offs[i])
        np.testing.assert_array_equal(out[o: o + n_i], oracle.ctr(key, bits, ivs[i], payload[o: o + n_i]),
                                      err_msg=f"request {i}")


def test_zero_length_requests_with_slot_reuse(cuda, aes, ncpu):
    """A zero-length request completes when the device reads it, so its slot
    can be reused for a later request before the claim cursor reaches it.
    Interleave zero-length requests (polled and their slots reused at once)
    with real ones on a server with few slots: everything must complete and
    the real requests must match the oracle."""
    srv = aes.Server(slots=4, max_keys=2, ctas=16, idle_timeout_us=500_000)
    try:
        g = W.rng(66)
        key = W.random_bytes(g, 16)
        ks = srv.key_register(key.tobytes(), 128)
        n_real, size = 48, 256 << 10
        payload, offs, src, dst = arena(cuda, g, [size] * n_real)
        ivs = [W.random_bytes(g, 16) for _ in range(n_real)]
        pending = []
        zeros = 0
        for i in range(n_real):
            while True:
                rc, t = srv.submit_status(ks, ivs[i].tobytes(), src.data_ptr() + int(offs[i]),
                                          dst.data_ptr() + int(offs[i]), size)
                if rc == aes.AES_OK:
                    break
                assert rc == aes.AES_EAGAIN
                assert srv.wait(pending.pop(0), WAIT_US) == aes.AES_OK
            pending.append(t)
            for _ in range(3):  # zero-length requests behind it, reaped at once
                rc, tz = srv.submit_status(ks, ivs[i].tobytes(), src.data_ptr(), dst.data_ptr(), 0)
                if rc == aes.AES_EAGAIN:
                    continue
                assert rc == aes.AES_OK
                assert srv.wait(tz, WAIT_US) == aes.AES_OK
                zeros += 1
        for t in pending:
            assert srv.wait(t, WAIT_US) == aes.AES_OK
        assert zeros > 0
        out = to_host(dst)
        for i in range(n_real):
            o = int(offs[i])
            np.testing.assert_array_equal(out[o: o + size], oracle.ctr_mt(key, 128, ivs[i], payload[o: o + size], ncpu))
    finally:
        assert srv.close() == aes.AES_OK


def test_served_pinned_host_buffers(cuda, aes, ncpu):
    """Served requests whose input and output live in pinned host memory: the
    resident kernel writes the output over NVLink-C2C and orders it at system
    scope before raising the completion flag the host polls."""
    srv = aes.Server(slots=16, max_keys=2, ctas=16, idle_timeout_us=500_000)
    try:
        g = W.rng(67)
        key = W.random_bytes(g, 32)
        ks = srv.key_register(key.tobytes(), 256)
        sizes = [16, 4096 + 3, 1 << 20, (1 << 20) + 1, 2 << 20]
        pad = [(n + 255) // 256 * 256 + 256 for n in sizes]
        offs = np.concatenate([[0], np.cumsum(pad)[:-1]]).astype(np.int64)
        total = int(sum(pad))
        payload = W.random_bytes(g, total)
        hsrc = cuda.from_numpy(payload.copy()).pin_memory()
        hdst = cuda.full((total,), 0xA5, dtype=cuda.uint8).pin_memory()
        ivs = [W.random_bytes(g, 16) for _ in sizes]
        tickets = [srv.submit(ks, ivs[i].tobytes(), hsrc.data_ptr() + int(offs[i]), hdst.data_ptr() + int(offs[i]),
                              n) for i, n in enumerate(sizes)]
        for t in tickets:
            assert srv.wait(t, WAIT_US) == aes.AES_OK
        out = hdst.numpy()  # no device synchronisation: the completion flag orders the output
        for i, n in enumerate(sizes):
            o = int(offs[i])
            np.testing.assert_array_equal(out[o: o + n], oracle.ctr_mt(key, 256, ivs[i], payload[o: o + n], ncpu))
            assert (out[o + n: o + n + 16] == 0xA5).all()
    finally:
        assert srv.close() == aes.AES_OK


def test_poll_many(cuda, aes, ncpu):
    """offload_poll_many reports finished tickets (and releases them) and
    times out with 0 when nothing is done."""
    srv = aes.Server(slots=16, max_keys=2, ctas=16, idle_timeout_us=500_000)
    try:
        g = W.rng(68)
        key = W.random_bytes(g, 16)
        ks = srv.key_register(key.tobytes(), 128)
        sizes = [4096, 1 << 20, 16, 3 << 18]
        payload, offs, src, dst = arena(cuda, g, sizes)
        ivs = [W.random_bytes(g, 16) for _ in sizes]
        pending = {srv.submit(ks, ivs[i].tobytes(), src.data_ptr() + int(offs[i]), dst.data_ptr() + int(offs[i]), n): i
                   for i, n in enumerate(sizes)}
        deadline = time.time() + 10
        while pending and time.time() < deadline:
            tickets = list(pending)
            n, st = srv.poll_many(tickets, 100_000)
            assert n == int((st != aes.AES_PENDING).sum())
            for t, rc in zip(tickets, st.tolist()):
                if rc != aes.AES_PENDING:
                    assert rc == aes.AES_OK
                    assert srv.poll(t) == aes.AES_EINVAL  # released
                    del pending[t]
        assert not pending
        assert srv.poll_many([], 0)[0] == 0
        out = to_host(dst)
        for i, n in enumerate(sizes):
            o = int(offs[i])
            np.testing.assert_array_equal(out[o: o + n], oracle.ctr_mt(key, 128, ivs[i], payload[o: o + n], ncpu))
    finally:
        assert srv.close() == aes.AES_OK


def test_emulated_offload(cuda, aes):
    """An emulated offload takes the whole served path but holds a worker warp
    for its duration instead of encrypting; it moves no bytes."""
    srv = aes.Server(slots=16, max_keys=1, ctas=8, idle_timeout_us=500_000)
    try:
        t0 = time.perf_counter()
        t = srv.submit_emulated(2_000_000)
        assert srv.wait(t, WAIT_US) == aes.AES_OK
        assert time.perf_counter() - t0 >= 0.002
        tickets = [srv.submit_emulated(20_000) for _ in range(12)]
        for t in tickets:
            assert srv.wait(t, WAIT_US) == aes.AES_OK
        st = srv.stats()
        assert st["completed"] == 13 and st["bytes_completed"] == 0
        tk = ctypes.c_uint64(0)
        assert aes.lib().offload_submit_emulated(srv.handle, 20_000_000, ctypes.byref(tk)) == aes.AES_EINVAL
    finally:
        assert srv.close() == aes.AES_OK


@pytest.mark.parametrize("blocking", [True, False])
def test_emulated_open_loop_drivers(cuda, aes, blocking):
    """The blocking and overlapping servers of the load study, over emulated
    20 us offloads: every request completes, none faster than its offload."""
    srv = aes.Server(slots=64, max_keys=1, ctas=16, idle_timeout_us=500_000)
    try:
        n = 600
        reqs = np.zeros(n, dtype=aes.drive_dtype())
        reqs["arrival_s"] = W.poisson_arrivals(n, 30_000.0, seed=69)
        lat, res = aes.drive_served(srv, reqs, 4, blocking=blocking, emulated_ns=20_000)
        assert res["errors"] == 0
        assert (lat >= 20.0).all()
        assert res["bytes"] == 0
    finally:
        assert srv.close() == aes.AES_OK


@pytest.mark.parametrize("budget_gib", [20, 2])
def test_full_size_8mib_aes256_stream_sampled(cuda, aes, ncpu, budget_gib):
    """The 8 MiB AES-256 stream at full size, as the served study runs it:
    2048 requests (16 GiB), at most 512 in flight, an HBM budget of 20 GiB
    and of 2 GiB (back-pressure), a new key every 1024 requests, all offered
    at once through the native driver.  Sampled against the oracle: every
    64th request in full and four 4 KiB windows of every request (a window
    starts at T_1 + offset/16)."""
    MiB = 1 << 20
    n5, big = 2048, 8 * MiB
    gen = cuda.Generator(device="cuda").manual_seed(W.SEED_BASE + 5)
    src = cuda.randint(0, 256, (n5 * big,), dtype=cuda.uint8, device="cuda", generator=gen)
    dst = cuda.full((n5 * big,), 0xA5, dtype=cuda.uint8, device="cuda")
    cuda.cuda.synchronize()  # the served kernel runs on its own stream
    g = W.rng(W.SEED_BASE + 7)
    keys5 = [W.random_bytes(g, 32) for _ in range(n5 // 1024)]
    ivs5 = W.random_bytes(g, 16 * n5).reshape(n5, 16)
    srv = aes.Server(slots=512, max_keys=4, hbm_budget=budget_gib << 30, idle_timeout_us=2_000_000)
    try:
        ks = [srv.key_register(k.tobytes(), 256) for k in keys5]
        r5 = np.zeros(n5, dtype=aes.drive_dtype())
        r5["key_slot"] = np.array(ks)[np.arange(n5) // 1024]
        r5["iv"] = ivs5
        r5["inp"] = src.data_ptr() + np.arange(n5) * big
        r5["out"] = dst.data_ptr() + np.arange(n5) * big
        r5["len"] = big
        lat, res = aes.drive_served(srv, r5, 8)
        assert res["errors"] == 0 and (lat > 0).all()
    finally:
        assert srv.close() == aes.AES_OK
    cuda.cuda.synchronize()
    gw = W.rng(W.SEED_BASE + 8)
    for i in range(n5):
        key = keys5[i // 1024]
        base = i * big
        spans = [(0, big)] if i % 64 == 0 else []
        spans += [(int(o) * 16, int(o) * 16 + 4096) for o in gw.integers(0, (big - 4096) // 16, 4)]
        for a, b in spans:
            want = oracle.ctr_mt(key, 256, iv_plus(ivs5[i], a // 16), src[base + a: base + b].cpu().numpy(), ncpu)
            np.testing.assert_array_equal(dst[base + a: base + b].cpu().numpy(), want,
                                          err_msg=f"request {i} bytes [{a}, {b})")
    del src, dst
    cuda.cuda.empty_cache()


@pytest.mark.parametrize("rate", [100_000.0, None], ids=["poisson_100k", "all_at_once"])
def test_served_open_loop_mix_matches_oracle(cuda, aes, ncpu, rate):
    """The served open-loop workload as the served study offers it -- sizes
    70% 1 MiB, 10% 8 MiB (uncapped), 20% log-uniform 4-64 KiB; 64 registered
    keys, AES-128/256 50/50, one drawn per request; 8 native submitter
    threads, Poisson arrivals or everything at once -- and every byte of every
    request compared with the oracle."""
    import concurrent.futures as cf

    n = 384
    sizes = W.served_sizes(n, seed=W.SEED_BASE + 4)
    kbits, kbytes = W.key_set(64, seed=W.SEED_BASE + 5)
    g = W.rng(W.SEED_BASE + 6)
    key_idx = g.integers(0, 64, n)
    ivs = W.random_bytes(g, 16 * n).reshape(n, 16)
    payload, offs, src, dst = arena(cuda, g, [int(x) for x in sizes])
    srv = aes.Server(slots=1024, max_keys=64, idle_timeout_us=2_000_000)
    try:
        slots = np.array([srv.key_register(kbytes[i, : kbits[i] // 8].tobytes(), int(kbits[i])) for i in range(64)])
        reqs = np.zeros(n, dtype=aes.drive_dtype())
        reqs["key_slot"] = slots[key_idx]
        reqs["iv"] = ivs
        reqs["inp"] = src.data_ptr() + offs
        reqs["out"] = dst.data_ptr() + offs
        reqs["len"] = sizes
        reqs["arrival_s"] = 0.0 if rate is None else W.poisson_arrivals(n, rate, seed=W.SEED_BASE + 44)
        lat, res = aes.drive_served(srv, reqs, 8)
        assert res["errors"] == 0 and res["bytes"] == int(sizes.sum()) and (lat > 0).all()
    finally:
        assert srv.close() == aes.AES_OK
    out = to_host(dst)

    def check(i):
        k = int(key_idx[i])
        o, m = int(offs[i]), int(sizes[i])
        want = oracle.ctr_mt(kbytes[k, : kbits[k] // 8], int(kbits[k]), ivs[i], payload[o: o + m], 2)
        if not np.array_equal(out[o: o + m], want):
            return f"request {i} (len {m}) differs"
        if not (out[o + m: o + m + 16] == 0xA5).all():
            return f"request {i}: bytes past len were written"
        return None

    with cf.ThreadPoolExecutor(max(1, ncpu // 2)) as ex:
        errors = [e for e in ex.map(check, range(n)) if e]
    assert not errors, errors[:5]


@pytest.mark.parametrize("cfg", [dict(threads=64, ctas=2, tile_blocks=64), dict(threads=96, ctas=1, tile_blocks=128),
                                 dict(threads=512, tile_blocks=256), dict()])
def test_server_shapes_match_oracle(cuda, aes, ncpu, cfg):
    """The smallest CTAs (one worker warp), a single CTA, fixed tile sizes and
    the defaults all give the oracle's bytes on a mix of lengths and keys."""
    srv = aes.Server(slots=32, max_keys=4, idle_timeout_us=500_000, **cfg)
    try:
        g = W.rng(73)
        keys = [(W.random_bytes(g, b // 8), b) for b in (128, 256, 192)]
        slots = [srv.key_register(k.tobytes(), b) for k, b in keys]
        sizes = [0, 15, 16, 17, 4096 + 3, 65536, (1 << 20) + 9]
        payload, offs, src, dst = arena(cuda, g, sizes)
        ivs = [W.random_bytes(g, 16) for _ in sizes]
        tickets = [srv.submit(slots[i % 3], ivs[i].tobytes(), src.data_ptr() + int(offs[i]),
                              dst.data_ptr() + int(offs[i]), n) for i, n in enumerate(sizes)]
        for t in tickets:
            assert srv.wait(t, WAIT_US) == aes.AES_OK
        out = to_host(dst)
        for i, n in enumerate(sizes):
            o = int(offs[i])
            key, bits = keys[i % 3]
            np.testing.assert_array_equal(out[o: o + n], oracle.ctr_mt(key, bits, ivs[i], payload[o: o + n], ncpu))
            assert (out[o + n: o + n + 16] == 0xA5).all()
    finally:
        assert srv.close() == aes.AES_OK


@pytest.mark.parametrize("cfg", [{}, {"tile_blocks": 64}, {"tile_blocks": 1024}], ids=["per_request", "t64", "t1024"])
def test_served_counter_carries_match_oracle(cuda, aes, ncpu, cfg):
    """Initial counters 8 blocks below a carry out of the low 32 and 64 bits
    and below the 2^128 wrap: every served request's bytes match the
    oracle's full 128-bit counter (SP 800-38A App. B.1, m = 128)."""
    srv = aes.Server(slots=32, max_keys=2, idle_timeout_us=500_000, **cfg)
    try:
        g = W.rng(69)
        keys = [(W.random_bytes(g, 16), 128), (W.random_bytes(g, 32), 256)]
        slots = [srv.key_register(k.tobytes(), b) for k, b in keys]
        sizes = [100, 129, 4096 + 5, 65536 + 7, (1 << 20) + 9]
        kinds = ["low32", "low64", "wrap128"]
        cases = [(n, kind, j % 2) for j, (n, kind) in enumerate((n, k) for n in sizes for k in kinds)]
        payload, offs, src, dst = arena(cuda, g, [n for n, _, _ in cases])
        tickets = []
        for i, (n, kind, k) in enumerate(cases):
            iv = iv_with_low(g, kind)
            o = int(offs[i])
            t = srv.submit(slots[k], iv.tobytes(), src.data_ptr() + o, dst.data_ptr() + o, n)
            tickets.append((t, iv, o, n, k))
        for t, *_ in tickets:
            assert srv.wait(t, WAIT_US) == aes.AES_OK
        out = to_host(dst)
        for t, iv, o, n, k in tickets:
            key, bits = keys[k]
            np.testing.assert_array_equal(out[o: o + n], oracle.ctr_mt(key, bits, iv, payload[o: o + n], ncpu))
    finally:
        assert srv.close() == aes.AES_OK


def test_served_in_place_matches_oracle(cuda, aes, ncpu):
    """Served requests that encrypt in place (in == out) give the oracle's
    bytes."""
    srv = aes.Server(slots=16, max_keys=1, idle_timeout_us=500_000)
    try:
        g = W.rng(70)
        key = W.random_bytes(g, 32)
        slot = srv.key_register(key.tobytes(), 256)
        sizes = [1, 16, 4096 + 3, (1 << 20) + 5, 3 << 20]
        payload, offs, src, _ = arena(cuda, g, sizes)
        ivs = [W.random_bytes(g, 16) for _ in sizes]
        tickets = [srv.submit(slot, ivs[i].tobytes(), src.data_ptr() + int(offs[i]), src.data_ptr() + int(offs[i]),
                              n) for i, n in enumerate(sizes)]
        for t in tickets:
            assert srv.wait(t, WAIT_US) == aes.AES_OK
        out = to_host(src)
        for i, n in enumerate(sizes):
            o = int(offs[i])
            np.testing.assert_array_equal(out[o: o + n], oracle.ctr_mt(key, 256, ivs[i], payload[o: o + n], ncpu))
    finally:
        assert srv.close() == aes.AES_OK


@pytest.mark.parametrize("bits", [128, 256])
def test_served_every_length_0_to_64(cuda, aes, ncpu, bits):
    """Served requests of every length from 0 to 64 bytes, all in flight
    together; bytes past each length stay untouched."""
    srv = aes.Server(slots=128, max_keys=1, ctas=16, idle_timeout_us=500_000)
    try:
        g = W.rng(71 + bits)
        key = W.random_bytes(g, bits // 8)
        slot = srv.key_register(key.tobytes(), bits)
        sizes = list(range(65))
        payload, offs, src, dst = arena(cuda, g, sizes)
        ivs = [W.random_bytes(g, 16) for _ in sizes]
        tickets = [srv.submit(slot, ivs[i].tobytes(), src.data_ptr() + int(offs[i]), dst.data_ptr() + int(offs[i]),
                              n) for i, n in enumerate(sizes)]
        for t in tickets:
            assert srv.wait(t, WAIT_US) == aes.AES_OK
        out = to_host(dst)
        for i, n in enumerate(sizes):
            o = int(offs[i])
            np.testing.assert_array_equal(out[o: o + n], oracle.ctr(key, bits, ivs[i], payload[o: o + n]),
                                          err_msg=f"len={n}")
            assert (out[o + n: o + n + 16] == 0xA5).all(), f"bytes past len {n} were written"
    finally:
        assert srv.close() == aes.AES_OK


def test_trace_build_stamps(cuda, aes, claim_mode):
    """The trace build (libaesoffload_trace.so, built here) stamps each served
    request's steps, in protocol order.  Run as its own process
    (paper_2607_02630_gb300.served_trace), which loads that library instead
    of the normal one."""
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-m", "paper_2607_02630_gb300.served_trace", "--requests", "40",
                        "--claim-mode", str(claim_mode)],
                       capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stdout + r.stderr
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["ordered"] and res["median_us"]["done"] > 0, res
    assert res["claim_mode"] == claim_mode
