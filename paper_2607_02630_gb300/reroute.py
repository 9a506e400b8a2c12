"""Offload rerouting on a single-event-loop server (the block-size sweep).

The paper's recipe reroutes an offload through a server's own concurrency:
submit it to a background executor, suspend the request with the server's
deferred-response primitive, and resume it when the offload completes
(Sec. 3).  Its block-size sweep drives one Python asyncio server with a
32-thread executor at 50 concurrent clients and reports, per AES block size
from 4 KiB to 8 MiB, the single-op GPU latency and the synchronous and
asynchronous throughput (App. A, Table 2).  This module reproduces that shape
on the library's entry points:

* ``sync``: the request handler calls the blocking offload on the
  event-loop thread (``aes_ctr_sync``: launch, then poll its completion
  event), so the loop serves nobody else meanwhile;
* ``executor``: the paper's recipe -- the handler hands the blocking call to
  a thread pool (``run_in_executor``), suspends on the future and is resumed
  when a pool thread finishes;
* ``served``: the same suspend/resume, with the library's served path as the
  executor -- the handler calls ``offload_submit`` (returns at once), suspends
  on a future, and one completion thread waiting in ``offload_poll_many``
  resumes it.

Clients are a separate process of 50 asyncio connections, each sending one
request and waiting for its reply before the next (closed loop) over
127.0.0.1 TCP.  Every request encrypts the connection's own block (resident
in HBM) with the connection's key and IV.
"""
from __future__ import annotations

import asyncio
import concurrent.futures
import multiprocessing as mp
import struct
import threading
import time

REQ = struct.Struct("<Q")


# ------------------------------------------------------------------ backends

class PerCallOffload:
    """Blocking offload: ``aes_ctr_sync`` (launch on the calling thread's
    stream, then poll the completion event; the GIL is released for the
    whole call).  One stream per calling thread."""

    def __init__(self, aes, torch, device, ctx_of, bufs):
        self.aes = aes
        self.torch = torch
        self.device = device
        self.ctx_of = ctx_of  # connection -> (Context, iv bytes)
        self.bufs = bufs      # connection -> (in ptr, out ptr)
        self.local = threading.local()

    def _stream(self):
        s = getattr(self.local, "stream", None)
        if s is None:
            self.torch.cuda.set_device(self.device)
            s = self.local.stream = self.torch.cuda.Stream(device=self.device)
        return s

    def run_blocking(self, conn: int, nbytes: int):
        ctx, iv = self.ctx_of(conn)
        src, dst = self.bufs(conn)
        self.aes.ctr_sync(ctx, iv, src, dst, nbytes, stream=self._stream())


class ServedOffload:
    """Non-blocking offload through the served path: submit returns a ticket
    at once; one completion thread waits on all outstanding tickets with
    ``offload_poll_many`` (GIL released while it waits) and resumes the
    suspended handlers on their event loop."""

    def __init__(self, aes, server, key_slot_of, bufs, poll_timeout_us: int = 200):
        self.aes = aes
        self.server = server
        self.key_slot_of = key_slot_of  # connection -> (key slot, iv bytes)
        self.bufs = bufs
        self.poll_timeout_us = poll_timeout_us
        self.pending = {}
        self.lock = threading.Lock()
        self.wake = threading.Event()
        self.stopping = False
        self.thread = threading.Thread(target=self._completions, daemon=True)
        self.thread.start()

    def submit(self, loop, conn: int, nbytes: int) -> asyncio.Future:
        slot, iv = self.key_slot_of(conn)
        src, dst = self.bufs(conn)
        fut = loop.create_future()
        while True:
            rc, ticket = self.server.submit_status(slot, iv, src, dst, nbytes)
            if rc == self.aes.AES_OK:
                break
            if rc != self.aes.AES_EAGAIN:
                raise self.aes.AesError(rc, "offload_submit")
            time.sleep(0)  # back-pressure: let the completion thread free a slot
        with self.lock:
            self.pending[ticket] = (loop, fut)
        self.wake.set()
        return fut

    def _completions(self):
        pend = self.aes.AES_PENDING
        while not self.stopping:
            self.wake.clear()
            with self.lock:
                tickets = list(self.pending)
            if not tickets:
                self.wake.wait(0.01)
                continue
            n, status = self.server.poll_many(tickets, self.poll_timeout_us)
            if n == 0:
                continue
            for ticket, rc in zip(tickets, status.tolist()):
                if rc == pend:
                    continue
                with self.lock:
                    loop, fut = self.pending.pop(ticket)
                if rc == self.aes.AES_OK:
                    loop.call_soon_threadsafe(_resolve, fut, None)
                else:
                    loop.call_soon_threadsafe(_fail, fut, self.aes.AesError(rc, "offload_poll"))

    def close(self):
        self.stopping = True
        self.wake.set()
        self.thread.join(timeout=5)


def _resolve(fut, value):
    if not fut.done():
        fut.set_result(value)


def _fail(fut, exc):
    if not fut.done():
        fut.set_exception(exc)


# -------------------------------------------------------------------- server

class RerouteServer:
    """Single-event-loop TCP server; mode in {"sync", "executor", "served"}.

    ``offload`` is a PerCallOffload (sync, executor) or a ServedOffload
    (served); any object with the same methods works, which is how the
    harness logic is tested without a GPU."""

    def __init__(self, mode: str, offload, nbytes: int, executor_threads: int = 32):
        if mode not in ("sync", "executor", "served"):
            raise ValueError(mode)
        self.mode = mode
        self.offload = offload
        self.nbytes = nbytes
        self.pool = concurrent.futures.ThreadPoolExecutor(executor_threads) if mode == "executor" else None
        self.conns = 0
        self.served = 0

    async def handle(self, reader: asyncio.StreamReader, writer: asyncio.StreamWriter):
        conn = self.conns
        self.conns += 1
        loop = asyncio.get_running_loop()
        try:
            while True:
                try:
                    msg = await reader.readexactly(REQ.size)
                except asyncio.IncompleteReadError:
                    break
                if self.mode == "sync":
                    self.offload.run_blocking(conn, self.nbytes)      # the loop waits here
                elif self.mode == "executor":
                    await loop.run_in_executor(self.pool, self.offload.run_blocking, conn, self.nbytes)
                else:
                    await self.offload.submit(loop, conn, self.nbytes)  # submit, suspend, resume
                self.served += 1
                writer.write(msg)
                await writer.drain()
        finally:
            writer.close()

    def close(self):
        if self.pool:
            self.pool.shutdown(wait=True)


# ------------------------------------------------------------------- clients

async def _clients(port: int, nclients: int, seconds: float, warmup: float):
    conns = []
    for _ in range(nclients):
        conns.append(await asyncio.open_connection("127.0.0.1", port))
    counts = [0] * nclients
    t0 = time.perf_counter()
    t_start, t_end = t0 + warmup, t0 + warmup + seconds

    async def one(i, reader, writer):
        k = 0
        while True:
            now = time.perf_counter()
            if now >= t_end:
                break
            writer.write(REQ.pack(k))
            await writer.drain()
            got = await reader.readexactly(REQ.size)
            if REQ.unpack(got)[0] != k:
                raise RuntimeError("reply out of order")
            if time.perf_counter() >= t_start and now >= t_start:
                counts[i] += 1
            k += 1

    await asyncio.gather(*(one(i, r, w) for i, (r, w) in enumerate(conns)))
    for _, w in conns:
        w.close()
    return sum(counts) / seconds


def _client_proc(port, nclients, seconds, warmup, out):
    try:
        out.put(("ok", asyncio.run(_clients(port, nclients, seconds, warmup))))
    except Exception as e:  # reported to the parent
        out.put(("error", repr(e)))


def drive(server: RerouteServer, nclients: int = 50, seconds: float = 2.0, warmup: float = 0.5) -> float:
    """Run the server on this thread's event loop, load it from a client
    process (spawned) with `nclients` closed-loop connections, and return the
    completed requests per second over `seconds` after `warmup`."""
    ctx = mp.get_context("spawn")
    out = ctx.Queue()

    async def main():
        srv = await asyncio.start_server(server.handle, "127.0.0.1", 0)
        port = srv.sockets[0].getsockname()[1]
        proc = ctx.Process(target=_client_proc, args=(port, nclients, seconds, warmup, out))
        proc.start()
        loop = asyncio.get_running_loop()
        result = await loop.run_in_executor(None, out.get, True, 120 + seconds + warmup)
        await loop.run_in_executor(None, proc.join, 30)
        srv.close()
        await srv.wait_closed()
        return result

    status, value = asyncio.run(main())
    if status != "ok":
        raise RuntimeError(f"client process failed: {value}")
    return value


# --------------------------------------------------------------- one block size

def single_op_latency_us(aes, ctx, iv, src, dst, nbytes: int, stream, reps: int = 200) -> float:
    """Median host time of one blocking offload (aes_ctr_sync), one in flight:
    the 'single-op GPU latency' column of the block-size sweep."""
    for _ in range(10):
        aes.ctr_sync(ctx, iv, src, dst, nbytes, stream=stream)
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        aes.ctr_sync(ctx, iv, src, dst, nbytes, stream=stream)
        ts.append(time.perf_counter() - t0)
    ts.sort()
    return ts[len(ts) // 2] * 1e6


def run_point(aes, torch, device, nbytes: int, server, key: bytes, bits: int = 128, nclients: int = 50,
              seconds: float = 2.0, warmup: float = 0.5, executor_threads: int = 32,
              modes=("sync", "executor", "served"), seed: int = 0) -> dict:
    """One row of the block-size sweep: every client connection owns an
    `nbytes` input block (random) and output block in HBM and its own IV;
    each mode serves the same requests.  `server` is an open aes.Server (the
    served mode registers `key` on it).  Returns requests/s per mode, the
    single-op latency, and whether every mode produced the same ciphertext."""
    gen = torch.Generator(device=device).manual_seed(seed)
    src = torch.randint(0, 256, (nclients, nbytes), dtype=torch.uint8, device=device, generator=gen)
    ivs = [bytes((seed + 31 * i + j) & 255 for j in range(16)) for i in range(nclients)]
    ctx = aes.Context(key, bits)
    outs = {}
    row = {"block_bytes": nbytes, "clients": nclients, "executor_threads": executor_threads}
    stream = torch.cuda.Stream(device=device)
    probe_dst = torch.empty(nbytes, dtype=torch.uint8, device=device)
    # the offloads run on streams of their own: wait for torch's initialisation
    torch.cuda.synchronize(device)
    row["single_op_us"] = round(single_op_latency_us(aes, ctx, ivs[0], src[0].data_ptr(), probe_dst.data_ptr(),
                                                     nbytes, stream), 2)
    slot = server.key_register(key, bits) if "served" in modes else None
    for mode in modes:
        dst = torch.zeros((nclients, nbytes), dtype=torch.uint8, device=device)
        torch.cuda.synchronize(device)

        def bufs(conn, dst=dst):
            return src[conn].data_ptr(), dst[conn].data_ptr()

        if mode == "served":
            off = ServedOffload(aes, server, lambda c: (slot, ivs[c]), bufs)
        else:
            off = PerCallOffload(aes, torch, device, lambda c: (ctx, ivs[c]), bufs)
        srv = RerouteServer(mode, off, nbytes, executor_threads)
        try:
            row[f"{mode}_rps"] = round(drive(srv, nclients, seconds, warmup), 1)
        finally:
            srv.close()
            if mode == "served":
                off.close()
        torch.cuda.synchronize(device)
        outs[mode] = dst
    first = outs[modes[0]]
    row["modes_agree"] = all(bool(torch.equal(first, o)) for o in outs.values())
    if "sync" in modes:
        for mode in modes:
            if mode != "sync":
                row[f"{mode}_speedup"] = round(row[f"{mode}_rps"] / max(row["sync_rps"], 1e-9), 2)
    row["_outputs"] = (src, outs, ivs)
    return row
