"""Python binding of libaesoffload.so (ctypes; argument marshalling only).

Every computation happens in the library's CUDA kernels.  PyTorch is used
only to hand over device pointers (``tensor.data_ptr()``) and streams
(``torch.cuda.Stream.cuda_stream``); plain integers work as well.  If the
library has not been built the first call raises -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

# status codes (include/aesoffload.h)
AES_OK = 0
AES_PENDING = 1
AES_EINVAL = -1
AES_EKEYBITS = -2
AES_EALIGN = -3
AES_EOVERLAP = -4
AES_EAGAIN = -5
AES_ETIMEOUT = -6
AES_ECUDA = -7
AES_ESTOPPED = -8
AES_ENOMEM = -9
AES_ETOOBIG = -10
AES_EPTR = -11
AES_EDESC = -12

VARIANT_AUTO = 0
VARIANT_TTABLE = 1
VARIANT_BITSLICE = 2

_lock = threading.Lock()
_lib = None
_lib_path = None  # set by use_trace_build() before the first call


class AesError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = code
        msg = strerror(code)
        extra = last_error()
        super().__init__(f"{where}: {msg}" + (f" ({extra})" if extra and code == AES_ECUDA else ""))


class LaunchShape(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("threads", ctypes.c_int),
                ("blocks_per_thread", ctypes.c_int), ("ctas", ctypes.c_int)]


class Desc(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("iv", ctypes.c_uint8 * 16), ("inp", ctypes.c_void_p),
                ("out", ctypes.c_void_p), ("len", ctypes.c_size_t)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("threads", ctypes.c_int), ("tile_blocks", ctypes.c_int),
                ("ctas", ctypes.c_int), ("tile_order_seed", ctypes.c_uint32), ("blocks_per_thread", ctypes.c_int)]


class Peaks(ctypes.Structure):
    _fields_ = [("sms", ctypes.c_int), ("lds32_per_clk_sm", ctypes.c_double), ("lop3_per_clk_sm", ctypes.c_double),
                ("prmt_per_clk_sm", ctypes.c_double), ("iadd_per_clk_sm", ctypes.c_double),
                ("sm_mhz_during_probe", ctypes.c_double), ("h2d_gbs", ctypes.c_double), ("d2h_gbs", ctypes.c_double),
                ("h2d_d2h_each_way_gbs", ctypes.c_double), ("zero_copy_each_way_gbs", ctypes.c_double)]


class ServerCfg(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int), ("max_keys", ctypes.c_int), ("hbm_budget", ctypes.c_uint64),
                ("ctas", ctypes.c_int), ("threads", ctypes.c_int), ("tile_blocks", ctypes.c_int),
                ("idle_timeout_us", ctypes.c_uint32), ("claim_mode", ctypes.c_int),
                ("trace_requests", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("rejected_eagain", ctypes.c_uint64), ("device_errors", ctypes.c_uint64),
                ("relaunches", ctypes.c_uint64), ("bytes_completed", ctypes.c_uint64),
                ("kernel_status", ctypes.c_uint32), ("running", ctypes.c_int)]


class CdetCfg(ctypes.Structure):
    _fields_ = [("handlers", ctypes.c_int), ("requests", ctypes.c_int), ("counters", ctypes.c_int),
                ("counters_per_page", ctypes.c_int), ("mode", ctypes.c_int), ("offload_ns", ctypes.c_uint64),
                ("srv", ctypes.c_void_p), ("key_slot", ctypes.c_int), ("buf_in", ctypes.c_void_p),
                ("buf_out", ctypes.c_void_p), ("bytes", ctypes.c_size_t), ("pattern", ctypes.c_int),
                ("store_mode", ctypes.c_int)]


class CdetResult(ctypes.Structure):
    _fields_ = [("final_count", ctypes.c_uint64), ("lost_updates", ctypes.c_uint64), ("conflicts", ctypes.c_uint64),
                ("restarts", ctypes.c_uint64), ("elapsed_s", ctypes.c_double),
                ("emulated_stores", ctypes.c_uint64), ("protect_calls", ctypes.c_uint64)]


CDET_UNPROTECTED, CDET_LOCK, CDET_DETECT, CDET_ENFORCE = 0, 1, 2, 3
CDET_PATTERN_SHARED, CDET_PATTERN_READONLY, CDET_PATTERN_PER_CONN, CDET_PATTERN_LOCKED = 0, 1, 2, 3
CDET_STORES_EMULATE, CDET_STORES_UNPROTECT = 0, 1


class DriveOpts(ctypes.Structure):
    _fields_ = [("blocking", ctypes.c_int), ("emulated_ns", ctypes.c_uint64)]


class DriveResult(ctypes.Structure):
    _fields_ = [("elapsed_s", ctypes.c_double), ("bytes", ctypes.c_uint64),
                ("eagain_retries", ctypes.c_uint64), ("errors", ctypes.c_int)]


_SIGS = {
    "aes_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "aes_last_error": (ctypes.c_char_p, []),
    "aes_version": (ctypes.c_int, []),
    "aes_ctx_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_int]),
    "aes_ctx_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "aes_ctx_bits": (ctypes.c_int, [ctypes.c_void_p]),
    "aes_ctx_round_keys": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "aes_ctr": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_size_t, ctypes.c_void_p]),
    "aes_ctr_sync": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_size_t, ctypes.c_void_p]),
    "aes_ctr_ex": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_size_t, ctypes.c_void_p, ctypes.POINTER(LaunchShape)]),
    "aes_ctr_batch": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_int, ctypes.c_void_p]),
    "aes_ctr_batch_ex": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_int, ctypes.c_void_p,
                                        ctypes.POINTER(BatchOpts)]),
    "aes_batch_plan_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Desc),
                                             ctypes.c_int, ctypes.POINTER(BatchOpts)]),
    "aes_batch_plan_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "aes_batch_plan_bytes": (ctypes.c_int64, [ctypes.c_void_p]),
    "aes_batch_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "aes_autotune": (ctypes.c_int, [ctypes.c_char_p]),
    "aes_autotune_load": (ctypes.c_int, [ctypes.c_char_p]),
    "aes_tuned_shape": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(LaunchShape)]),
    "aes_batch_autotune": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_int, ctypes.c_void_p,
                                          ctypes.POINTER(BatchOpts)]),
    "aes_batch_tuned_shape": (ctypes.c_int, [ctypes.POINTER(BatchOpts)]),
    "aes_measure_peaks": (ctypes.c_int, [ctypes.POINTER(Peaks)]),
    "aes_batch_tune_results": (ctypes.c_int, [ctypes.POINTER(BatchOpts), ctypes.POINTER(ctypes.c_float),
                                              ctypes.c_int]),
    "aes_ctr_batch_noalloc": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_int, ctypes.c_void_p]),
    "offload_server_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ServerCfg)]),
    "offload_key_register": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_int)]),
    "offload_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_uint64)]),
    "offload_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "offload_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64]),
    "offload_poll_many": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.c_uint64]),
    "offload_server_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ServerStats)]),
    "offload_server_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "offload_submit_emulated": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]),
    "offload_drive_ex": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(DriveOpts), ctypes.c_void_p, ctypes.POINTER(DriveResult)]),
    "cdet_run": (ctypes.c_int, [ctypes.POINTER(CdetCfg), ctypes.POINTER(CdetResult)]),
    "offload_server_trace": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64), ctypes.c_size_t]),
    "cdet_store_selftest": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_uint64),
                                           ctypes.POINTER(ctypes.c_uint64)]),
    "offload_drive": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.POINTER(DriveResult)]),
    "aes_ctr_drive": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(DriveResult)]),
}


def library_path() -> str:
    return _lib_path or _build.LIB


def use_trace_build() -> str:
    """Load libaesoffload_trace.so (the served kernel with per-request timer
    stamps compiled in; see Server.trace) instead of libaesoffload.so.  Call
    before anything else uses the library in this process; builds it if
    needed."""
    global _lib_path
    with _lock:
        if _lib is not None and _lib_path != _build.LIB_TRACE:
            raise RuntimeError("the library is already loaded; choose the trace build first")
        _lib_path = _build.build_trace()
    return _lib_path


def lib():
    """The loaded library; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                path = _lib_path or _build.LIB
                if not os.path.exists(path):
                    raise RuntimeError(
                        f"{os.path.basename(path)} is not built; run paper_2607_02630_gb300.build.build() "
                        "(needs nvcc) -- there is no CPU fallback")
                L = ctypes.CDLL(path)
                for name, (res, args) in _SIGS.items():
                    f = getattr(L, name, None)
                    if f is None:
                        continue
                    f.restype = res
                    f.argtypes = args
                _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().aes_strerror(code).decode()


def last_error() -> str:
    return lib().aes_last_error().decode()


def _check(rc: int, where: str) -> int:
    if rc < 0:
        raise AesError(rc, where)
    return rc


def ptr(x) -> int:
    """Device address of a torch tensor, or an int passed through."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def stream_handle(s) -> int:
    if s is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def _iv_bytes(iv) -> bytes:
    """The 16-byte initial counter block as bytes.  Passed by pointer: the
    library copies it before the call returns, so no ctypes copy is made."""
    b = iv if type(iv) is bytes else bytes(iv) if isinstance(iv, bytearray) else memoryview(iv).tobytes()
    if len(b) != 16:
        raise ValueError("iv must be 16 bytes")
    return b


def _bytes16(iv) -> ctypes.Array:
    """The initial counter block as a uint8[16] (descriptor fields)."""
    return (ctypes.c_uint8 * 16).from_buffer_copy(_iv_bytes(iv))


def _keybuf(key, bits: int) -> bytes:
    """The key's bytes; the library reads bits / 8 of them, so a shorter key
    is refused here (a key size the library rejects is passed through)."""
    kb = bytes(bytearray(key if isinstance(key, (bytes, bytearray)) else memoryview(key).tobytes()))
    if int(bits) in (128, 192, 256) and len(kb) < int(bits) // 8:
        raise ValueError(f"a {bits}-bit key needs {int(bits) // 8} bytes, got {len(kb)}")
    return kb


class Context:
    """A device-resident AES key schedule (aes_ctx_create)."""

    def __init__(self, key, bits: int):
        kb = _keybuf(key, bits)
        h = ctypes.c_void_p()
        buf = ctypes.create_string_buffer(kb, max(len(kb), 1))
        _check(lib().aes_ctx_create(ctypes.byref(h), buf, int(bits)), "aes_ctx_create")
        self.handle = h.value
        self.bits = int(bits)

    def round_keys(self) -> bytes:
        out = ctypes.create_string_buffer(240)
        n = _check(lib().aes_ctx_round_keys(self.handle, out, 240), "aes_ctx_round_keys")
        return out.raw[:n]

    def close(self):
        if getattr(self, "handle", None):
            lib().aes_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ctr_status(ctx: Context, iv, src, dst, nbytes: int, stream=None, variant: int = 0,
               threads: int = 0, blocks_per_thread: int = 0, ctas: int = 0) -> int:
    """aes_ctr_ex returning the raw status code."""
    h = ctx.handle if ctx else None
    if not (variant or threads or blocks_per_thread or ctas):  # the tuned shape: no options struct
        return lib().aes_ctr(h, _iv_bytes(iv), ptr(src), ptr(dst), int(nbytes), stream_handle(stream))
    shape = LaunchShape(variant, threads, blocks_per_thread, ctas)
    return lib().aes_ctr_ex(h, _iv_bytes(iv), ptr(src), ptr(dst), int(nbytes), stream_handle(stream),
                            ctypes.byref(shape))


def ctr(ctx: Context, iv, src, dst, nbytes: int | None = None, stream=None, **shape) -> None:
    """dst[:n] = src[:n] xor AES-CTR keystream (asynchronous on `stream`)."""
    if nbytes is None:
        nbytes = src.numel() * src.element_size()
    _check(ctr_status(ctx, iv, src, dst, nbytes, stream, **shape), "aes_ctr")


def ctr_sync(ctx: Context, iv, src, dst, nbytes: int, stream=None) -> None:
    """The blocking offload call: aes_ctr, then poll its completion event
    (aes_ctr_sync; the GIL is released for the whole call)."""
    _check(lib().aes_ctr_sync(ctx.handle, _iv_bytes(iv), ptr(src), ptr(dst), int(nbytes), stream_handle(stream)),
           "aes_ctr_sync")


def _descs(requests):
    arr = (Desc * max(len(requests), 1))()
    for i, (ctx, iv, src, dst, n) in enumerate(requests):
        arr[i].ctx = ctx.handle
        arr[i].iv = _bytes16(iv)
        arr[i].inp = ptr(src)
        arr[i].out = ptr(dst)
        arr[i].len = int(n)
    return arr


def batch_status(requests, stream=None, variant=0, threads=0, tile_blocks=0, ctas=0,
                 tile_order_seed=0, blocks_per_thread=0) -> int:
    arr = _descs(requests)
    opts = BatchOpts(variant, threads, tile_blocks, ctas, tile_order_seed, blocks_per_thread)
    return lib().aes_ctr_batch_ex(arr, len(requests), stream_handle(stream), ctypes.byref(opts))


def batch_noalloc_status(requests, stream=None) -> int:
    """aes_ctr_batch_noalloc (no device allocation; at most 1024 requests)."""
    arr = _descs(requests)
    return lib().aes_ctr_batch_noalloc(arr, len(requests), stream_handle(stream))


def batch(requests, stream=None, **opts) -> None:
    """One persistent launch over requests = [(ctx, iv, src, dst, nbytes), ...]."""
    _check(batch_status(requests, stream, **opts), "aes_ctr_batch")


class BatchPlan:
    """aes_batch_plan_*: a device-resident descriptor table + captured CUDA graph."""

    def __init__(self, requests, variant=0, threads=0, tile_blocks=0, ctas=0, tile_order_seed=0,
                 blocks_per_thread=0):
        arr = _descs(requests)
        opts = BatchOpts(variant, threads, tile_blocks, ctas, tile_order_seed, blocks_per_thread)
        h = ctypes.c_void_p()
        _check(lib().aes_batch_plan_create(ctypes.byref(h), arr, len(requests), ctypes.byref(opts)),
               "aes_batch_plan_create")
        self.handle = h.value

    @property
    def nbytes(self) -> int:
        return int(lib().aes_batch_plan_bytes(self.handle))

    def launch(self, stream=None) -> None:
        _check(lib().aes_batch_plan_launch(self.handle, stream_handle(stream)), "aes_batch_plan_launch")

    def close(self):
        if getattr(self, "handle", None):
            lib().aes_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(path: str | None = None) -> None:
    _check(lib().aes_autotune(path.encode() if path else None), "aes_autotune")


def autotune_load(path: str) -> None:
    _check(lib().aes_autotune_load(path.encode()), "aes_autotune_load")


def _batch_opts_dict(o: BatchOpts) -> dict:
    return {"variant": o.variant, "threads": o.threads, "tile_blocks": o.tile_blocks, "ctas": o.ctas,
            "blocks_per_thread": o.blocks_per_thread}


def batch_autotune(requests, stream=None) -> dict:
    """aes_batch_autotune: time every batch shape on these requests (their
    outputs are overwritten) and make the fastest the device's batch shape."""
    arr = _descs(requests)
    best = BatchOpts()
    _check(lib().aes_batch_autotune(arr, len(requests), stream_handle(stream), ctypes.byref(best)),
           "aes_batch_autotune")
    return _batch_opts_dict(best)


def batch_tune_results() -> list:
    """The last batch-shape sweep: [(shape dict, median ms), ...]."""
    shapes = (BatchOpts * 64)()
    ms = (ctypes.c_float * 64)()
    n = _check(lib().aes_batch_tune_results(shapes, ms, 64), "aes_batch_tune_results")
    return [(_batch_opts_dict(shapes[i]), float(ms[i])) for i in range(n)]


def batch_tuned_shape() -> dict:
    o = BatchOpts()
    _check(lib().aes_batch_tuned_shape(ctypes.byref(o)), "aes_batch_tuned_shape")
    return _batch_opts_dict(o)


def measure_peaks() -> dict:
    """aes_measure_peaks: per-SM issue rates and host-link bandwidths."""
    p = Peaks()
    _check(lib().aes_measure_peaks(ctypes.byref(p)), "aes_measure_peaks")
    return {name: getattr(p, name) for name, _ in Peaks._fields_}


def tuned_shape(nbytes: int, bits: int) -> dict:
    s = LaunchShape()
    _check(lib().aes_tuned_shape(int(nbytes), int(bits), ctypes.byref(s)), "aes_tuned_shape")
    return {"variant": s.variant, "threads": s.threads, "blocks_per_thread": s.blocks_per_thread,
            "ctas": s.ctas}


class Server:
    """Served mode: a resident kernel polling mapped descriptors (offload_*)."""

    def __init__(self, slots=0, max_keys=0, hbm_budget=0, ctas=0, threads=0, tile_blocks=0,
                 idle_timeout_us=0, claim_mode=0, trace_requests=0):
        cfg = ServerCfg(slots, max_keys, hbm_budget, ctas, threads, tile_blocks, idle_timeout_us, claim_mode,
                        trace_requests)
        self.trace_requests = int(trace_requests)
        h = ctypes.c_void_p()
        _check(lib().offload_server_create(ctypes.byref(h), ctypes.byref(cfg)), "offload_server_create")
        self.handle = h.value

    def key_register(self, key, bits: int) -> int:
        slot = ctypes.c_int(-1)
        kb = _keybuf(key, bits)
        buf = ctypes.create_string_buffer(kb, max(len(kb), 1))
        _check(lib().offload_key_register(self.handle, buf, int(bits), ctypes.byref(slot)),
               "offload_key_register")
        return slot.value

    def submit_status(self, key_slot: int, iv, src, dst, nbytes: int):
        t = ctypes.c_uint64(0)
        rc = lib().offload_submit(self.handle, int(key_slot), _iv_bytes(iv), ptr(src), ptr(dst),
                                  int(nbytes), ctypes.byref(t))
        return rc, t.value

    def submit(self, key_slot: int, iv, src, dst, nbytes: int) -> int:
        rc, t = self.submit_status(key_slot, iv, src, dst, nbytes)
        _check(rc, "offload_submit")
        return t

    def submit_emulated(self, duration_ns: int) -> int:
        """offload_submit_emulated: an emulated offload holding one worker warp
        for duration_ns; returns its ticket."""
        t = ctypes.c_uint64(0)
        _check(lib().offload_submit_emulated(self.handle, int(duration_ns), ctypes.byref(t)),
               "offload_submit_emulated")
        return t.value

    def poll(self, ticket: int) -> int:
        return lib().offload_poll(self.handle, ctypes.c_uint64(ticket))

    def poll_many(self, tickets, timeout_us: int = 1000):
        """offload_poll_many over a sequence of tickets: (number done, status
        per ticket); the GIL is released while it waits."""
        import numpy as np

        t = np.ascontiguousarray(np.asarray(tickets, dtype=np.uint64))
        st = np.empty(t.size, dtype=np.int32)
        rc = lib().offload_poll_many(self.handle, t.ctypes.data, int(t.size), st.ctypes.data, int(timeout_us))
        if rc < 0:
            raise AesError(rc, "offload_poll_many")
        return rc, st

    def wait(self, ticket: int, timeout_us: int = 5_000_000) -> int:
        return lib().offload_wait(self.handle, ctypes.c_uint64(ticket), ctypes.c_uint64(timeout_us))

    TRACE_POINTS = ("dispatched", "published", "first_claim", "first_pop", "record_loaded", "keys_loaded",
                    "first_tile_done", "done")

    def trace(self):
        """Trace builds: the stamp buffer as a uint64 array [trace_requests,
        8] (ns; 0 = not reached); row s % trace_requests is request s
        (sequence numbers count submits from 1)."""
        import numpy as np

        n = self.trace_requests * len(self.TRACE_POINTS)
        out = np.zeros(n, dtype=np.uint64)
        _check(lib().offload_server_trace(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), n),
               "offload_server_trace")
        return out.reshape(self.trace_requests, len(self.TRACE_POINTS))

    def stats(self) -> dict:
        s = ServerStats()
        _check(lib().offload_server_stats(self.handle, ctypes.byref(s)), "offload_server_stats")
        return {f: getattr(s, f) for f, _ in ServerStats._fields_}

    def close(self) -> int:
        rc = 0
        if getattr(self, "handle", None):
            rc = lib().offload_server_destroy(self.handle)
            self.handle = None
        return rc

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# aes_drive_req_t as a numpy record (C layout: int, 16 bytes, pad, 3 x 8-byte fields, double)
def drive_dtype():
    import numpy as np

    return np.dtype({"names": ["key_slot", "iv", "inp", "out", "len", "arrival_s"],
                     "formats": ["<i4", ("u1", 16), "<u8", "<u8", "<u8", "<f8"],
                     "offsets": [0, 4, 24, 32, 40, 48], "itemsize": 56})


def _drive_result(res: DriveResult) -> dict:
    return {"elapsed_s": res.elapsed_s, "bytes": res.bytes, "eagain_retries": res.eagain_retries,
            "errors": res.errors}


def drive_served(server: "Server", reqs, nthreads: int = 8, blocking: bool = False, emulated_ns: int = 0):
    """offload_drive_ex over a drive_dtype() array; returns (latency_us array,
    result dict).  blocking: each thread waits for its offload before the
    next request; emulated_ns > 0: emulated offloads of that duration."""
    import numpy as np

    reqs = np.ascontiguousarray(reqs, dtype=drive_dtype())
    lat = np.zeros(len(reqs), np.float64)
    res = DriveResult()
    opts = DriveOpts(1 if blocking else 0, int(emulated_ns))
    _check(lib().offload_drive_ex(server.handle, reqs.ctypes.data, len(reqs), int(nthreads), ctypes.byref(opts),
                                  lat.ctypes.data, ctypes.byref(res)), "offload_drive_ex")
    return lat, _drive_result(res)


def drive_per_call(ctxs, reqs, nthreads: int = 8):
    """aes_ctr_drive with key_slot indexing `ctxs`; returns (latency_us array, result dict)."""
    import numpy as np

    reqs = np.ascontiguousarray(reqs, dtype=drive_dtype())
    handles = (ctypes.c_void_p * len(ctxs))(*[c.handle for c in ctxs])
    lat = np.zeros(len(reqs), np.float64)
    res = DriveResult()
    _check(lib().aes_ctr_drive(handles, len(ctxs), reqs.ctypes.data, len(reqs), int(nthreads),
                               lat.ctypes.data, ctypes.byref(res)), "aes_ctr_drive")
    return lat, _drive_result(res)


def conflict_run(mode: int, handlers: int = 16, requests: int = 4000, counters: int = 64, counters_per_page: int = 1,
                 offload_ns: int = 50_000, server: "Server | None" = None, key_slot: int = 0, buf_in=0, buf_out=0,
                 nbytes: int = 0, pattern: int = 0, emulate_stores: bool = True) -> dict:
    """cdet_run: the conflict detector's synthetic server (read a shared
    counter, park at an offload, write it back incremented) in one of the
    CDET_* modes, with the shared state in one of the CDET_PATTERN_*
    patterns; returns the result as a dict (requests/s added).
    emulate_stores: CDET_STORES_EMULATE (the default) or, if False,
    CDET_STORES_UNPROTECT."""
    cfg = CdetCfg(int(handlers), int(requests), int(counters), int(counters_per_page), int(mode), int(offload_ns),
                  server.handle if server else None, int(key_slot), ptr(buf_in) or None, ptr(buf_out) or None,
                  int(nbytes), int(pattern), CDET_STORES_EMULATE if emulate_stores else CDET_STORES_UNPROTECT)
    res = CdetResult()
    _check(lib().cdet_run(ctypes.byref(cfg), ctypes.byref(res)), "cdet_run")
    out = {f: getattr(res, f) for f, _ in CdetResult._fields_}
    out["req_per_s"] = requests / res.elapsed_s if res.elapsed_s > 0 else 0.0
    return out


def store_selftest(rounds: int = 6000) -> dict:
    """cdet_store_selftest: guarded stores of every width on this CPU,
    performed by the detector's fault handler where it decodes them; raises
    if the region does not match its shadow copy."""
    emulated, fallbacks = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().cdet_store_selftest(int(rounds), ctypes.byref(emulated), ctypes.byref(fallbacks)),
           "cdet_store_selftest")
    return {"emulated": emulated.value, "fallbacks": fallbacks.value}
