"""Helpers shared by the GPU parity tests (device buffers, oracle calls)."""
import json

import numpy as np


def to_dev(torch, a: np.ndarray, pad: int = 0):
    """uint8 device tensor holding `a` (plus `pad` trailing bytes of 0xA5)."""
    t = torch.full((a.size + pad,), 0xA5, dtype=torch.uint8, device="cuda")
    if a.size:
        t[: a.size].copy_(torch.from_numpy(np.ascontiguousarray(a)))
    return t


def to_host(t) -> np.ndarray:
    return t.cpu().numpy()


def iv_plus(iv: np.ndarray, j: int) -> np.ndarray:
    v = (int.from_bytes(iv.tobytes(), "big") + j) % (1 << 128)
    return np.frombuffer(v.to_bytes(16, "big"), np.uint8).copy()


def iv_with_low(g, kind: str) -> np.ndarray:
    """Random IV whose low bits sit just below a carry boundary."""
    iv = np.frombuffer(g.bytes(16), np.uint8).copy()
    v = int.from_bytes(iv.tobytes(), "big")
    if kind == "low32":
        v = (v >> 32 << 32) | ((1 << 32) - 8)
    elif kind == "low64":
        v = (v >> 64 << 64) | ((1 << 64) - 8)
    elif kind == "wrap128":
        v = (1 << 128) - 8
    elif kind == "random":
        pass
    else:
        raise ValueError(kind)
    return np.frombuffer(v.to_bytes(16, "big"), np.uint8).copy()


def set_batch_shape(torch, aes, path, shape):
    """Make `shape` = (variant, threads, tile_blocks, blocks_per_thread) the
    device's tuned batch shape by loading a table file (aes_autotune_load)
    written for this device; returns the shape that was in place before."""
    before = aes.batch_tuned_shape()
    props = torch.cuda.get_device_properties(0)
    head = json.dumps({"device": props.name, "sms": props.multi_processor_count}).rstrip("}")
    # one ctr row (bucket 0, the default shape) -- the loader wants at least one
    path.write_text(head + ', "ctr": [\n  [0, 0, 1, 256, 1]\n],\n"batch": [%d, %d, %d, %d]}\n' % tuple(shape))
    aes.autotune_load(str(path))
    got = aes.batch_tuned_shape()
    assert (got["variant"], got["threads"], got["tile_blocks"], got["blocks_per_thread"]) == tuple(shape), got
    return (before["variant"], before["threads"], before["tile_blocks"], before["blocks_per_thread"])
