"""CPU oracle for AES-CTR (FIPS-197 cipher, SP 800-38A counter mode).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
under ``paper_2607_02630_gb300`` never imports this package, and this package
never imports it.

The arithmetic lives in ``aes_oracle.c`` (plain C, byte oriented, written in
the order of FIPS-197 Sec. 5.1-5.3 and SP 800-38A Sec. 6.5); this module only
compiles it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aes_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_aes.so")
_lock = threading.Lock()
_lib = None

KEY_BITS = (128, 192, 256)


def build(force: bool = False) -> str:
    """Compile aes_oracle.c into liboracle_aes.so next to it (gcc, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC]
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u8p = ctypes.c_void_p
            lib.oracle_sbox.argtypes = [u8p]
            lib.oracle_inv_sbox.argtypes = [u8p]
            lib.oracle_gf_mul.argtypes = [ctypes.c_int, ctypes.c_int]
            lib.oracle_key_expansion.argtypes = [u8p, ctypes.c_int, u8p]
            lib.oracle_cipher.argtypes = [u8p, ctypes.c_int, u8p, u8p]
            lib.oracle_inv_cipher.argtypes = [u8p, ctypes.c_int, u8p, u8p]
            lib.oracle_cipher_blocks.argtypes = [u8p, ctypes.c_int, u8p, u8p, ctypes.c_size_t]
            lib.oracle_counter_add.argtypes = [u8p, ctypes.c_uint64, u8p]
            lib.oracle_ctr.argtypes = [u8p, ctypes.c_int, u8p, u8p, u8p, ctypes.c_size_t]
            lib.oracle_ctr_mt.argtypes = [u8p, ctypes.c_int, u8p, u8p, u8p, ctypes.c_size_t,
                                          ctypes.c_int]
            _lib = lib
    return _lib


def _buf(a, n=None) -> np.ndarray:
    if isinstance(a, (bytes, bytearray, memoryview)):
        a = np.frombuffer(bytes(a), dtype=np.uint8)
    a = np.ascontiguousarray(a, dtype=np.uint8)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} bytes, got {a.size}")
    return a


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else None


def _check(rc: int) -> None:
    if rc != 0:
        raise ValueError(f"oracle call failed with status {rc}")


def nr_for_bits(bits: int) -> int:
    """FIPS-197 Sec. 5 (Fig. 4): Nr = Nk + 6 with Nk = bits / 32."""
    return bits // 32 + 6


def sbox() -> np.ndarray:
    out = np.zeros(256, np.uint8)
    _check(_load().oracle_sbox(_ptr(out)))
    return out


def inv_sbox() -> np.ndarray:
    out = np.zeros(256, np.uint8)
    _check(_load().oracle_inv_sbox(_ptr(out)))
    return out


def gf_mul(a: int, b: int) -> int:
    return int(_load().oracle_gf_mul(a, b))


def key_expansion(key, bits: int) -> np.ndarray:
    """FIPS-197 Sec. 5.2: the 4*(Nr+1) round-key words as 16*(Nr+1) bytes."""
    k = _buf(key, bits // 8)
    w = np.zeros(16 * (nr_for_bits(bits) + 1), np.uint8)
    _check(_load().oracle_key_expansion(_ptr(k), bits, _ptr(w)))
    return w


def cipher(key, bits: int, block) -> np.ndarray:
    k, b = _buf(key, bits // 8), _buf(block, 16)
    out = np.zeros(16, np.uint8)
    _check(_load().oracle_cipher(_ptr(k), bits, _ptr(b), _ptr(out)))
    return out


def inv_cipher(key, bits: int, block) -> np.ndarray:
    k, b = _buf(key, bits // 8), _buf(block, 16)
    out = np.zeros(16, np.uint8)
    _check(_load().oracle_inv_cipher(_ptr(k), bits, _ptr(b), _ptr(out)))
    return out


def cipher_blocks(key, bits: int, blocks) -> np.ndarray:
    k, b = _buf(key, bits // 8), _buf(blocks)
    if b.size % 16:
        raise ValueError("blocks must be a multiple of 16 bytes")
    out = np.zeros_like(b)
    _check(_load().oracle_cipher_blocks(_ptr(k), bits, _ptr(b), _ptr(out), b.size // 16))
    return out


def counter_add(iv, j: int) -> np.ndarray:
    """T_1 + j mod 2^128 (big-endian), j < 2^64."""
    v = _buf(iv, 16)
    out = np.zeros(16, np.uint8)
    _check(_load().oracle_counter_add(_ptr(v), ctypes.c_uint64(j), _ptr(out)))
    return out


def ctr(key, bits: int, iv, data) -> np.ndarray:
    """SP 800-38A Sec. 6.5 counter mode from T_1 = iv; encryption = decryption."""
    k, v, d = _buf(key, bits // 8), _buf(iv, 16), _buf(data)
    out = np.zeros_like(d)
    _check(_load().oracle_ctr(_ptr(k), bits, _ptr(v), _ptr(d), _ptr(out), d.size))
    return out


def ctr_mt(key, bits: int, iv, data, nthreads: int) -> np.ndarray:
    """ctr() with the block range split over nthreads host threads."""
    k, v, d = _buf(key, bits // 8), _buf(iv, 16), _buf(data)
    out = np.zeros_like(d)
    _check(_load().oracle_ctr_mt(_ptr(k), bits, _ptr(v), _ptr(d), _ptr(out), d.size,
                                 int(nthreads)))
    return out


def ctr_mt_into(key, bits: int, iv, data: np.ndarray, out: np.ndarray, nthreads: int) -> None:
    """ctr_mt() writing into a caller-provided uint8 array (no allocation)."""
    k, v = _buf(key, bits // 8), _buf(iv, 16)
    if data.dtype != np.uint8 or out.dtype != np.uint8 or out.size < data.size:
        raise ValueError("data/out must be uint8 and out at least as long as data")
    if not (data.flags.c_contiguous and out.flags.c_contiguous):
        raise ValueError("data/out must be contiguous")
    _check(_load().oracle_ctr_mt(_ptr(k), bits, _ptr(v), _ptr(data), _ptr(out), data.size,
                                 int(nthreads)))
