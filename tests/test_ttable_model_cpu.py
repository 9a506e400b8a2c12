"""A CPU model of the method the GPU kernels use -- T-table rounds on
little-endian column words with counter-mode caching of rounds 1-2 -- checked
against the oracle.  It pins the derivation, not the kernel code: that the
256 counters of a group share round-1 columns 1..3 and all but one lookup of
each round-2 column, so that a block needs 5 lookups for rounds 1-2 on top of
27 per group (the group constants), and that the final round's S-box bytes
can be read from the T-table entries.  The model derives its own tables from
GF(2^8) arithmetic; only the key schedule and the expected keystream come from
the oracle."""
import numpy as np
import pytest

import oracle
from paper_2607_02630_gb300 import workloads as W


def xtime(a):
    a <<= 1
    return (a ^ 0x11B) if a & 0x100 else a


def gmul(a, b):
    r = 0
    while b:
        if b & 1:
            r ^= a
        a = xtime(a)
        b >>= 1
    return r


def sbox():
    # inverse by exhaustive search, then the affine map (x -> x ^ rotl1..4 ^ 0x63)
    out = []
    for x in range(256):
        inv = next((y for y in range(1, 256) if gmul(x, y) == 1), 0)
        s = inv
        for k in range(1, 5):
            s ^= ((inv << k) | (inv >> (8 - k))) & 0xFF
        out.append(s ^ 0x63)
    return out


S = sbox()
TE0 = [gmul(s, 2) | s << 8 | s << 16 | gmul(s, 3) << 24 for s in S]


def rotl(w, r):
    return ((w << r) | (w >> (32 - r))) & 0xFFFFFFFF if r else w


TE = [[rotl(v, 8 * t) for v in TE0] for t in range(4)]


def byte(w, k):
    return (w >> (8 * k)) & 0xFF


def words(block16):
    return [int.from_bytes(bytes(block16[4 * c: 4 * c + 4]), "little") for c in range(4)]


def full_round(s, k):
    return [TE[0][byte(s[c], 0)] ^ TE[1][byte(s[(c + 1) % 4], 1)] ^ TE[2][byte(s[(c + 2) % 4], 2)]
            ^ TE[3][byte(s[(c + 3) % 4], 3)] ^ k[c] for c in range(4)]


def final_round(s, k):
    # byte r of output column c is S(byte r of column c + r), read from the
    # T-table byte that holds the plain S-box value: Te2 b0, Te3 b1, Te0 b2, Te1 b3
    src = [(2, 0), (3, 1), (0, 2), (1, 3)]
    out = []
    for c in range(4):
        w = 0
        for r in range(4):
            t, bpos = src[r]
            w |= byte(TE[t][byte(s[(c + r) % 4], r)], bpos) << (8 * r)
        out.append(w ^ k[c])
    return out


def keystream_cached(key, bits, iv, nblocks):
    nr = bits // 32 + 6
    w = oracle.key_expansion(key, bits)  # FIPS-197 Sec. 5.2 schedule, bytes
    rk = [words(w[16 * r: 16 * r + 16]) for r in range(nr + 1)]
    t1 = int.from_bytes(bytes(iv), "big")
    out = bytearray()
    group = None
    for j in range(nblocks):
        ctr = (t1 + j) % (1 << 128)
        g, L = ctr >> 8, ctr & 0xFF
        if g != group:  # the group's constants: 27 lookups
            group = g
            base = words((g << 8).to_bytes(16, "big"))
            s = [base[c] ^ rk[0][c] for c in range(4)]
            k15 = rk[0][3] >> 24
            k1, k2 = rk[1], rk[2]
            p0 = TE[0][byte(s[0], 0)] ^ TE[1][byte(s[1], 1)] ^ TE[2][byte(s[2], 2)] ^ k1[0]
            c1, c2, c3 = full_round(s, k1)[1:]
            q0 = TE[1][byte(c1, 1)] ^ TE[2][byte(c2, 2)] ^ TE[3][byte(c3, 3)] ^ k2[0]
            q1 = TE[0][byte(c1, 0)] ^ TE[1][byte(c2, 1)] ^ TE[2][byte(c3, 2)] ^ k2[1]
            q2 = TE[0][byte(c2, 0)] ^ TE[1][byte(c3, 1)] ^ TE[3][byte(c1, 3)] ^ k2[2]
            q3 = TE[0][byte(c3, 0)] ^ TE[2][byte(c1, 2)] ^ TE[3][byte(c2, 3)] ^ k2[3]
        # per block: 5 lookups for rounds 1-2
        r10 = p0 ^ TE[3][L ^ k15]
        st = [q0 ^ TE[0][byte(r10, 0)], q1 ^ TE[3][byte(r10, 3)], q2 ^ TE[2][byte(r10, 2)],
              q3 ^ TE[1][byte(r10, 1)]]
        for r in range(3, nr):
            st = full_round(st, rk[r])
        st = final_round(st, rk[nr])
        out += b"".join(x.to_bytes(4, "little") for x in st)
    return np.frombuffer(bytes(out), np.uint8)


def test_model_sbox_is_the_oracles():
    assert S == [int(x) for x in oracle.sbox()]


@pytest.mark.parametrize("bits", [128, 192, 256])
@pytest.mark.parametrize("low", [0x00, 0x01, 0xF0, 0xFF])
def test_counter_cached_ttable_keystream_matches_oracle(bits, low):
    g = W.rng(90 + bits + low)
    key = W.random_bytes(g, bits // 8)
    iv = W.random_bytes(g, 16).copy()
    iv[15] = low
    if low == 0xFF:
        iv[8:15] = 0xFF  # the group change carries through eight bytes
    n = 300  # crosses at least one counter-group boundary
    want = oracle.ctr(key, bits, iv, np.zeros(16 * n, np.uint8))
    np.testing.assert_array_equal(keystream_cached(key, bits, iv, n), want)


def test_lookup_count_per_block_and_group():
    # rounds 1-2 cost 5 lookups per block + 27 per group instead of 32 per block
    group_lookups = 3 + 4 + 4 + 4 + 3 * 4  # p0, c1..c3, q0..q3
    assert group_lookups == 27
    for nr in (10, 12, 14):
        per_block = 5 + 16 * (nr - 2)
        assert per_block == 16 * nr - 27
