"""Pins of the CPU oracle to facts that do not come from the oracle itself.

Each test checks the oracle (FIPS-197 cipher, SP 800-38A counter mode)
against something independent of its code: a second derivation of the S-box
by another method, the textbook invariants of the S-box and the field, the
round trip through the inverse cipher, an independent AES implementation
(OpenSSL via python-cryptography, where installed), big-integer counter
arithmetic, and the structural invariants of counter mode.  A dropped term,
a wrong index or a transposed operand anywhere in the oracle fails at least
one of them.
"""
import numpy as np
import pytest

from paper_2607_02630_gb300 import workloads

BITS = (128, 192, 256)


# ------------------------------------------------------------ field and S-box

def clmul_reduce(a: int, b: int) -> int:
    """GF(2^8) product by carry-less multiplication followed by polynomial
    long division by m(x) = x^8 + x^4 + x^3 + x + 1 (FIPS-197 Sec. 4.2)."""
    p = 0
    for i in range(8):
        if (b >> i) & 1:
            p ^= a << i
    for deg in range(14, 7, -1):
        if (p >> deg) & 1:
            p ^= 0x11B << (deg - 8)
    return p


def inverse_by_power(x: int) -> int:
    """x^{-1} = x^254 in GF(2^8)* (order 255), by square-and-multiply."""
    result, base, e = 1, x, 254
    while e:
        if e & 1:
            result = clmul_reduce(result, base)
        base = clmul_reduce(base, base)
        e >>= 1
    return result if x else 0


def rotl8(v: int, r: int) -> int:
    return ((v << r) | (v >> (8 - r))) & 0xFF


def sbox_second_derivation() -> np.ndarray:
    """S(x) = A(x^254) + {63}, with the affine map written in its circulant
    form b + rotl(b,1) + rotl(b,2) + rotl(b,3) + rotl(b,4)."""
    out = np.zeros(256, np.uint8)
    for x in range(256):
        b = inverse_by_power(x)
        out[x] = b ^ rotl8(b, 1) ^ rotl8(b, 2) ^ rotl8(b, 3) ^ rotl8(b, 4) ^ 0x63
    return out


def test_gf_mul_matches_clmul_for_all_pairs(oracle_mod):
    for a in range(256):
        row = [oracle_mod.gf_mul(a, b) for b in range(256)]
        assert row == [clmul_reduce(a, b) for b in range(256)], a


def test_gf_mul_field_axioms(oracle_mod):
    g = workloads.rng(11)
    triples = g.integers(0, 256, size=(2000, 3))
    m = oracle_mod.gf_mul
    for a, b, c in triples.tolist():
        assert m(a, b) == m(b, a)
        assert m(m(a, b), c) == m(a, m(b, c))
        assert m(a, b ^ c) == m(a, b) ^ m(a, c)
    for a in range(256):
        assert m(a, 1) == a and m(a, 0) == 0
    # every nonzero element has exactly one inverse
    for a in range(1, 256):
        assert sum(1 for b in range(1, 256) if m(a, b) == 1) == 1


def test_sbox_equals_second_derivation(oracle_mod):
    np.testing.assert_array_equal(oracle_mod.sbox(), sbox_second_derivation())


def test_sbox_textbook_invariants(oracle_mod):
    s = oracle_mod.sbox().astype(int)
    inv = oracle_mod.inv_sbox().astype(int)
    assert sorted(s.tolist()) == list(range(256)), "S-box is a permutation"
    assert all(s[x] != x for x in range(256)), "no fixed points"
    assert all(s[x] != (x ^ 0xFF) for x in range(256)), "no opposite fixed points"
    assert all(inv[s[x]] == x for x in range(256))
    # affine constant: S(0) is the affine image of 0, i.e. the constant {63}
    assert s[0] == 0x63


# ------------------------------------------------------------- block cipher

@pytest.mark.parametrize("bits", BITS)
def test_inv_cipher_round_trip(oracle_mod, bits):
    g = workloads.rng(100 + bits)
    for _ in range(200):
        key = workloads.random_bytes(g, bits // 8)
        block = workloads.random_bytes(g, 16)
        c = oracle_mod.cipher(key, bits, block)
        assert not np.array_equal(c, block)
        np.testing.assert_array_equal(oracle_mod.inv_cipher(key, bits, c), block)


@pytest.mark.parametrize("bits", BITS)
def test_key_expansion_shape_and_prefix(oracle_mod, bits):
    g = workloads.rng(200 + bits)
    key = workloads.random_bytes(g, bits // 8)
    w = oracle_mod.key_expansion(key, bits)
    assert w.size == 16 * (bits // 32 + 7)
    np.testing.assert_array_equal(w[: bits // 8], key)


@pytest.mark.parametrize("bits", BITS)
def test_key_expansion_inverts(oracle_mod, bits):
    """The schedule recurrence is invertible: running w[i-Nk] = w[i] ^ temp(w[i-1])
    backwards from the last Nk words must give back the key.  Uses the S-box
    from the second derivation and Rcon from powers of x computed by clmul."""
    nk = bits // 32
    total = 4 * (nk + 7)
    s = sbox_second_derivation()
    rcon = [0, 1]
    while len(rcon) < 16:
        rcon.append(clmul_reduce(rcon[-1], 2))
    g = workloads.rng(300 + bits)
    key = workloads.random_bytes(g, bits // 8)
    w = oracle_mod.key_expansion(key, bits).reshape(total, 4).astype(int).tolist()
    words = [None] * total
    words[total - nk:] = w[total - nk:]
    for i in range(total - 1, nk - 1, -1):
        prev = words[i - 1] if words[i - 1] is not None else None
        assert prev is not None
        temp = list(prev)
        if i % nk == 0:
            temp = temp[1:] + temp[:1]
            temp = [int(s[t]) for t in temp]
            temp[0] ^= rcon[i // nk]
        elif nk > 6 and i % nk == 4:
            temp = [int(s[t]) for t in temp]
        words[i - nk] = [a ^ b for a, b in zip(words[i], temp)]
    np.testing.assert_array_equal(np.array(words[:nk], np.uint8).ravel(), key)


def _openssl():
    ciphers = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    return ciphers


@pytest.mark.parametrize("bits", BITS)
def test_cipher_matches_independent_library(oracle_mod, bits):
    c = _openssl()
    g = workloads.rng(400 + bits)
    for _ in range(20):
        key = workloads.random_bytes(g, bits // 8)
        blocks = workloads.random_bytes(g, 16 * 64)
        enc = c.Cipher(c.algorithms.AES(key.tobytes()), c.modes.ECB()).encryptor()
        ref = np.frombuffer(enc.update(blocks.tobytes()) + enc.finalize(), np.uint8)
        np.testing.assert_array_equal(oracle_mod.cipher_blocks(key, bits, blocks), ref)


# -------------------------------------------------------------- counter mode

def bigint_counter(iv: np.ndarray, j: int) -> np.ndarray:
    v = (int.from_bytes(iv.tobytes(), "big") + j) % (1 << 128)
    return np.frombuffer(v.to_bytes(16, "big"), np.uint8)


CARRY_IVS = {
    "low32": (1 << 32) - 8,
    "low64": (1 << 64) - 8,
    "wrap128": (1 << 128) - 8,
    "byte": 0xFE,
}


def carry_iv(g, kind):
    iv = workloads.random_bytes(g, 16)
    v = int.from_bytes(iv.tobytes(), "big")
    if kind == "low32":
        v = (v >> 32 << 32) | CARRY_IVS[kind]
    elif kind == "low64":
        v = (v >> 64 << 64) | CARRY_IVS[kind]
    elif kind == "wrap128":
        v = CARRY_IVS[kind]
    elif kind == "byte":
        v = (v >> 8 << 8) | CARRY_IVS[kind]
    return np.frombuffer(v.to_bytes(16, "big"), np.uint8).copy()


@pytest.mark.parametrize("kind", sorted(CARRY_IVS))
def test_counter_add_matches_bigint(oracle_mod, kind):
    g = workloads.rng(500)
    iv = carry_iv(g, kind)
    for j in list(range(0, 40)) + [255, 256, 65535, 1 << 20, (1 << 32) + 5, (1 << 64) - 1]:
        np.testing.assert_array_equal(oracle_mod.counter_add(iv, j), bigint_counter(iv, j))


@pytest.mark.parametrize("bits", (128, 256))
@pytest.mark.parametrize("kind", sorted(CARRY_IVS))
def test_keystream_is_cipher_of_counters(oracle_mod, bits, kind):
    """With P = 0 the output is the keystream O_j = CIPH_K(T_j), T_j = T_1 + j."""
    g = workloads.rng(600 + bits)
    key = workloads.random_bytes(g, bits // 8)
    iv = carry_iv(g, kind)
    nblk = 40
    ks = oracle_mod.ctr(key, bits, iv, np.zeros(16 * nblk, np.uint8))
    counters = np.concatenate([bigint_counter(iv, j) for j in range(nblk)])
    np.testing.assert_array_equal(ks, oracle_mod.cipher_blocks(key, bits, counters))


@pytest.mark.parametrize("bits", BITS)
def test_ctr_brute_force_tiny_lengths_vs_library(oracle_mod, bits):
    c = _openssl()
    g = workloads.rng(700 + bits)
    for n in range(0, 65):
        key = workloads.random_bytes(g, bits // 8)
        iv = workloads.random_bytes(g, 16)
        data = workloads.random_bytes(g, n)
        enc = c.Cipher(c.algorithms.AES(key.tobytes()), c.modes.CTR(iv.tobytes())).encryptor()
        ref = np.frombuffer(enc.update(data.tobytes()) + enc.finalize(), np.uint8)
        np.testing.assert_array_equal(oracle_mod.ctr(key, bits, iv, data), ref)


@pytest.mark.parametrize("bits", (128, 256))
@pytest.mark.parametrize("kind", sorted(CARRY_IVS))
def test_ctr_carry_cases_vs_library(oracle_mod, bits, kind):
    """OpenSSL's CTR increments all 128 counter bits big-endian, which is the
    reading taken for the paper's unspecified counter (SP 800-38A App. B.1,
    m = 128)."""
    c = _openssl()
    g = workloads.rng(800 + bits)
    key = workloads.random_bytes(g, bits // 8)
    iv = carry_iv(g, kind)
    data = workloads.random_bytes(g, 16 * 20 + 7)
    enc = c.Cipher(c.algorithms.AES(key.tobytes()), c.modes.CTR(iv.tobytes())).encryptor()
    ref = np.frombuffer(enc.update(data.tobytes()) + enc.finalize(), np.uint8)
    np.testing.assert_array_equal(oracle_mod.ctr(key, bits, iv, data), ref)


@pytest.mark.parametrize("bits", (128, 256))
def test_ctr_random_lengths_vs_library(oracle_mod, bits):
    c = _openssl()
    g = workloads.rng(900 + bits)
    for _ in range(6):
        n = int(g.integers(1, 300_000))
        key = workloads.random_bytes(g, bits // 8)
        iv = workloads.random_bytes(g, 16)
        data = workloads.random_bytes(g, n)
        enc = c.Cipher(c.algorithms.AES(key.tobytes()), c.modes.CTR(iv.tobytes())).encryptor()
        ref = np.frombuffer(enc.update(data.tobytes()) + enc.finalize(), np.uint8)
        np.testing.assert_array_equal(oracle_mod.ctr(key, bits, iv, data), ref)


@pytest.mark.parametrize("bits", BITS)
def test_ctr_decrypt_equals_encrypt(oracle_mod, bits):
    g = workloads.rng(1000 + bits)
    key = workloads.random_bytes(g, bits // 8)
    iv = workloads.random_bytes(g, 16)
    data = workloads.random_bytes(g, 4099)
    c = oracle_mod.ctr(key, bits, iv, data)
    assert not np.array_equal(c, data)
    np.testing.assert_array_equal(oracle_mod.ctr(key, bits, iv, c), data)


@pytest.mark.parametrize("bits", (128, 256))
def test_ctr_block_independence(oracle_mod, bits):
    """Blocks [a, b) computed alone from T_1 + a equal that slice of the whole."""
    g = workloads.rng(1100 + bits)
    key = workloads.random_bytes(g, bits // 8)
    iv = carry_iv(g, "low32")
    data = workloads.random_bytes(g, 16 * 50 + 9)
    full = oracle_mod.ctr(key, bits, iv, data)
    for a, b in [(0, 1), (3, 17), (7, 9), (8, 50), (49, 51)]:
        lo, hi = 16 * a, min(16 * b, data.size)
        part = oracle_mod.ctr(key, bits, bigint_counter(iv, a), data[lo:hi])
        np.testing.assert_array_equal(part, full[lo:hi])


@pytest.mark.parametrize("nthreads", [1, 2, 3, 5, 8, 13])
def test_ctr_mt_equals_single_thread(oracle_mod, nthreads):
    g = workloads.rng(1200 + nthreads)
    key = workloads.random_bytes(g, 32)
    iv = carry_iv(g, "low32")
    for n in (0, 1, 15, 16, 17, 16 * nthreads + 3, 10_001):
        data = workloads.random_bytes(g, n)
        np.testing.assert_array_equal(oracle_mod.ctr_mt(key, 256, iv, data, nthreads),
                                      oracle_mod.ctr(key, 256, iv, data))


def test_oracle_rejects_bad_key_size(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.ctr(np.zeros(24, np.uint8), 200, np.zeros(16, np.uint8), np.zeros(16, np.uint8))


@pytest.mark.parametrize("n", list(range(0, 49)))
def test_ctr_never_writes_past_len(oracle_mod, n):
    """Bytes of the output buffer after len stay untouched (partial last block
    uses only the first u bytes of O_n, SP 800-38A Sec. 6.5)."""
    g = workloads.rng(1300 + n)
    key = workloads.random_bytes(g, 16)
    iv = workloads.random_bytes(g, 16)
    data = workloads.random_bytes(g, n)
    out = np.full(n + 32, 0xA5, np.uint8)
    oracle_mod.ctr_mt_into(key, 128, iv, data, out, 1)
    assert (out[n:] == 0xA5).all()
    np.testing.assert_array_equal(out[:n], oracle_mod.ctr(key, 128, iv, data))
