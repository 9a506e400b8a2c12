/*
 * aes_oracle.c -- the CPU oracle for the AES-CTR offload.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and
 * the CPU-baseline leg of the benchmark may load this library.  The product
 * path (the CUDA library) never links, loads or calls it, and this file shares
 * no code, header, table or constant generator with it.
 *
 * What it computes.  The paper offloads "AES" on a GPU stream (Sec. 6,
 * experimental setup; App. A, Table 2) without fixing mode or key size.  The
 * reading taken here is AES-128/192/256 (FIPS-197) in counter mode
 * (NIST SP 800-38A, Sec. 6.5), with the whole 16-byte initial counter block
 * T_1 supplied by the caller and the standard incrementing function of
 * SP 800-38A App. B.1 applied to all 128 bits (m = 128): carries propagate
 * through every byte and the counter wraps modulo 2^128.
 *
 * How.  Deliberately plain and byte oriented, in the order and notation of
 * FIPS-197: the S-box is derived from its algebraic definition (multiplicative
 * inverse in GF(2^8) found by exhaustive search, then the affine map of
 * FIPS-197 Sec. 5.1.1); Rcon is built by repeated xtime; the state is the 4x4
 * byte array s[r][c] = in[r + 4c]; every transformation is its own function.
 * No table-driven round, no word packing, no blocking.
 *
 * Parity pins (tests/test_oracle_pins.py): S-box against a second derivation
 * (inverse as x^254 by square-and-multiply) and its textbook invariants;
 * InvCipher(Cipher(x)) = x; Cipher and CTR against an independent library
 * (OpenSSL through python-cryptography, where installed); CTR invariants
 * (decrypt = encrypt, block independence, keystream = Cipher(T_j)); counter
 * sequence against big-integer arithmetic.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <pthread.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)

/* ---------------------------------------------------------------- GF(2^8) */

/* FIPS-197 Sec. 4.2.1: multiplication by x, reduced modulo
 * m(x) = x^8 + x^4 + x^3 + x + 1 (0x11b). */
static uint8_t xtime(uint8_t b)
{
    uint16_t t = (uint16_t)b << 1;
    if (t & 0x100)
        t ^= 0x11b;
    return (uint8_t)t;
}

/* FIPS-197 Sec. 4.2: product of two field elements as repeated xtime and
 * conditional addition (shift-and-add over the bits of b). */
static uint8_t gf_mul(uint8_t a, uint8_t b)
{
    uint8_t acc = 0;
    for (int i = 0; i < 8; ++i) {
        if (b & 1)
            acc ^= a;
        a = xtime(a);
        b >>= 1;
    }
    return acc;
}

/* ------------------------------------------------------------------ S-box */

static uint8_t g_sbox[256];
static uint8_t g_inv_sbox[256];
static pthread_once_t g_once = PTHREAD_ONCE_INIT;

/* FIPS-197 Sec. 5.1.1: S(x) = affine(x^{-1}), with 0 mapped to 0.
 * The inverse is found by trying every y until x*y = 1. */
static void build_tables(void)
{
    for (int x = 0; x < 256; ++x) {
        uint8_t inv = 0;
        if (x != 0) {
            for (int y = 1; y < 256; ++y) {
                if (gf_mul((uint8_t)x, (uint8_t)y) == 1) {
                    inv = (uint8_t)y;
                    break;
                }
            }
        }
        /* b'_i = b_i + b_{(i+4)%8} + b_{(i+5)%8} + b_{(i+6)%8} + b_{(i+7)%8} + c_i,
         * c = {63} */
        uint8_t out = 0;
        for (int i = 0; i < 8; ++i) {
            int bit = ((inv >> i) & 1) ^ ((inv >> ((i + 4) % 8)) & 1) ^
                      ((inv >> ((i + 5) % 8)) & 1) ^ ((inv >> ((i + 6) % 8)) & 1) ^
                      ((inv >> ((i + 7) % 8)) & 1) ^ ((0x63 >> i) & 1);
            out |= (uint8_t)(bit << i);
        }
        g_sbox[x] = out;
    }
    /* FIPS-197 Sec. 5.3.2: InvSubBytes uses the inverse permutation. */
    for (int x = 0; x < 256; ++x)
        g_inv_sbox[g_sbox[x]] = (uint8_t)x;
}

static void ensure_tables(void)
{
    pthread_once(&g_once, build_tables);
}

/* ---------------------------------------------------------- key expansion */

static int nk_from_bits(int bits)
{
    switch (bits) {
    case 128: return 4;
    case 192: return 6;
    case 256: return 8;
    default: return 0;
    }
}

/* FIPS-197 Sec. 5.2.  w holds 4*(Nr+1) words, each as 4 bytes
 * w[i] = (w[4i], w[4i+1], w[4i+2], w[4i+3]). */
static void key_expansion(const uint8_t *key, int nk, uint8_t *w)
{
    int nr = nk + 6;
    int total = 4 * (nr + 1);
    for (int i = 0; i < nk; ++i)
        for (int b = 0; b < 4; ++b)
            w[4 * i + b] = key[4 * i + b];
    uint8_t rc = 1; /* Rcon[1] = x^0; Rcon[j] = xtime(Rcon[j-1]) */
    for (int i = nk; i < total; ++i) {
        uint8_t temp[4];
        for (int b = 0; b < 4; ++b)
            temp[b] = w[4 * (i - 1) + b];
        if (i % nk == 0) {
            /* RotWord: [a0,a1,a2,a3] -> [a1,a2,a3,a0] */
            uint8_t t0 = temp[0];
            temp[0] = temp[1];
            temp[1] = temp[2];
            temp[2] = temp[3];
            temp[3] = t0;
            /* SubWord */
            for (int b = 0; b < 4; ++b)
                temp[b] = g_sbox[temp[b]];
            /* xor Rcon[i/Nk] = [rc, 0, 0, 0] */
            temp[0] ^= rc;
            rc = xtime(rc);
        } else if (nk > 6 && i % nk == 4) {
            for (int b = 0; b < 4; ++b)
                temp[b] = g_sbox[temp[b]];
        }
        for (int b = 0; b < 4; ++b)
            w[4 * i + b] = w[4 * (i - nk) + b] ^ temp[b];
    }
}

/* ------------------------------------------------------------------ cipher */

typedef uint8_t state_t[4][4]; /* s[r][c] */

static void add_round_key(state_t s, const uint8_t *w, int round)
{
    /* FIPS-197 Sec. 5.1.4: column c is xored with word w[round*Nb + c]. */
    for (int c = 0; c < 4; ++c)
        for (int r = 0; r < 4; ++r)
            s[r][c] ^= w[4 * (4 * round + c) + r];
}

static void sub_bytes(state_t s)
{
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c)
            s[r][c] = g_sbox[s[r][c]];
}

static void inv_sub_bytes(state_t s)
{
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c)
            s[r][c] = g_inv_sbox[s[r][c]];
}

/* FIPS-197 Sec. 5.1.2: row r is rotated left by r positions. */
static void shift_rows(state_t s)
{
    for (int r = 1; r < 4; ++r) {
        uint8_t row[4];
        for (int c = 0; c < 4; ++c)
            row[c] = s[r][(c + r) % 4];
        for (int c = 0; c < 4; ++c)
            s[r][c] = row[c];
    }
}

/* FIPS-197 Sec. 5.3.1: row r is rotated right by r positions. */
static void inv_shift_rows(state_t s)
{
    for (int r = 1; r < 4; ++r) {
        uint8_t row[4];
        for (int c = 0; c < 4; ++c)
            row[(c + r) % 4] = s[r][c];
        for (int c = 0; c < 4; ++c)
            s[r][c] = row[c];
    }
}

/* Multiply each column by the fixed matrix m (a circulant of a(x) or
 * a^{-1}(x) modulo x^4 + 1). */
static void mix_with(state_t s, const uint8_t m[4][4])
{
    for (int c = 0; c < 4; ++c) {
        uint8_t col[4];
        for (int r = 0; r < 4; ++r)
            col[r] = s[r][c];
        for (int r = 0; r < 4; ++r) {
            uint8_t acc = 0;
            for (int k = 0; k < 4; ++k)
                acc ^= gf_mul(m[r][k], col[k]);
            s[r][c] = acc;
        }
    }
}

/* FIPS-197 Sec. 5.1.3: a(x) = {03}x^3 + {01}x^2 + {01}x + {02}. */
static const uint8_t k_mix[4][4] = {
    {2, 3, 1, 1}, {1, 2, 3, 1}, {1, 1, 2, 3}, {3, 1, 1, 2}};
/* FIPS-197 Sec. 5.3.3: a^{-1}(x) = {0b}x^3 + {0d}x^2 + {09}x + {0e}. */
static const uint8_t k_inv_mix[4][4] = {
    {0x0e, 0x0b, 0x0d, 0x09}, {0x09, 0x0e, 0x0b, 0x0d},
    {0x0d, 0x09, 0x0e, 0x0b}, {0x0b, 0x0d, 0x09, 0x0e}};

/* FIPS-197 Sec. 5.1, Cipher(). */
static void cipher(const uint8_t in[16], uint8_t out[16], const uint8_t *w, int nr)
{
    state_t s;
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c)
            s[r][c] = in[r + 4 * c];
    add_round_key(s, w, 0);
    for (int round = 1; round < nr; ++round) {
        sub_bytes(s);
        shift_rows(s);
        mix_with(s, k_mix);
        add_round_key(s, w, round);
    }
    sub_bytes(s);
    shift_rows(s);
    add_round_key(s, w, nr);
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c)
            out[r + 4 * c] = s[r][c];
}

/* FIPS-197 Sec. 5.3, InvCipher(). */
static void inv_cipher(const uint8_t in[16], uint8_t out[16], const uint8_t *w, int nr)
{
    state_t s;
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c)
            s[r][c] = in[r + 4 * c];
    add_round_key(s, w, nr);
    for (int round = nr - 1; round >= 1; --round) {
        inv_shift_rows(s);
        inv_sub_bytes(s);
        add_round_key(s, w, round);
        mix_with(s, k_inv_mix);
    }
    inv_shift_rows(s);
    inv_sub_bytes(s);
    add_round_key(s, w, 0);
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c)
            out[r + 4 * c] = s[r][c];
}

/* --------------------------------------------------------------- counters */

/* SP 800-38A App. B.1 with m = 128: T <- T + 1 mod 2^128, the 16 bytes read
 * as one big-endian integer. */
static void counter_increment(uint8_t t[16])
{
    for (int i = 15; i >= 0; --i) {
        t[i] = (uint8_t)(t[i] + 1);
        if (t[i] != 0)
            break;
    }
}

/* T <- T + j mod 2^128 (big-endian), byte by byte with carry. */
static void counter_add(uint8_t t[16], uint64_t j)
{
    unsigned carry = 0;
    for (int i = 15; i >= 0; --i) {
        unsigned add = (unsigned)(j & 0xff);
        j >>= 8;
        unsigned sum = (unsigned)t[i] + add + carry;
        t[i] = (uint8_t)sum;
        carry = sum >> 8;
    }
}

/* SP 800-38A Sec. 6.5 for blocks [first, first + nblocks) of a message:
 * O_j = CIPH_K(T_j), C_j = P_j xor O_j; the last partial block uses the
 * first u bytes of O_n. */
static void ctr_range(const uint8_t *w, int nr, const uint8_t iv[16], const uint8_t *in,
                      uint8_t *out, size_t len, uint64_t first, uint64_t nblocks)
{
    uint8_t t[16];
    memcpy(t, iv, 16);
    counter_add(t, first);
    for (uint64_t j = first; j < first + nblocks; ++j) {
        uint8_t o[16];
        cipher(t, o, w, nr);
        size_t off = (size_t)j * 16;
        size_t u = len - off < 16 ? len - off : 16;
        for (size_t b = 0; b < u; ++b)
            out[off + b] = in[off + b] ^ o[b];
        counter_increment(t);
    }
}

/* ------------------------------------------------------------- public API */

int oracle_sbox(uint8_t out[256])
{
    ensure_tables();
    memcpy(out, g_sbox, 256);
    return ORACLE_OK;
}

int oracle_inv_sbox(uint8_t out[256])
{
    ensure_tables();
    memcpy(out, g_inv_sbox, 256);
    return ORACLE_OK;
}

int oracle_gf_mul(int a, int b)
{
    return gf_mul((uint8_t)a, (uint8_t)b);
}

/* w receives 16*(Nr+1) bytes: 176 / 208 / 240 for 128 / 192 / 256 bits. */
int oracle_key_expansion(const uint8_t *key, int bits, uint8_t *w)
{
    int nk = nk_from_bits(bits);
    if (!nk || !key || !w)
        return ORACLE_EINVAL;
    ensure_tables();
    key_expansion(key, nk, w);
    return ORACLE_OK;
}

int oracle_cipher(const uint8_t *key, int bits, const uint8_t in[16], uint8_t out[16])
{
    uint8_t w[240];
    int nk = nk_from_bits(bits);
    if (!nk || !key || !in || !out)
        return ORACLE_EINVAL;
    ensure_tables();
    key_expansion(key, nk, w);
    cipher(in, out, w, nk + 6);
    return ORACLE_OK;
}

int oracle_inv_cipher(const uint8_t *key, int bits, const uint8_t in[16], uint8_t out[16])
{
    uint8_t w[240];
    int nk = nk_from_bits(bits);
    if (!nk || !key || !in || !out)
        return ORACLE_EINVAL;
    ensure_tables();
    key_expansion(key, nk, w);
    inv_cipher(in, out, w, nk + 6);
    return ORACLE_OK;
}

/* Many blocks under one key: in/out hold n*16 bytes (ECB-style application
 * of Cipher, used only to pin the keystream). */
int oracle_cipher_blocks(const uint8_t *key, int bits, const uint8_t *in, uint8_t *out, size_t n)
{
    uint8_t w[240];
    int nk = nk_from_bits(bits);
    if (!nk || !key || (n && (!in || !out)))
        return ORACLE_EINVAL;
    ensure_tables();
    key_expansion(key, nk, w);
    for (size_t i = 0; i < n; ++i)
        cipher(in + 16 * i, out + 16 * i, w, nk + 6);
    return ORACLE_OK;
}

/* T_1 + j mod 2^128 into out. */
int oracle_counter_add(const uint8_t iv[16], uint64_t j, uint8_t out[16])
{
    if (!iv || !out)
        return ORACLE_EINVAL;
    memcpy(out, iv, 16);
    counter_add(out, j);
    return ORACLE_OK;
}

/* One message, sequentially from T_1 = iv (SP 800-38A Sec. 6.5). */
int oracle_ctr(const uint8_t *key, int bits, const uint8_t iv[16], const uint8_t *in, uint8_t *out,
               size_t len)
{
    uint8_t w[240];
    int nk = nk_from_bits(bits);
    if (!nk || !key || !iv || (len && (!in || !out)))
        return ORACLE_EINVAL;
    ensure_tables();
    key_expansion(key, nk, w);
    ctr_range(w, nk + 6, iv, in, out, len, 0, (len + 15) / 16);
    return ORACLE_OK;
}

struct mt_job {
    const uint8_t *w;
    int nr;
    const uint8_t *iv;
    const uint8_t *in;
    uint8_t *out;
    size_t len;
    uint64_t first, count;
};

static void *mt_worker(void *arg)
{
    struct mt_job *j = (struct mt_job *)arg;
    if (j->count)
        ctr_range(j->w, j->nr, j->iv, j->in, j->out, j->len, j->first, j->count);
    return NULL;
}

/* The same result as oracle_ctr, with the block range split into nthreads
 * contiguous pieces; piece t starts from T_1 + first_t.  Used to time the
 * oracle on all host cores. */
int oracle_ctr_mt(const uint8_t *key, int bits, const uint8_t iv[16], const uint8_t *in,
                  uint8_t *out, size_t len, int nthreads)
{
    uint8_t w[240];
    int nk = nk_from_bits(bits);
    if (!nk || !key || !iv || (len && (!in || !out)) || nthreads < 1 || nthreads > 1024)
        return ORACLE_EINVAL;
    ensure_tables();
    key_expansion(key, nk, w);
    uint64_t nblocks = (len + 15) / 16;
    pthread_t tid[1024];
    int spawned[1024];
    struct mt_job jobs[1024];
    uint64_t per = (nblocks + (uint64_t)nthreads - 1) / (uint64_t)nthreads;
    for (int t = 0; t < nthreads; ++t) {
        uint64_t first = per * (uint64_t)t;
        uint64_t count = first >= nblocks ? 0 : (nblocks - first < per ? nblocks - first : per);
        jobs[t] = (struct mt_job){w, nk + 6, iv, in, out, len, first, count};
        spawned[t] = pthread_create(&tid[t], NULL, mt_worker, &jobs[t]) == 0;
        if (!spawned[t])
            mt_worker(&jobs[t]); /* no thread available: do the piece here */
    }
    for (int t = 0; t < nthreads; ++t)
        if (spawned[t])
            pthread_join(tid[t], NULL);
    return ORACLE_OK;
}
