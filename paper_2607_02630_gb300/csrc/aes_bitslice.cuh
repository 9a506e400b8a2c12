// aes_bitslice.cuh -- bitsliced AES round functions (32 blocks per thread).
//
// Representation: a thread holds the states of 32 blocks as 128 "planes".
// Plane 8*i + b is a 32-bit word whose bit k is bit b (b = 0 the least
// significant) of byte i of block k, with byte i of the state at row i % 4,
// column i / 4 (the FIPS-197 Sec. 3.4 input-to-state mapping).  ShiftRows is
// then a renaming of planes, AddRoundKey an xor with all-zeros / all-ones
// masks, and SubBytes and MixColumns boolean circuits on planes.
//
// SubBytes uses the depth-16, 113-gate circuit of Boyar and Peralta
// ("A depth-16 circuit for the AES S-box", 2012): a linear top layer, a
// shared nonlinear middle layer (32 ANDs) and a linear bottom layer.
// Variable names follow the paper (U: input bits, MSB first; T, M, L
// intermediates; S: output bits, MSB first).  Xor chains are left to the
// compiler, which fuses them into three-input LOP3s.
#pragma once
#include <stdint.h>

#ifndef AES_HD
#define AES_HD __device__ __forceinline__
#endif

namespace aesbs {

// Forward S-box on one bitsliced byte.  x[b] holds bit b (LSB = 0).
AES_HD void sbox(uint32_t x[8])
{
    const uint32_t U0 = x[7], U1 = x[6], U2 = x[5], U3 = x[4];
    const uint32_t U4 = x[3], U5 = x[2], U6 = x[1], U7 = x[0];
    // top linear layer
    const uint32_t T1 = U0 ^ U3, T2 = U0 ^ U5, T3 = U0 ^ U6, T4 = U3 ^ U5;
    const uint32_t T5 = U4 ^ U6, T6 = T1 ^ T5, T7 = U1 ^ U2, T8 = U7 ^ T6;
    const uint32_t T9 = U7 ^ T7, T10 = T6 ^ T7, T11 = U1 ^ U5, T12 = U2 ^ U5;
    const uint32_t T13 = T3 ^ T4, T14 = T6 ^ T11, T15 = T5 ^ T11, T16 = T5 ^ T12;
    const uint32_t T17 = T9 ^ T16, T18 = U3 ^ U7, T19 = T7 ^ T18, T20 = T1 ^ T19;
    const uint32_t T21 = U6 ^ U7, T22 = T7 ^ T21, T23 = T2 ^ T22, T24 = T2 ^ T10;
    const uint32_t T25 = T20 ^ T17, T26 = T3 ^ T16, T27 = T1 ^ T12;
    // nonlinear middle layer
    const uint32_t M1 = T13 & T6, M2 = T23 & T8, M3 = T14 ^ M1, M4 = T19 & U7;
    const uint32_t M5 = M4 ^ M1, M6 = T3 & T16, M7 = T22 & T9, M8 = T26 ^ M6;
    const uint32_t M9 = T20 & T17, M10 = M9 ^ M6, M11 = T1 & T15, M12 = T4 & T27;
    const uint32_t M13 = M12 ^ M11, M14 = T2 & T10, M15 = M14 ^ M11, M16 = M3 ^ M2;
    const uint32_t M17 = M5 ^ T24, M18 = M8 ^ M7, M19 = M10 ^ M15, M20 = M16 ^ M13;
    const uint32_t M21 = M17 ^ M15, M22 = M18 ^ M13, M23 = M19 ^ T25, M24 = M22 ^ M23;
    const uint32_t M25 = M22 & M20, M26 = M21 ^ M25, M27 = M20 ^ M21, M28 = M23 ^ M25;
    const uint32_t M29 = M28 & M27, M30 = M26 & M24, M31 = M20 & M23, M32 = M27 & M31;
    const uint32_t M33 = M27 ^ M25, M34 = M21 & M22, M35 = M24 & M34, M36 = M24 ^ M25;
    const uint32_t M37 = M21 ^ M29, M38 = M32 ^ M33, M39 = M23 ^ M30, M40 = M35 ^ M36;
    const uint32_t M41 = M38 ^ M40, M42 = M37 ^ M39, M43 = M37 ^ M38, M44 = M39 ^ M40;
    const uint32_t M45 = M42 ^ M41;
    const uint32_t M46 = M44 & T6, M47 = M40 & T8, M48 = M39 & U7, M49 = M43 & T16;
    const uint32_t M50 = M38 & T9, M51 = M37 & T17, M52 = M42 & T15, M53 = M45 & T27;
    const uint32_t M54 = M41 & T10, M55 = M44 & T13, M56 = M40 & T23, M57 = M39 & T19;
    const uint32_t M58 = M43 & T3, M59 = M38 & T22, M60 = M37 & T20, M61 = M42 & T1;
    const uint32_t M62 = M45 & T4, M63 = M41 & T2;
    // bottom linear layer
    const uint32_t L0 = M61 ^ M62, L1 = M50 ^ M56, L2 = M46 ^ M48, L3 = M47 ^ M55;
    const uint32_t L4 = M54 ^ M58, L5 = M49 ^ M61, L6 = M62 ^ L5, L7 = M46 ^ L3;
    const uint32_t L8 = M51 ^ M59, L9 = M52 ^ M53, L10 = M53 ^ L4, L11 = M60 ^ L2;
    const uint32_t L12 = M48 ^ M51, L13 = M50 ^ L0, L14 = M52 ^ M61, L15 = M55 ^ L1;
    const uint32_t L16 = M56 ^ L0, L17 = M57 ^ L1, L18 = M58 ^ L8, L19 = M63 ^ L4;
    const uint32_t L20 = L0 ^ L1, L21 = L1 ^ L7, L22 = L3 ^ L12, L23 = L18 ^ L2;
    const uint32_t L24 = L15 ^ L9, L25 = L6 ^ L10, L26 = L7 ^ L9, L27 = L8 ^ L10;
    const uint32_t L28 = L11 ^ L14, L29 = L11 ^ L17;
    x[7] = L6 ^ L24;          // S0
    x[6] = ~(L16 ^ L26);      // S1
    x[5] = ~(L19 ^ L28);      // S2
    x[4] = L6 ^ L21;          // S3
    x[3] = L20 ^ L22;         // S4
    x[2] = L25 ^ L29;         // S5
    x[1] = ~(L13 ^ L27);      // S6
    x[0] = ~(L6 ^ L23);       // S7
}

// xtime (multiplication by {02}, FIPS-197 Sec. 4.2.1) on a bitsliced byte:
// shift up one bit and fold bit 7 back in at the positions of {1b}.
AES_HD void xtime(const uint32_t x[8], uint32_t y[8])
{
    y[0] = x[7];
    y[1] = x[0] ^ x[7];
    y[2] = x[1];
    y[3] = x[2] ^ x[7];
    y[4] = x[3] ^ x[7];
    y[5] = x[4];
    y[6] = x[5];
    y[7] = x[6];
}

// ShiftRows + MixColumns + AddRoundKey from planes x into planes y.
// Byte i of the state sits at row i % 4, column i / 4; after ShiftRows,
// column c row r holds the old byte r + 4((c + r) % 4).  With
// t = a0 ^ a1 ^ a2 ^ a3, MixColumns (FIPS-197 Sec. 5.1.3) is
// b_r = a_r ^ t ^ xtime(a_r ^ a_{r+1}).
template <class KEY>
AES_HD void shift_mix_ark(const uint32_t x[128], uint32_t y[128], const KEY &key)
{
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const uint32_t *a[4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
            a[r] = x + 8 * (r + 4 * ((c + r) & 3));
        uint32_t t[8];
#pragma unroll
        for (int b = 0; b < 8; ++b)
            t[b] = a[0][b] ^ a[1][b] ^ a[2][b] ^ a[3][b];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            uint32_t d[8], xd[8];
#pragma unroll
            for (int b = 0; b < 8; ++b)
                d[b] = a[r][b] ^ a[(r + 1) & 3][b];
            xtime(d, xd);
#pragma unroll
            for (int b = 0; b < 8; ++b)
                y[8 * (r + 4 * c) + b] = a[r][b] ^ t[b] ^ xd[b] ^ key(8 * (r + 4 * c) + b);
        }
    }
}

// ShiftRows + AddRoundKey (the final round has no MixColumns).
template <class KEY>
AES_HD void shift_ark(const uint32_t x[128], uint32_t y[128], const KEY &key)
{
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int b = 0; b < 8; ++b)
                y[8 * (r + 4 * c) + b] = x[8 * (r + 4 * ((c + r) & 3)) + b] ^ key(8 * (r + 4 * c) + b);
}

// One shift/mask stage of the transpose: for every row pair (k, k + J) with
// bit J of k clear, swap the J-bit sub-blocks selected by mask M.
template <int J>
AES_HD void swap_stage(uint32_t a[32], uint32_t m)
{
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        if (k & J)
            continue;
        const uint32_t t = ((a[k] >> J) ^ a[k + J]) & m;
        a[k + J] ^= t;
        a[k] ^= t << J;
    }
}

// In-place transpose of a 32x32 bit matrix: afterwards bit k of a[p] is what
// bit p of a[k] was (an involution).  Five swap stages; the 16- and 8-bit
// stages are byte permutations (PRMT), the others shift/mask swaps.
AES_HD void transpose32(uint32_t a[32])
{
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const uint32_t lo = a[k], hi = a[k + 16];
        a[k] = __byte_perm(lo, hi, 0x5410);
        a[k + 16] = __byte_perm(lo, hi, 0x7632);
    }
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        if (k & 8)
            continue;
        const uint32_t lo = a[k], hi = a[k + 8];
        a[k] = __byte_perm(lo, hi, 0x6240);
        a[k + 8] = __byte_perm(lo, hi, 0x7351);
    }
    swap_stage<4>(a, 0x0f0f0f0fu);
    swap_stage<2>(a, 0x33333333u);
    swap_stage<1>(a, 0x55555555u);
}

// All NR rounds on 128 planes (initial AddRoundKey NOT included: the caller
// folds round key 0 into the counter planes).  key(r, P) returns the mask of
// bit P of round key r.
template <int NR, class KEYS>
AES_HD void encrypt_rounds(uint32_t x[128], const KEYS &keys)
{
    uint32_t y[128];
#pragma unroll 1
    for (int r = 1; r < NR; ++r) {
#pragma unroll
        for (int i = 0; i < 16; ++i)
            sbox(x + 8 * i);
        shift_mix_ark(x, y, [&](int P) { return keys(r, P); });
#pragma unroll
        for (int P = 0; P < 128; ++P)
            x[P] = y[P];
    }
#pragma unroll
    for (int i = 0; i < 16; ++i)
        sbox(x + 8 * i);
    shift_ark(x, y, [&](int P) { return keys(NR, P); });
#pragma unroll
    for (int P = 0; P < 128; ++P)
        x[P] = y[P];
}

}  // namespace aesbs
