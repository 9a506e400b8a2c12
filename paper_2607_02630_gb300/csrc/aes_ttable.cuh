// aes_ttable.cuh -- AES rounds from T-tables in bank-replicated shared memory.
//
// One full round (FIPS-197 Sec. 5.1: SubBytes, ShiftRows, MixColumns,
// AddRoundKey) is, per output column c,
//   t_c = Te0[s_c.b0] ^ Te1[s_{c+1}.b1] ^ Te2[s_{c+2}.b2] ^ Te3[s_{c+3}.b3] ^ k_c
// where s_c is column c of the state as a little-endian word (byte r = row
// r), s_c.b_r its byte r, and Te_r[x] the column r of the MixColumns matrix
// times S(x): Te0[x] = (2S, S, S, 3S) in bytes 0..3 and Te_r = Te0 rotated
// left by 8r bits.  The final round has no MixColumns and takes S(x) out of
// the byte of Te_r that holds the plain S(x).
//
// Layout (128 KiB per CTA): region h in {0, 1} at byte h * 65536 holds Te_{2h}
// and Te_{2h+1}; entry e of Te_{2h+t}, copy for lane l, is the word at byte
// h*65536 + e*256 + t*128 + l*4.  Every lane reads its own copy, so the 32
// lanes of a warp always hit 32 distinct banks (conflict-free), and the byte
// offset of a lookup is one PRMT: byte 1 <- the state byte, byte 0 <- the
// lane's l*4 (+128 for odd tables), bytes 2..3 <- 0.
#pragma once
#include <stdint.h>

namespace aestt {

constexpr uint32_t kRegionBytes = 65536;
constexpr uint32_t kTableBytes = 2 * kRegionBytes;

// PRMT selector giving (x.byte_k << 8) | sel.byte0.
template <int K>
__device__ __forceinline__ uint32_t off(uint32_t x, uint32_t sel)
{
    return __byte_perm(x, sel, 0x5504 | (K << 4));
}

__device__ __forceinline__ uint32_t lds(const uint8_t *base, uint32_t o)
{
    return *reinterpret_cast<const uint32_t *>(base + o);
}

// Fill the replicated tables from Te0 (256 words in global memory).  Must be
// followed by __syncthreads() before the first lookup.
__device__ __forceinline__ void fill_tables(uint8_t *smem, const uint32_t *__restrict__ te0)
{
    for (uint32_t q = threadIdx.x; q < kTableBytes / 16; q += blockDim.x) {
        const uint32_t h = q >> 12;              // region
        const uint32_t w = (q & 4095u) * 4u;     // word index inside the region
        const uint32_t e = w >> 6;               // table entry
        const uint32_t t = (w >> 5) & 1u;        // even / odd table of the region
        const uint32_t v = __ldg(te0 + e);
        const uint32_t r = 8u * (2u * h + t);
        const uint32_t val = r ? __funnelshift_l(v, v, r) : v;
        *reinterpret_cast<uint4 *>(smem + h * kRegionBytes + w * 4u) = make_uint4(val, val, val, val);
    }
}

// Lane selectors for the PRMT: byte 0 = lane*4 (even table) or lane*4 + 128
// (odd table), bytes 1..3 = 0.
struct Lanes {
    uint32_t s0, s1;
    __device__ __forceinline__ Lanes()
    {
        const uint32_t lane = threadIdx.x & 31u;
        s0 = lane * 4u;
        s1 = lane * 4u + 128u;
    }
};

// Round keys stored as kernel parameters (constant bank) -- the single-key
// launch.  Indices are compile-time after unrolling, so the words are
// instruction operands and cost no registers or loads.
struct RkConst {
    const uint32_t *w;
    __device__ __forceinline__ uint4 get(int r) const
    {
        return make_uint4(w[4 * r], w[4 * r + 1], w[4 * r + 2], w[4 * r + 3]);
    }
};

// Round keys staged in shared memory (per-request keys of the batch and
// served kernels); one broadcast 16-byte load per round.
struct RkShared {
    const uint4 *w;
    __device__ __forceinline__ uint4 get(int r) const { return w[r]; }
};

// Encrypt NB blocks held as s[b][0..3] (little-endian column words) in
// place: Nr rounds, initial AddRoundKey included.
template <int NR, int NB, class RK>
__device__ __forceinline__ void encrypt(uint32_t (&s)[NB][4], const uint8_t *tab, const Lanes &ln,
                                        const RK &rk)
{
    const uint8_t *tabA = tab;
    const uint8_t *tabB = tab + kRegionBytes;
    {
        const uint4 k = rk.get(0);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            s[b][0] ^= k.x;
            s[b][1] ^= k.y;
            s[b][2] ^= k.z;
            s[b][3] ^= k.w;
        }
    }
#pragma unroll
    for (int r = 1; r < NR; ++r) {
        const uint4 k = rk.get(r);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const uint32_t a0 = s[b][0], a1 = s[b][1], a2 = s[b][2], a3 = s[b][3];
            s[b][0] = lds(tabA, off<0>(a0, ln.s0)) ^ lds(tabA, off<1>(a1, ln.s1)) ^
                      lds(tabB, off<2>(a2, ln.s0)) ^ lds(tabB, off<3>(a3, ln.s1)) ^ k.x;
            s[b][1] = lds(tabA, off<0>(a1, ln.s0)) ^ lds(tabA, off<1>(a2, ln.s1)) ^
                      lds(tabB, off<2>(a3, ln.s0)) ^ lds(tabB, off<3>(a0, ln.s1)) ^ k.y;
            s[b][2] = lds(tabA, off<0>(a2, ln.s0)) ^ lds(tabA, off<1>(a3, ln.s1)) ^
                      lds(tabB, off<2>(a0, ln.s0)) ^ lds(tabB, off<3>(a1, ln.s1)) ^ k.z;
            s[b][3] = lds(tabA, off<0>(a3, ln.s0)) ^ lds(tabA, off<1>(a0, ln.s1)) ^
                      lds(tabB, off<2>(a1, ln.s0)) ^ lds(tabB, off<3>(a2, ln.s1)) ^ k.w;
        }
    }
    {
        // Final round: byte r of output column c is S(s_{c+r}.b_r), taken
        // from the byte of a T-table entry that holds the plain S-box value:
        // Te2 byte 0, Te3 byte 1, Te0 byte 2, Te1 byte 3.
        const uint4 k = rk.get(NR);
        const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const uint32_t a[4] = {s[b][0], s[b][1], s[b][2], s[b][3]};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint32_t x0 = lds(tabB, off<0>(a[c], ln.s0));            // Te2, byte 0
                const uint32_t x1 = lds(tabB, off<1>(a[(c + 1) & 3], ln.s1));  // Te3, byte 1
                const uint32_t x2 = lds(tabA, off<2>(a[(c + 2) & 3], ln.s0));  // Te0, byte 2
                const uint32_t x3 = lds(tabA, off<3>(a[(c + 3) & 3], ln.s1));  // Te1, byte 3
                const uint32_t lo = __byte_perm(x0, x1, 0x3250);
                const uint32_t hi = __byte_perm(x2, x3, 0x7210);
                s[b][c] = __byte_perm(lo, hi, 0x7610) ^ kk[c];
            }
        }
    }
}

}  // namespace aestt
