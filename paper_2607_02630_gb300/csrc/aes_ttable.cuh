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
// followed by __syncthreads() before the first lookup.  Te0 is first staged
// in a 1 KiB shared array (one global round trip for the whole CTA), then
// store q (16 bytes) writes four lane copies of one entry, consecutive
// threads writing consecutive 16-byte chunks (no bank conflicts; the staged
// entry is a broadcast read for 16 consecutive stores).  The fill is most of
// a short launch's fixed cost, so it waits for global memory only once.
__device__ __forceinline__ void fill_tables(uint8_t *smem, const uint32_t *__restrict__ te0)
{
    __shared__ uint32_t s_te0[256];
    for (uint32_t e = threadIdx.x; e < 256u; e += blockDim.x)
        s_te0[e] = __ldg(te0 + e);
    __syncthreads();
    constexpr uint32_t kStores = kTableBytes / 16;
#pragma unroll 4
    for (uint32_t q = threadIdx.x; q < kStores; q += blockDim.x) {
        const uint32_t h = q >> 12;              // region
        const uint32_t w = (q & 4095u) * 4u;     // word index inside the region
        const uint32_t t = (w >> 5) & 1u;        // even / odd table of the region
        const uint32_t r = 8u * (2u * h + t);
        const uint32_t v = s_te0[w >> 6];        // entry e = word / 64
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

// Round keys held in registers -- the batch kernel's warps, one request at a
// time.  The schedule is read once per tile (NR + 1 uniform 16-byte loads);
// indices are compile-time after unrolling, so every round's key is four
// register operands and costs no shared-memory wavefront.  The price is
// 4 * (NR + 1) registers a thread, which the 512-thread batch CTA can pay.
template <int NR>
struct RkRegs {
    uint4 w[NR + 1];
    __device__ __forceinline__ explicit RkRegs(const uint4 *__restrict__ g)
    {
#pragma unroll
        for (int r = 0; r <= NR; ++r)
            w[r] = __ldg(g + r);
    }
    __device__ __forceinline__ uint4 get(int r) const { return w[r]; }
};

// Rounds R0..NR-1 (full) and the final round NR on NB blocks held as
// s[b][0..3] (little-endian column words), in place.  The state passed in is
// the output of round R0 - 1.
template <int R0, int NR, int NB, class RK>
__device__ __forceinline__ void rounds(uint32_t (&s)[NB][4], const uint8_t *tab, const Lanes &ln,
                                       const RK &rk)
{
    const uint8_t *tabA = tab;
    const uint8_t *tabB = tab + kRegionBytes;
#pragma unroll
    for (int r = R0; r < NR; ++r) {
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

// Encrypt NB blocks held as s[b][0..3] in place: initial AddRoundKey, then
// Nr rounds.
template <int NR, int NB, class RK>
__device__ __forceinline__ void encrypt(uint32_t (&s)[NB][4], const uint8_t *tab, const Lanes &ln,
                                        const RK &rk)
{
    const uint4 k = rk.get(0);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        s[b][0] ^= k.x;
        s[b][1] ^= k.y;
        s[b][2] ^= k.z;
        s[b][3] ^= k.w;
    }
    rounds<1, NR, NB>(s, tab, ln, rk);
}

// Counter-mode caching.  The 256 counter blocks T = G*256 + L (L = 0..255)
// of one counter group share bytes 0..14, so after AddRoundKey only byte 15
// (row 3 of column 3, through Te3 into output column 0) varies in round 1:
// round 1 gives columns (P0 ^ Te3[L ^ k15], C1, C2, C3) with P0, C1..C3 fixed
// for the group.  In round 2 the varying column 0 feeds exactly one lookup of
// each output column (row r of column 0 reaches column -r mod 4), so round 2
// is Q_c ^ (one lookup) with Q0..Q3 fixed for the group.  A block then needs 5
// lookups for rounds 1-2 instead of 32; the group constants cost 27 lookups
// once per group.
struct Group {
    uint32_t p0, c1, c2, c3, q0, q1, q2, q3, k15;
};

// base: the group's first counter block (byte 15 = 0) as column words.
template <class RK>
__device__ __forceinline__ Group group_consts(const uint32_t base[4], const uint8_t *tab, const Lanes &ln,
                                              const RK &rk)
{
    const uint8_t *A = tab;                 // Te0 (lane sel s0), Te1 (s1)
    const uint8_t *B = tab + kRegionBytes;  // Te2 (s0), Te3 (s1)
    const uint4 k0 = rk.get(0), k1 = rk.get(1), k2 = rk.get(2);
    const uint32_t s0 = base[0] ^ k0.x, s1 = base[1] ^ k0.y, s2 = base[2] ^ k0.z, s3 = base[3] ^ k0.w;
    Group g;
    g.k15 = k0.w >> 24;
    g.p0 = lds(A, off<0>(s0, ln.s0)) ^ lds(A, off<1>(s1, ln.s1)) ^ lds(B, off<2>(s2, ln.s0)) ^ k1.x;
    g.c1 = lds(A, off<0>(s1, ln.s0)) ^ lds(A, off<1>(s2, ln.s1)) ^ lds(B, off<2>(s3, ln.s0)) ^
           lds(B, off<3>(s0, ln.s1)) ^ k1.y;
    g.c2 = lds(A, off<0>(s2, ln.s0)) ^ lds(A, off<1>(s3, ln.s1)) ^ lds(B, off<2>(s0, ln.s0)) ^
           lds(B, off<3>(s1, ln.s1)) ^ k1.z;
    g.c3 = lds(A, off<0>(s3, ln.s0)) ^ lds(A, off<1>(s0, ln.s1)) ^ lds(B, off<2>(s1, ln.s0)) ^
           lds(B, off<3>(s2, ln.s1)) ^ k1.w;
    g.q0 = lds(A, off<1>(g.c1, ln.s1)) ^ lds(B, off<2>(g.c2, ln.s0)) ^ lds(B, off<3>(g.c3, ln.s1)) ^ k2.x;
    g.q1 = lds(A, off<0>(g.c1, ln.s0)) ^ lds(A, off<1>(g.c2, ln.s1)) ^ lds(B, off<2>(g.c3, ln.s0)) ^ k2.y;
    g.q2 = lds(A, off<0>(g.c2, ln.s0)) ^ lds(A, off<1>(g.c3, ln.s1)) ^ lds(B, off<3>(g.c1, ln.s1)) ^ k2.z;
    g.q3 = lds(A, off<0>(g.c3, ln.s0)) ^ lds(B, off<2>(g.c1, ln.s0)) ^ lds(B, off<3>(g.c2, ln.s1)) ^ k2.w;
    return g;
}

// Keystream of NB blocks of one group, L[b] = the blocks' low counter bytes.
template <int NR, int NB, class RK>
__device__ __forceinline__ void encrypt_group(uint32_t (&s)[NB][4], const uint32_t (&L)[NB], const Group &g,
                                              const uint8_t *tab, const Lanes &ln, const RK &rk)
{
    const uint8_t *A = tab;
    const uint8_t *B = tab + kRegionBytes;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const uint32_t r10 = g.p0 ^ lds(B, off<0>(L[b] ^ g.k15, ln.s1));  // Te3[byte 15]
        s[b][0] = g.q0 ^ lds(A, off<0>(r10, ln.s0));                      // Te0[r10.b0]
        s[b][1] = g.q1 ^ lds(B, off<3>(r10, ln.s1));                      // Te3[r10.b3]
        s[b][2] = g.q2 ^ lds(B, off<2>(r10, ln.s0));                      // Te2[r10.b2]
        s[b][3] = g.q3 ^ lds(A, off<1>(r10, ln.s1));                      // Te1[r10.b1]
    }
    rounds<3, NR, NB>(s, tab, ln, rk);
}

}  // namespace aestt
