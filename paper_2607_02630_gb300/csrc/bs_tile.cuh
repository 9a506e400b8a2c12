// bs_tile.cuh -- xor the AES-CTR keystream into a range of 16-byte blocks of
// one message with the bitsliced cipher (shared by the single-buffer and
// batch kernels).
//
// A warp takes 1024 consecutive blocks at a time: lane l holds blocks
// base + l + 32k (k = 0..31) as 128 bit planes (aes_bitslice.cuh), so every
// 16-byte load/store instruction of the warp moves 512 contiguous bytes.
// The counter blocks T_1 + j (SP 800-38A App. B.1, m = 128) are formed in
// registers; when the low 32-bit words of a lane's 32 counters do not carry,
// their upper 96 bits are equal and the planes of bytes 0..11 are constant
// masks.
#pragma once
#include <stdint.h>
#include "common.cuh"
#include "aes_bitslice.cuh"

namespace aesbs {

// Round-key bit planes in shared memory: word r*128 + P is all-ones iff bit
// P (P = 32*word + bit of the little-endian column words) of round key r is
// set, so AddRoundKey on planes is one xor per plane.
struct MaskKeys {
    const uint4 *m;
    __device__ __forceinline__ uint32_t operator()(int r, int P) const
    {
        const uint4 q = m[r * 32 + (P >> 2)];
        return (P & 3) == 0 ? q.x : (P & 3) == 1 ? q.y : (P & 3) == 2 ? q.z : q.w;
    }
};

// Masks of round keys 0..nr from the 4*(nr+1) schedule words `rk`, written
// by threads t = 0..nt-1 of the caller's group (a CTA or one warp).
__device__ __forceinline__ void build_masks(uint32_t *mask, const uint32_t *rk, int nr, uint32_t t, uint32_t nt)
{
    for (uint32_t q = t; q < (uint32_t)(nr + 1) * 128u; q += nt) {
        const uint32_t r = q >> 7, P = q & 127u;
        const uint32_t word = rk[4 * r + (P >> 5)];
        mask[q] = ((word >> (P & 31u)) & 1u) ? 0xffffffffu : 0u;
    }
}

// Blocks [first, last) of a message (in/out, len bytes, initial counter
// (iv_hi, iv_lo) as big-endian halves, rk0 = round key 0): the calling warp
// takes the 1024-block chunks starting at first + 1024 c for
// c = chunk0, chunk0 + chunk_stride, ...  The final partial block is done
// bytewise and nothing past len is touched.
template <int NR, class KEYS>
__device__ __forceinline__ void xor_range(const uint4 *__restrict__ in, uint4 *__restrict__ out, uint64_t len,
                                          uint64_t iv_hi, uint64_t iv_lo, const uint32_t (&rk0)[4], uint64_t first,
                                          uint64_t last, uint64_t chunk0, uint64_t chunk_stride, const KEYS &keys)
{
    const uint64_t nfull = len >> 4;
    const uint32_t tail = (uint32_t)(len & 15);
    const uint32_t lane = threadIdx.x & 31u;
    for (uint64_t base = first + chunk0 * 1024u; base < last; base += chunk_stride * 1024u) {
        uint32_t x[128];
        const uint64_t j0 = base + lane;  // block k of this lane is j0 + 32k
        uint32_t c0[4];
        aesdev::counter_block(iv_hi, iv_lo, j0, c0);
        const uint32_t L = aesdev::bswap32(c0[3]);
        if (L <= 0xffffffffu - 31u * 32u) {
            // The 32 counters differ only in their last word: the planes of
            // bytes 0..11 are all-zeros/all-ones masks (round key 0 folded in).
#pragma unroll
            for (int w = 0; w < 3; ++w) {
                const uint32_t v = c0[w] ^ rk0[w];
#pragma unroll
                for (int q = 0; q < 32; ++q)
                    x[32 * w + q] = 0u - ((v >> q) & 1u);
            }
#pragma unroll
            for (int k = 0; k < 32; ++k)
                x[96 + k] = aesdev::bswap32(L + 32u * (uint32_t)k) ^ rk0[3];
            transpose32(x + 96);
        } else {
            // A carry leaves the low word inside this lane's 32 blocks.
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                uint32_t c[4];
                aesdev::counter_block(iv_hi, iv_lo, j0 + 32u * (uint32_t)k, c);
#pragma unroll
                for (int w = 0; w < 4; ++w)
                    x[32 * w + k] = c[w] ^ rk0[w];
            }
#pragma unroll
            for (int w = 0; w < 4; ++w)
                transpose32(x + 32 * w);
        }
        encrypt_rounds<NR>(x, keys);
#pragma unroll
        for (int w = 0; w < 4; ++w)
            transpose32(x + 32 * w);
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const uint64_t j = j0 + 32u * (uint32_t)k;
            if (j >= last)
                continue;
            if (j < nfull) {
                const uint4 pt = aesdev::ld_stream(in + j);
                aesdev::st_stream(out + j, make_uint4(pt.x ^ x[k], pt.y ^ x[32 + k], pt.z ^ x[64 + k],
                                                      pt.w ^ x[96 + k]));
            } else if (j == nfull && tail) {
                aesdev::xor_tail(reinterpret_cast<const uint8_t *>(in + j), reinterpret_cast<uint8_t *>(out + j),
                                 x[k], x[32 + k], x[64 + k], x[96 + k], tail);
            }
        }
    }
}

}  // namespace aesbs
