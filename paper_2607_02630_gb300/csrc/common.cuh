// common.cuh -- device helpers shared by the CTR kernels.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

namespace aesdev {

// Byte swap of a 32-bit word (one PRMT).
__device__ __forceinline__ uint32_t bswap32(uint32_t x) { return __byte_perm(x, 0, 0x0123); }

// Counter block T_1 + j mod 2^128 (SP 800-38A App. B.1 with m = 128).  The
// initial counter is given as its two big-endian 64-bit halves (hi = bytes
// 0..7, lo = bytes 8..15 read as big-endian integers).  The result is the
// block as four little-endian words, i.e. w[c] holds bytes 4c..4c+3 -- the
// same layout the cipher uses for column c of the state.
__device__ __forceinline__ void counter_block(uint64_t hi, uint64_t lo, uint64_t j, uint32_t w[4])
{
    const uint64_t l = lo + j;
    const uint64_t h = hi + (l < lo ? 1ull : 0ull);
    w[0] = bswap32((uint32_t)(h >> 32));
    w[1] = bswap32((uint32_t)h);
    w[2] = bswap32((uint32_t)(l >> 32));
    w[3] = bswap32((uint32_t)l);
}

// Streaming 16-byte load / store: payload bytes are touched once.
__device__ __forceinline__ uint4 ld_stream(const uint4 *p)
{
    uint4 v;
    asm volatile("ld.global.cs.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}
__device__ __forceinline__ void st_stream(uint4 *p, uint4 v)
{
    asm volatile("st.global.cs.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w));
}

// xor of a keystream block into one payload block; `u` < 16 bytes of a final
// partial block are done bytewise so nothing past len is read or written.
__device__ __forceinline__ void xor_tail(const uint8_t *in, uint8_t *out, uint32_t k0, uint32_t k1,
                                         uint32_t k2, uint32_t k3, uint32_t u)
{
    for (uint32_t b = 0; b < u; ++b) {
        const uint32_t w = b < 4 ? k0 : b < 8 ? k1 : b < 12 ? k2 : k3;
        out[b] = in[b] ^ (uint8_t)(w >> (8 * (b & 3)));
    }
}

}  // namespace aesdev
