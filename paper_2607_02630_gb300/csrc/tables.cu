// tables.cu -- device-side table generation and key expansion.
//
// Te0 is derived on the device from the field arithmetic itself: the
// multiplicative group of GF(2^8) is cyclic with generator {03}, so one
// thread walks the powers of {03} to build antilog/log tables, and every
// thread then forms x^{-1} = {03}^(255 - log x), applies the affine map of
// FIPS-197 Sec. 5.1.1 and packs the MixColumns column (2S, S, S, 3S).
#include "internal.h"
#include "common.cuh"

namespace {

__device__ __forceinline__ uint32_t xtime8(uint32_t b)
{
    b <<= 1;
    return (b & 0x100u) ? (b ^ 0x11bu) : b;
}

__global__ void te0_init_kernel(uint32_t *__restrict__ te0)
{
    __shared__ uint8_t alog[256];
    __shared__ uint8_t lg[256];
    if (threadIdx.x == 0) {
        uint32_t a = 1;
        for (int i = 0; i < 255; ++i) {
            alog[i] = (uint8_t)a;
            lg[a] = (uint8_t)i;
            a ^= xtime8(a);  // a * {03}
        }
        alog[255] = alog[0];
        lg[0] = 0;
    }
    __syncthreads();
    const uint32_t x = threadIdx.x;
    uint32_t inv = x ? alog[(255u - lg[x]) % 255u] : 0u;
    // affine map: b ^ rotl(b,1) ^ rotl(b,2) ^ rotl(b,3) ^ rotl(b,4) ^ {63}
    uint32_t r = inv | (inv << 8);
    uint32_t s = (inv ^ (r >> 7) ^ (r >> 6) ^ (r >> 5) ^ (r >> 4) ^ 0x63u) & 0xffu;
    const uint32_t s2 = xtime8(s);
    te0[x] = s2 | (s << 8) | (s << 16) | ((s2 ^ s) << 24);
}

// FIPS-197 Sec. 5.2 for a batch of keys, one thread per key.  keys: n rows of
// 32 bytes (the first bits/8 used); bits: n entries; w: n rows of 60 words
// (4*(Nr+1) used), word i = bytes 4i..4i+3 of the schedule, little-endian.
__global__ void key_expand_kernel(const uint8_t *__restrict__ keys, const int32_t *__restrict__ bits,
                                  const uint32_t *__restrict__ te0, uint32_t *__restrict__ w, int n)
{
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n)
        return;
    const int nk = bits[id] / 32;
    const int total = 4 * (nk + 7);
    const uint8_t *key = keys + 32 * id;
    uint32_t *out = w + 60 * id;
    uint32_t sched[60];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (i < nk)
            sched[i] = key[4 * i] | (key[4 * i + 1] << 8) | (key[4 * i + 2] << 16) |
                       ((uint32_t)key[4 * i + 3] << 24);
    }
    auto sub = [&](uint32_t v) {
        return ((te0[v & 0xff] >> 8) & 0xff) | (((te0[(v >> 8) & 0xff] >> 8) & 0xff) << 8) |
               (((te0[(v >> 16) & 0xff] >> 8) & 0xff) << 16) |
               (((te0[(v >> 24) & 0xff] >> 8) & 0xff) << 24);
    };
    uint32_t rc = 1;
    for (int i = nk; i < total; ++i) {
        uint32_t t = sched[i - 1];
        if (i % nk == 0) {
            t = sub((t >> 8) | (t << 24)) ^ rc;  // SubWord(RotWord) ^ Rcon
            rc = xtime8(rc);
        } else if (nk > 6 && i % nk == 4) {
            t = sub(t);
        }
        sched[i] = sched[i - nk] ^ t;
    }
    for (int i = 0; i < total; ++i)
        out[i] = sched[i];
}

}  // namespace

namespace aesrt {

cudaError_t launch_te0_init(uint32_t *te0, cudaStream_t stream)
{
    te0_init_kernel<<<1, 256, 0, stream>>>(te0);
    return cudaGetLastError();
}

cudaError_t launch_key_expand(const uint8_t *keys, const int32_t *bits, const uint32_t *te0,
                              uint32_t *w, int n, cudaStream_t stream)
{
    if (n <= 0)
        return cudaSuccess;
    const int threads = 128;
    key_expand_kernel<<<(n + threads - 1) / threads, threads, 0, stream>>>(keys, bits, te0, w, n);
    return cudaGetLastError();
}

}  // namespace aesrt
