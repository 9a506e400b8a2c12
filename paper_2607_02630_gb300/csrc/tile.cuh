// tile.cuh -- encrypt one tile [first, last) of 16-byte blocks of a request
// with T-table rounds (shared by the batch and served kernels).
#pragma once
#include "internal.h"
#include "common.cuh"
#include "aes_ttable.cuh"

namespace aestile {

// Blocks are dealt to warps in chunks of 32*NB consecutive blocks (lane l of
// a chunk takes blocks base + 32b + l), so every 16-byte load/store
// instruction of a warp covers 512 contiguous bytes.
template <int NR, int NB>
__device__ __forceinline__ void run_tile(const aesrt::BatchReq &rq, uint64_t first, uint64_t last,
                                         const uint8_t *smem, const aestt::Lanes &ln,
                                         const uint4 *s_rk)
{
    const aestt::RkShared rk{s_rk};
    const uint64_t nfull = rq.len >> 4;
    const uint32_t tail = (uint32_t)(rq.len & 15);
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t nwarps = blockDim.x >> 5;
    constexpr uint64_t CH = 32 * NB;
    for (uint64_t base = first + (uint64_t)warp * CH; base < last; base += (uint64_t)nwarps * CH) {
        uint32_t s[NB][4];
        uint4 pt[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const uint64_t j = base + 32 * b + lane;
            aesdev::counter_block(rq.iv_hi, rq.iv_lo, j, s[b]);
            pt[b] = (j < nfull && j < last) ? aesdev::ld_stream(rq.in + j) : make_uint4(0, 0, 0, 0);
        }
        aestt::encrypt<NR, NB>(s, smem, ln, rk);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const uint64_t j = base + 32 * b + lane;
            if (j >= last)
                continue;
            if (j < nfull) {
                aesdev::st_stream(rq.out + j, make_uint4(pt[b].x ^ s[b][0], pt[b].y ^ s[b][1],
                                                         pt[b].z ^ s[b][2], pt[b].w ^ s[b][3]));
            } else if (j == nfull && tail) {
                aesdev::xor_tail(reinterpret_cast<const uint8_t *>(rq.in + j),
                                 reinterpret_cast<uint8_t *>(rq.out + j), s[b][0], s[b][1], s[b][2],
                                 s[b][3], tail);
            }
        }
    }
}

}  // namespace aestile
