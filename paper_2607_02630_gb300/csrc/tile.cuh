// tile.cuh -- xor the AES-CTR keystream into a range of 16-byte blocks of
// one message with T-table rounds and counter-mode caching (shared by the
// single-buffer, batch and served kernels).
#pragma once
#include "internal.h"
#include "common.cuh"
#include "aes_ttable.cuh"

namespace aestile {

// Blocks [first, last) of a message (in/out, len bytes, initial counter
// (iv_hi, iv_lo) as big-endian halves) are walked by counter group: group g
// holds blocks j = 256g - v0 + L, v0 = the IV's low byte, L = 0..255 the
// counter's low byte.  Lane l of a warp owns L = l + 32m (m = 0..7), so every
// 16-byte load/store instruction of a warp covers 32 consecutive blocks.  A
// group is split into `parts` work units (1, 2, 4 or 8; unit p covers
// m in [p*8/parts, (p+1)*8/parts)); warp w0, w0 + stride, ... take the units
// in order.  Whole groups amortise the 27 group-constant lookups best; parts
// spread a short message over more warps.  NB blocks per lane are in flight
// at once with their plaintext loaded before the keystream is computed.  The
// final partial block is done bytewise and nothing past len is touched.
template <int NR, int NB, class RK>
__device__ __forceinline__ void xor_range(const uint4 *__restrict__ in, uint4 *__restrict__ out, uint64_t len,
                                          uint64_t iv_hi, uint64_t iv_lo, uint64_t first, uint64_t last,
                                          uint64_t warp0, uint64_t warp_stride, uint32_t parts,
                                          const uint8_t *tab, const aestt::Lanes &ln, const RK &rk)
{
    if (first >= last)
        return;
    const uint64_t nfull = len >> 4;
    const uint32_t tail = (uint32_t)(len & 15);
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t v0 = iv_lo & 255u;
    const uint64_t base_lo = iv_lo & ~(uint64_t)255u;
    const uint64_t g_first = (v0 + first) >> 8, g_end = ((v0 + last - 1) >> 8) + 1;
    const uint32_t per = 8u / parts;
    const uint64_t u_end = (g_end - g_first) * parts;
    uint64_t gc_for = ~0ull;
    aestt::Group gc;
    const uint64_t pf_end = last < nfull ? last : nfull;  // full blocks only: never past the input
    for (uint64_t u = warp0; u < u_end; u += warp_stride) {
        const uint64_t g = g_first + u / parts;
        const uint32_t m_begin = (uint32_t)(u % parts) * per;
        if (NB == 1 && lane == 0 && u + warp_stride < u_end) {
            // With one block per lane in flight a warp has little of its own
            // to hide the payload's DRAM latency with: ask L2 now for the
            // plaintext of the warp's next unit (one bulk prefetch, a hint
            // that reads nothing into registers; the range stays inside the
            // input's full blocks).  Measured on the batch workload: 833 ->
            // 868 GB/s with one block per lane; with two it cost ~1.5 %, so
            // it is not compiled in there.
            const uint64_t un = u + warp_stride;
            const uint64_t jb = ((g_first + un / parts) << 8) - v0 + 32u * ((uint32_t)(un % parts) * per);
            const uint64_t a = jb < first ? first : jb;
            const uint64_t b = jb + 32u * per < pf_end ? jb + 32u * per : pf_end;
            if (a < b)  // also false when jb wrapped below 0 (the first group)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(in + a), "r"((uint32_t)((b - a) * 16u))
                             : "memory");
        }
        if (g != gc_for) {
            uint32_t base[4];
            const uint64_t l = base_lo + (g << 8);
            const uint64_t h = iv_hi + (l < base_lo ? 1ull : 0ull);
            base[0] = aesdev::bswap32((uint32_t)(h >> 32));
            base[1] = aesdev::bswap32((uint32_t)h);
            base[2] = aesdev::bswap32((uint32_t)(l >> 32));
            base[3] = aesdev::bswap32((uint32_t)l);
            gc = aestt::group_consts(base, tab, ln, rk);
            gc_for = g;
        }
        const uint64_t j0 = (g << 8) - v0;  // block of L = 0 (wraps below 0 in the first group)
#pragma unroll 1
        for (uint32_t m0 = m_begin; m0 < m_begin + per; m0 += NB) {
            uint32_t L[NB], s[NB][4];
            uint4 pt[NB];
            bool ok[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                L[b] = lane + 32u * (m0 + (uint32_t)b);
                const uint64_t j = j0 + L[b];
                // a wrapped index is huge and fails j < last; m past the unit is skipped
                ok[b] = m0 + (uint32_t)b < m_begin + per && j >= first && j < last;
                pt[b] = (ok[b] && j < nfull) ? aesdev::ld_stream(in + j) : make_uint4(0, 0, 0, 0);
            }
            aestt::encrypt_group<NR, NB>(s, L, gc, tab, ln, rk);
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const uint64_t j = j0 + L[b];
                if (!ok[b])
                    continue;
                if (j < nfull) {
                    aesdev::st_stream(out + j, make_uint4(pt[b].x ^ s[b][0], pt[b].y ^ s[b][1],
                                                          pt[b].z ^ s[b][2], pt[b].w ^ s[b][3]));
                } else if (tail) {  // j == nfull: the final partial block
                    aesdev::xor_tail(reinterpret_cast<const uint8_t *>(in + j),
                                     reinterpret_cast<uint8_t *>(out + j), s[b][0], s[b][1], s[b][2],
                                     s[b][3], tail);
                }
            }
        }
    }
}

// Blocks [first, last) of the `tile`-th run of `tile_groups` counter groups
// of a request with nb blocks and IV low byte v0 (tiles are group-aligned so
// no group is split between two tiles).
__device__ __forceinline__ void tile_blocks_of(uint64_t tile, uint32_t tile_groups, uint64_t v0, uint64_t nb,
                                               uint64_t *first, uint64_t *last)
{
    const uint64_t g0 = tile * tile_groups, g1 = g0 + tile_groups;
    *first = g0 == 0 ? 0 : (g0 << 8) - v0;
    const uint64_t e = (g1 << 8) - v0;
    *last = e < nb ? e : nb;
}

// One tile [first, last) of a batch/served request, spread over the CTA's
// warps (the CTA-wide loop of the no-alloc batch kernel).
template <int NR, int NB>
__device__ __forceinline__ void run_tile(const aesrt::BatchReq &rq, uint64_t first, uint64_t last,
                                         const uint8_t *smem, const aestt::Lanes &ln, const uint4 *s_rk)
{
    const aestt::RkShared rk{s_rk};
    xor_range<NR, NB>(rq.in, rq.out, rq.len, rq.iv_hi, rq.iv_lo, first, last, threadIdx.x >> 5,
                      blockDim.x >> 5, 1, smem, ln, rk);
}

// One tile [first, last) of a request, done by the calling warp alone.
template <int NR, int NB>
__device__ __forceinline__ void run_tile_warp(const aesrt::BatchReq &rq, uint64_t first, uint64_t last,
                                              const uint8_t *smem, const aestt::Lanes &ln, const uint4 *w_rk)
{
    const aestt::RkShared rk{w_rk};
    xor_range<NR, NB>(rq.in, rq.out, rq.len, rq.iv_hi, rq.iv_lo, first, last, 0, 1, 1, smem, ln, rk);
}

// One tile [first, last) of a request, done by the calling warp alone, with
// the request's round keys loaded into registers.
template <int NR, int NB>
__device__ __forceinline__ void run_tile_warp_regs(const aesrt::BatchReq &rq, uint64_t first, uint64_t last,
                                                   const uint8_t *smem, const aestt::Lanes &ln)
{
    const aestt::RkRegs<NR> rk(rq.rk);
    xor_range<NR, NB>(rq.in, rq.out, rq.len, rq.iv_hi, rq.iv_lo, first, last, 0, 1, 1, smem, ln, rk);
}

// Part `part` of `parts` of the single counter group [first, last) of a
// request, done by the calling warp alone (parts > 1 cuts a group's 8 blocks
// per lane into parts, so one request spreads over more warps).
template <int NR, int NB>
__device__ __forceinline__ void run_tile_warp(const aesrt::BatchReq &rq, uint64_t first, uint64_t last,
                                              uint32_t part, uint32_t parts, const uint8_t *smem,
                                              const aestt::Lanes &ln, const uint4 *w_rk)
{
    const aestt::RkShared rk{w_rk};
    xor_range<NR, NB>(rq.in, rq.out, rq.len, rq.iv_hi, rq.iv_lo, first, last, part, parts, parts, smem, ln, rk);
}

}  // namespace aestile
