// ctr.cu -- single-buffer AES-CTR kernels (SP 800-38A Sec. 6.5).
//
// Two variants of the block cipher, same contract:
//   T-table  : each warp owns whole 256-block counter groups (lane l takes the
//              blocks whose counter low byte is l + 32m, so every load/store
//              instruction of the warp moves 512 contiguous bytes); rounds from
//              T-tables in bank-replicated shared memory with counter-mode
//              caching of rounds 1-2 (aes_ttable.cuh, tile.cuh).  128 KiB of
//              shared memory, one CTA per SM.
//   bitsliced: each warp owns 1024 consecutive blocks; lane l holds blocks
//              base + l + 32k (k = 0..31) as 128 bit planes (aes_bitslice.cuh),
//              so loads/stores are again 512 contiguous bytes per instruction.
// Both compute the counter block T_1 + j in registers, xor the keystream
// into the plaintext with 16-byte streaming loads/stores, and handle the
// final partial block bytewise without touching bytes past len.
#include "internal.h"
#include "common.cuh"
#include "aes_ttable.cuh"
#include "aes_bitslice.cuh"
#include "tile.cuh"

namespace {

using aesrt::CtrParams;

template <int NR, int NB>
__global__ void __launch_bounds__(1024, 1) ctr_ttable_kernel(const __grid_constant__ CtrParams p)
{
    extern __shared__ __align__(128) uint8_t smem[];
    aestt::fill_tables(smem, p.te0);
    __syncthreads();
    const aestt::Lanes ln;
    const aestt::RkConst rk{p.rk};
    const uint64_t nblocks = (p.len + 15) >> 4;
    const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    aestile::xor_range<NR, NB>(p.in, p.out, p.len, p.iv_hi, p.iv_lo, 0, nblocks, gwarp, nwarps, p.parts, smem,
                               ln, rk);
}

// Bit-plane masks of the round keys: mask[r*128 + P] = all-ones iff bit P of
// round key r is set (P = 8*byte + bit).
struct BsKeys {
    const uint4 *m;
    __device__ __forceinline__ uint32_t operator()(int r, int P) const
    {
        const uint4 q = m[r * 32 + (P >> 2)];
        return (P & 3) == 0 ? q.x : (P & 3) == 1 ? q.y : (P & 3) == 2 ? q.z : q.w;
    }
};

template <int NR>
__global__ void __launch_bounds__(128) ctr_bitslice_kernel(const __grid_constant__ CtrParams p)
{
    __shared__ __align__(16) uint32_t bsk[(NR + 1) * 128];
    for (int q = threadIdx.x; q < (NR + 1) * 128; q += blockDim.x) {
        const int r = q >> 7, P = q & 127;
        const uint32_t word = p.rk[4 * r + (P >> 5)];
        bsk[q] = ((word >> (P & 31)) & 1u) ? 0xffffffffu : 0u;
    }
    __syncthreads();
    const BsKeys keys{reinterpret_cast<const uint4 *>(bsk)};
    const uint64_t nfull = p.len >> 4;
    const uint32_t tail = (uint32_t)(p.len & 15);
    const uint64_t nblocks = nfull + (tail ? 1 : 0);
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t base = gwarp * 1024; base < nblocks; base += nwarps * 1024) {
        uint32_t x[128];
        const uint64_t j0 = base + lane;  // block k of this lane is j0 + 32k
        uint32_t c0[4];
        aesdev::counter_block(p.iv_hi, p.iv_lo, j0, c0);
        const uint32_t L = aesdev::bswap32(c0[3]);
        if (L <= 0xffffffffu - 31u * 32u) {
            // The 32 counters differ only in their last word: the planes of
            // bytes 0..11 are all-zeros/all-ones masks (round key 0 folded in).
#pragma unroll
            for (int w = 0; w < 3; ++w) {
                const uint32_t v = c0[w] ^ p.rk[w];
#pragma unroll
                for (int q = 0; q < 32; ++q)
                    x[32 * w + q] = 0u - ((v >> q) & 1u);
            }
#pragma unroll
            for (int k = 0; k < 32; ++k)
                x[96 + k] = aesdev::bswap32(L + 32u * (uint32_t)k) ^ p.rk[3];
            aesbs::transpose32(x + 96);
        } else {
            // A carry leaves the low word inside this lane's 32 blocks.
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                uint32_t c[4];
                aesdev::counter_block(p.iv_hi, p.iv_lo, j0 + 32u * (uint32_t)k, c);
#pragma unroll
                for (int w = 0; w < 4; ++w)
                    x[32 * w + k] = c[w] ^ p.rk[w];
            }
#pragma unroll
            for (int w = 0; w < 4; ++w)
                aesbs::transpose32(x + 32 * w);
        }
        aesbs::encrypt_rounds<NR>(x, keys);
#pragma unroll
        for (int w = 0; w < 4; ++w)
            aesbs::transpose32(x + 32 * w);
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const uint64_t j = j0 + 32u * (uint32_t)k;
            if (j < nfull) {
                const uint4 pt = aesdev::ld_stream(p.in + j);
                aesdev::st_stream(p.out + j, make_uint4(pt.x ^ x[k], pt.y ^ x[32 + k],
                                                        pt.z ^ x[64 + k], pt.w ^ x[96 + k]));
            } else if (j == nfull && tail) {
                aesdev::xor_tail(reinterpret_cast<const uint8_t *>(p.in + j),
                                 reinterpret_cast<uint8_t *>(p.out + j), x[k], x[32 + k], x[64 + k],
                                 x[96 + k], tail);
            }
        }
    }
}

template <int NR>
cudaError_t launch_tt(const CtrParams &p, const aesrt::CtrShape &s, int ctas, cudaStream_t st)
{
    const size_t smem = aestt::kTableBytes;
    switch (s.nb) {
    case 1: ctr_ttable_kernel<NR, 1><<<ctas, s.threads, smem, st>>>(p); break;
    case 2: ctr_ttable_kernel<NR, 2><<<ctas, s.threads, smem, st>>>(p); break;
    case 4: ctr_ttable_kernel<NR, 4><<<ctas, s.threads, smem, st>>>(p); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int NR>
cudaError_t set_tt_attr()
{
    const int smem = (int)aestt::kTableBytes;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(ctr_ttable_kernel<NR, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
        return e;
    if ((e = cudaFuncSetAttribute(ctr_ttable_kernel<NR, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
        return e;
    return cudaFuncSetAttribute(ctr_ttable_kernel<NR, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

}  // namespace

namespace aesrt {

cudaError_t ctr_set_attributes()
{
    cudaError_t e;
    if ((e = set_tt_attr<10>()) || (e = set_tt_attr<12>()) || (e = set_tt_attr<14>()))
        return e;
    return cudaSuccess;
}

// Resident CTAs per SM: T-table is bound by its 128 KiB of shared memory
// (one CTA); bitsliced CTAs of 128 threads are bound by registers.
int ctr_max_ctas(const CtrShape &s, int nsm)
{
    if (s.variant == 2)
        return nsm * (s.threads <= 128 ? 2 : 1);
    return nsm;
}

void ctr_plan(uint64_t nblocks, uint32_t v0, const CtrShape &s, int nsm, int *ctas, uint32_t *parts)
{
    const uint64_t cap = (uint64_t)ctr_max_ctas(s, nsm);
    const uint64_t warps = (uint64_t)(s.threads / 32);
    uint64_t units;
    uint32_t pt = 1;
    if (s.variant == 2) {
        units = (nblocks + 1023) / 1024;  // a bitsliced warp takes 1024 blocks per pass
    } else {
        // A T-table warp takes a whole 256-block counter group, or a part of
        // one when the message is too short to give every warp of the
        // largest grid a group (keeping at least NB blocks per lane per part).
        const uint64_t groups = nblocks ? ((v0 + nblocks - 1) >> 8) + 1 : 1;
        while (pt < 8u / (uint32_t)s.nb && groups * pt < cap * warps)
            pt *= 2;
        units = groups * pt;
    }
    uint64_t want = (units + warps - 1) / warps;
    if (s.ctas > 0)
        want = (uint64_t)s.ctas;
    if (want > cap)
        want = cap;
    *ctas = want < 1 ? 1 : (int)want;
    *parts = pt;
}

cudaError_t launch_ctr(const CtrParams &p, int nr, const CtrShape &s, int nsm, cudaStream_t stream)
{
    const uint64_t nblocks = (p.len + 15) / 16;
    int ctas = 1;
    uint32_t parts = 1;
    ctr_plan(nblocks, (uint32_t)(p.iv_lo & 255u), s, nsm, &ctas, &parts);
    if (s.variant == 2) {
        if (s.threads != 128)
            return cudaErrorInvalidValue;
        switch (nr) {
        case 10: ctr_bitslice_kernel<10><<<ctas, 128, 0, stream>>>(p); break;
        case 12: ctr_bitslice_kernel<12><<<ctas, 128, 0, stream>>>(p); break;
        case 14: ctr_bitslice_kernel<14><<<ctas, 128, 0, stream>>>(p); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    CtrParams q = p;
    q.parts = parts;
    switch (nr) {
    case 10: return launch_tt<10>(q, s, ctas, stream);
    case 12: return launch_tt<12>(q, s, ctas, stream);
    case 14: return launch_tt<14>(q, s, ctas, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace aesrt
