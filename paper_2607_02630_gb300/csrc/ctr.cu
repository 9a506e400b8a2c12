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
#include "bs_tile.cuh"
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

template <int NR>
__global__ void __launch_bounds__(128) ctr_bitslice_kernel(const __grid_constant__ CtrParams p)
{
    __shared__ __align__(16) uint32_t bsk[(NR + 1) * 128];
    aesbs::build_masks(bsk, p.rk, NR, threadIdx.x, blockDim.x);
    __syncthreads();
    const uint32_t rk0[4] = {p.rk[0], p.rk[1], p.rk[2], p.rk[3]};
    const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    aesbs::xor_range<NR>(p.in, p.out, p.len, p.iv_hi, p.iv_lo, rk0, 0, (p.len + 15) >> 4, gwarp, nwarps,
                         aesbs::MaskKeys{reinterpret_cast<const uint4 *>(bsk)});
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
