// batch_noalloc.cu -- aes_ctr_batch_noalloc: the batched launch for callers
// that cannot allocate device memory.
//
// aes_ctr_batch allocates a small device image (descriptor table, tile map,
// claim counter) on every call.  Some callers cannot do that: a process whose
// whole HBM budget is already reserved by another framework's memory pool, a
// latency-critical path that must not pay for cudaMalloc/cudaFree (both can
// synchronise the device), or an embedded runtime that forbids dynamic
// allocation once it has started.  This entry point instead keeps its scratch
// -- up to AES_NOALLOC_MAX_REQUESTS descriptors plus the claim counter -- in
// one file-scope __device__ array that every GPU loading the library holds
// until the process exits.  The caller still owns the payload buffers and
// the key contexts (which must exist already: creating them is the only
// step that allocates).
//
// In host code the array's name is only a host-side stand-in, not a device
// address, so the first call on each device looks up the real address with
// cudaGetSymbolAddress (with that device current) and caches it; that first
// call should therefore come before any stream capture.  All calls share the
// one array and it keeps the previous call's contents: the claim counter is
// cleared on every call, and calls whose work overlaps on the GPU (two
// streams, or two threads) race on the array -- callers must serialise them.
#include "../../include/aesoffload.h"
#include "internal.h"
#include "runtime.h"
#include "common.cuh"
#include "aes_ttable.cuh"
#include "tile.cuh"

#include <cstring>
#include <mutex>

namespace {

using aesrt::BatchReq;

constexpr int kMaxReqs = AES_NOALLOC_MAX_REQUESTS;
constexpr size_t kReqBytes = sizeof(BatchReq) * (size_t)kMaxReqs;  // 64 KiB
constexpr size_t kScratchBytes = kReqBytes + 256;                    // + claim counter
constexpr size_t kSmem = aestt::kTableBytes + sizeof(uint64_t) * (size_t)kMaxReqs;

static __device__ __align__(256) uint8_t g_noalloc_scratch[kScratchBytes];

struct ScratchAddress {
    std::once_flag once;
    uint8_t *ptr = nullptr;
    cudaError_t err = cudaSuccess;
};
static ScratchAddress g_scratch[aesrt::kMaxDevices];

// The batch kernel without a tile map: each CTA copies the requests' first
// tile numbers into shared memory and finds the owner of a claimed tile by
// binary search.
template <int NB>
__global__ void __launch_bounds__(1024, 1)
    batch_noalloc_kernel(const BatchReq *__restrict__ reqs, int n, uint64_t total_tiles,
                         unsigned long long *__restrict__ counter, const uint32_t *__restrict__ te0,
                         uint32_t tile_blocks)
{
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t *s_begin = reinterpret_cast<uint64_t *>(smem + aestt::kTableBytes);
    __shared__ uint4 s_rk[15];
    __shared__ unsigned long long s_tile;
    __shared__ int s_req;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        s_begin[i] = reqs[i].tile_begin;
    aestt::fill_tables(smem, te0);
    const aestt::Lanes ln;
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned long long t = atomicAdd(counter, 1ull);
            if (t < total_tiles) {
                int lo = 0, hi = n - 1;  // last request whose first tile is <= t
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_begin[mid] <= t)
                        lo = mid;
                    else
                        hi = mid - 1;
                }
                s_req = lo;
            }
            s_tile = t;
        }
        __syncthreads();
        const unsigned long long t = s_tile;
        if (t >= total_tiles)
            break;
        const BatchReq rq = reqs[s_req];
        if (threadIdx.x <= rq.nr)
            s_rk[threadIdx.x] = rq.rk[threadIdx.x];
        __syncthreads();
        const uint64_t nblocks = (rq.len + 15) >> 4;
        const uint64_t first = (t - rq.tile_begin) * tile_blocks;
        const uint64_t last = min(first + tile_blocks, nblocks);
        switch (rq.nr) {
        case 10: aestile::run_tile<10, NB>(rq, first, last, smem, ln, s_rk); break;
        case 12: aestile::run_tile<12, NB>(rq, first, last, smem, ln, s_rk); break;
        default: aestile::run_tile<14, NB>(rq, first, last, smem, ln, s_rk); break;
        }
        __syncthreads();
    }
}

}  // namespace

using namespace aesrt;

extern "C" int aes_ctr_batch_noalloc(const aes_desc_t *descs, int n, void *stream)
{
    if (n < 0 || (n > 0 && !descs))
        return AES_EINVAL;
    if (n > kMaxReqs)
        return AES_ETOOBIG;
    if (n == 0)
        return AES_OK;
    DeviceState *st = nullptr;
    int rc = device_state_ready(&st);  // never initialises, so never allocates
    if (rc)
        return rc;
    ScratchAddress &sa = g_scratch[st->device];
    std::call_once(sa.once, [&sa] {
        sa.err = cudaGetSymbolAddress(reinterpret_cast<void **>(&sa.ptr), g_noalloc_scratch);
        if (sa.err == cudaSuccess) {
            sa.err = cudaFuncSetAttribute(batch_noalloc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)kSmem);
            if (sa.err == cudaSuccess)
                sa.err = cudaFuncSetAttribute(batch_noalloc_kernel<2>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
        }
    });
    if (sa.err != cudaSuccess)
        return cuda_fail(sa.err, "aes_ctr_batch_noalloc set-up");
    const BatchShape s = st->batch_tuned;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    // Validate every request before touching the shared scratch.
    uint64_t tiles = 0;
    for (int i = 0; i < n; ++i) {
        const aes_desc_t &d = descs[i];
        if (!d.ctx || d.ctx->device != st->device)
            return AES_EINVAL;
        if (d.len) {
            const void *din = nullptr;
            void *dout = nullptr;
            if ((rc = check_payload(d.in, d.out, d.len, st->device, &din, &dout)))
                return rc;
            tiles += ((d.len + 15) / 16 + (uint64_t)s.tile_blocks - 1) / (uint64_t)s.tile_blocks;
        }
    }
    if (tiles == 0)
        return AES_OK;
    // Descriptors go to the scratch in chunks staged on the stack (pageable
    // copies: each chunk buffer is free again when cudaMemcpyAsync returns).
    constexpr int kChunk = 32;
    BatchReq chunk[kChunk];
    uint64_t begin = 0;
    cudaError_t e = cudaSuccess;
    for (int i0 = 0; i0 < n && !e; i0 += kChunk) {
        const int cnt = n - i0 < kChunk ? n - i0 : kChunk;
        for (int k = 0; k < cnt; ++k) {
            const aes_desc_t &d = descs[i0 + k];
            BatchReq &r = chunk[k];
            std::memset(&r, 0, sizeof(r));
            r.len = d.len;
            iv_halves(d.iv, &r.iv_hi, &r.iv_lo);
            r.rk = reinterpret_cast<const uint4 *>(d.ctx->d_rk);
            r.nr = (uint32_t)d.ctx->nr;
            r.tile_begin = begin;
            if (d.len) {
                const void *din = nullptr;
                void *dout = nullptr;
                check_payload(d.in, d.out, d.len, st->device, &din, &dout);
                r.in = static_cast<const uint4 *>(din);
                r.out = static_cast<uint4 *>(dout);
                begin += ((d.len + 15) / 16 + (uint64_t)s.tile_blocks - 1) / (uint64_t)s.tile_blocks;
            }
        }
        e = cudaMemcpyAsync(sa.ptr + sizeof(BatchReq) * (size_t)i0, chunk, sizeof(BatchReq) * (size_t)cnt,
                            cudaMemcpyHostToDevice, cs);
    }
    unsigned long long *counter = reinterpret_cast<unsigned long long *>(sa.ptr + kReqBytes);
    if (!e)
        e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), cs);
    if (e)
        return cuda_fail(e, "aes_ctr_batch_noalloc copy");
    int ctas = s.ctas > 0 ? (s.ctas < st->nsm ? s.ctas : st->nsm) : st->nsm;
    if ((uint64_t)ctas > tiles)
        ctas = (int)tiles;
    const BatchReq *reqs = reinterpret_cast<const BatchReq *>(sa.ptr);
    if (s.tile_blocks / s.threads >= 2)
        batch_noalloc_kernel<2><<<ctas, s.threads, kSmem, cs>>>(reqs, n, tiles, counter, st->te0,
                                                                  (uint32_t)s.tile_blocks);
    else
        batch_noalloc_kernel<1><<<ctas, s.threads, kSmem, cs>>>(reqs, n, tiles, counter, st->te0,
                                                                  (uint32_t)s.tile_blocks);
    e = cudaGetLastError();
    return e ? cuda_fail(e, "batch_noalloc_kernel") : AES_OK;
}
