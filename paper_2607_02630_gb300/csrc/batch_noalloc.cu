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
// cudaGetSymbolAddress (with that device current) and caches it.  All calls
// share the one array and it keeps the previous call's contents: the claim
// counter is cleared on every call, and calls whose work overlaps on the GPU
// (two streams, or two threads) race on the array -- callers must serialise
// them.  A call copies its descriptors from a stack buffer with
// cudaMemcpyAsync (pageable host memory), so it must not be made while its
// stream is being captured into a CUDA graph; callers that want a graph use
// the batch plans (aes_batch_plan_create), which allocate once up front.
//
// The kernel is the batch kernel's search variant (batch.cu): the same
// persistent T-table CTAs, tiles of whole counter groups claimed by each warp
// from one counter, and the owner of a claimed tile found by a binary search
// over the requests' first tiles in shared memory instead of a tile map.
#include "../../include/aesoffload.h"
#include "internal.h"
#include "runtime.h"
#include <cstring>
#include <mutex>

namespace {

using aesrt::BatchReq;

constexpr int kMaxReqs = AES_NOALLOC_MAX_REQUESTS;
static_assert(kMaxReqs <= aesrt::kSearchMaxReqs, "the search kernel holds every request's first tile");
constexpr size_t kReqBytes = sizeof(BatchReq) * (size_t)kMaxReqs;  // 64 KiB
constexpr size_t kScratchBytes = kReqBytes + 256;                    // + claim counter

static __device__ __align__(256) uint8_t g_noalloc_scratch[kScratchBytes];

struct ScratchAddress {
    std::once_flag once;
    uint8_t *ptr = nullptr;
    cudaError_t err = cudaSuccess;
};
static ScratchAddress g_scratch[aesrt::kMaxDevices];

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
    });
    if (sa.err != cudaSuccess)
        return cuda_fail(sa.err, "aes_ctr_batch_noalloc set-up");
    // the tuned T-table shape (the search kernel has no bitsliced variant)
    BatchShape s = st->batch_tuned;
    if (s.variant != AES_VARIANT_TTABLE)
        s = BatchShape{AES_VARIANT_TTABLE, 512, 2048, 0, 2};
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
            tiles += tiles_of(d.len, d.iv[15], s.tile_blocks);
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
                begin += tiles_of(d.len, d.iv[15], s.tile_blocks);
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
    e = launch_batch_search(reinterpret_cast<const BatchReq *>(sa.ptr), n, tiles, counter, st->te0, s, st->nsm,
                            cs);
    return e ? cuda_fail(e, "aes_ctr_batch_noalloc launch") : AES_OK;
}
