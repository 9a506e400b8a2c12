// batch.cu -- many independent AES-CTR requests in one persistent launch.
//
// Every request (own key schedule, initial counter and length) is cut into
// tiles of tile_blocks / 256 whole counter groups (a counter group is 256
// blocks sharing the counter's upper 15 bytes, the unit of counter-mode
// caching).  A host-built table maps each tile to its request; the warps of
// the persistent CTAs (one per SM, T-tables filled once per CTA) each claim
// tiles through one device atomic counter until none are left, so long and
// short requests, AES-128 and AES-256, spread over all SMs (work stealing)
// without any CTA-wide barrier per tile.  The cipher is the same T-table
// round code as the single-buffer kernel.  Round keys: CTAs of up to 512
// threads (the default) hold the current request's schedule in registers
// (128 registers a thread), so the shared-memory pipe, the kernel's bound,
// serves T-table lookups only; larger CTAs stage it in each warp's slice of
// shared memory (one broadcast wavefront per round, about 5% of the pipe).
//
// The bitsliced kernel takes the same tiles with one warp per tile, 1024
// blocks at a time, as the autotuner's alternative to the T-tables.  A search
// variant of the T-table kernel finds a tile's request by binary search over
// the requests' first tiles instead of a tile map (aes_ctr_batch_noalloc).
//
// A nonzero `order` enables a test aid: tile t is processed as tile
// (a*t + b) mod T for a host-chosen a coprime to T (a permutation), so tiles
// complete in a scrambled order; results must not change.
#include "../../include/aesoffload.h"
#include "internal.h"
#include "runtime.h"
#include "common.cuh"
#include "aes_ttable.cuh"
#include "bs_tile.cuh"
#include "tile.cuh"

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

namespace {

using aesrt::BatchReq;

struct TileOrder {
    uint64_t a, b;  // t -> (a*t + b) mod T; a == 1, b == 0 is the identity
};

// CTA sizes up to this hold round keys in registers.
constexpr int kRegsMaxThreads = 512;
// The bitsliced batch kernel's CTA size (its warps are register-bound).
constexpr int kBsThreads = 128;

// The warp's next tile: lane 0 claims it from the device counter; returns
// the tile index (>= total_tiles when none are left), permuted if asked.
__device__ __forceinline__ unsigned long long claim_tile(unsigned long long *counter, uint64_t total_tiles,
                                                         const TileOrder &order)
{
    unsigned long long t = 0;
    if ((threadIdx.x & 31u) == 0)
        t = atomicAdd(counter, 1ull);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t < total_tiles && (order.a != 1 || order.b != 0))
        t = (order.a * t + order.b) % total_tiles;
    return t;
}

// Owner of tile t: the last request whose first tile is <= t (requests
// without tiles share their first tile number with the next request and are
// never chosen).  Lane 0 searches `begin[0..n)` in shared memory.
__device__ __forceinline__ uint32_t owner_of(const uint64_t *begin, int n, unsigned long long t)
{
    int lo = 0;
    if ((threadIdx.x & 31u) == 0) {
        int hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (begin[mid] <= t)
                lo = mid;
            else
                hi = mid - 1;
        }
    }
    return (uint32_t)__shfl_sync(0xffffffffu, lo, 0);
}

// The persistent T-table batch kernel.  NB: blocks per lane in flight;
// MAXT: largest CTA it is launched with; RK_REGS: round keys in registers
// (else in the warp's slice of shared memory); SEARCH: tile owners found by
// binary search over the requests' first tiles (copied into shared memory
// behind the tables) instead of read from the tile map.
template <int NB, int MAXT, bool RK_REGS, bool SEARCH>
__global__ void __launch_bounds__(MAXT, 1)
    batch_ttable_kernel(const BatchReq *__restrict__ reqs, const uint32_t *__restrict__ tile_req, int nreq,
                        uint64_t total_tiles, unsigned long long *__restrict__ counter,
                        const uint32_t *__restrict__ te0, uint32_t tile_groups, TileOrder order)
{
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ uint4 s_rk[RK_REGS ? 1 : MAXT / 32][15];  // round keys of each warp's current tile
    uint64_t *s_begin = reinterpret_cast<uint64_t *>(smem + aestt::kTableBytes);
    if (SEARCH)
        for (int i = threadIdx.x; i < nreq; i += blockDim.x)
            s_begin[i] = reqs[i].tile_begin;
    aestt::fill_tables(smem, te0);
    __syncthreads();
    const aestt::Lanes ln;
    const uint32_t lane = threadIdx.x & 31u;
    uint4 *w_rk = s_rk[RK_REGS ? 0 : threadIdx.x >> 5];
    // Every warp claims tiles on its own: no CTA-wide barrier per tile.
    for (;;) {
        const unsigned long long t = claim_tile(counter, total_tiles, order);
        if (t >= total_tiles)
            break;
        const uint32_t ri = SEARCH ? owner_of(s_begin, nreq, t) : __ldg(tile_req + t);
        const BatchReq rq = reqs[ri];
        uint64_t first, last;
        aestile::tile_blocks_of(t - rq.tile_begin, tile_groups, rq.iv_lo & 255u, (rq.len + 15) >> 4, &first,
                                &last);
        if (RK_REGS) {
            switch (rq.nr) {
            case 10: aestile::run_tile_warp_regs<10, NB>(rq, first, last, smem, ln); break;
            case 12: aestile::run_tile_warp_regs<12, NB>(rq, first, last, smem, ln); break;
            default: aestile::run_tile_warp_regs<14, NB>(rq, first, last, smem, ln); break;
            }
            continue;
        }
        if (lane <= rq.nr)
            w_rk[lane] = rq.rk[lane];
        __syncwarp();
        switch (rq.nr) {
        case 10: aestile::run_tile_warp<10, NB>(rq, first, last, smem, ln, w_rk); break;
        case 12: aestile::run_tile_warp<12, NB>(rq, first, last, smem, ln, w_rk); break;
        default: aestile::run_tile_warp<14, NB>(rq, first, last, smem, ln, w_rk); break;
        }
        __syncwarp();  // w_rk is rewritten by the next claim
    }
}

// The persistent bitsliced batch kernel: the same tiles and claims, each
// tile encrypted by one warp 1024 blocks at a time (bs_tile.cuh) with the
// request's round-key bit planes in the warp's slice of shared memory
// (rebuilt when the warp moves to a request with another key).
__global__ void __launch_bounds__(kBsThreads)
    batch_bitslice_kernel(const BatchReq *__restrict__ reqs, const uint32_t *__restrict__ tile_req,
                          uint64_t total_tiles, unsigned long long *__restrict__ counter, uint32_t tile_groups,
                          TileOrder order)
{
    __shared__ __align__(16) uint32_t s_mask[kBsThreads / 32][15 * 128];
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t *mask = s_mask[threadIdx.x >> 5];
    const uint4 *cur = nullptr;  // schedule whose masks are in `mask`
    for (;;) {
        const unsigned long long t = claim_tile(counter, total_tiles, order);
        if (t >= total_tiles)
            break;
        const BatchReq rq = reqs[__ldg(tile_req + t)];
        uint64_t first, last;
        aestile::tile_blocks_of(t - rq.tile_begin, tile_groups, rq.iv_lo & 255u, (rq.len + 15) >> 4, &first,
                                &last);
        if (rq.rk != cur) {
            __syncwarp();  // every lane is done with the previous masks
            aesbs::build_masks(mask, reinterpret_cast<const uint32_t *>(rq.rk), (int)rq.nr, lane, 32);
            __syncwarp();
            cur = rq.rk;
        }
        const uint4 k0 = __ldg(rq.rk);
        const uint32_t rk0[4] = {k0.x, k0.y, k0.z, k0.w};
        const aesbs::MaskKeys keys{reinterpret_cast<const uint4 *>(mask)};
        switch (rq.nr) {
        case 10: aesbs::xor_range<10>(rq.in, rq.out, rq.len, rq.iv_hi, rq.iv_lo, rk0, first, last, 0, 1, keys); break;
        case 12: aesbs::xor_range<12>(rq.in, rq.out, rq.len, rq.iv_hi, rq.iv_lo, rk0, first, last, 0, 1, keys); break;
        default: aesbs::xor_range<14>(rq.in, rq.out, rq.len, rq.iv_hi, rq.iv_lo, rk0, first, last, 0, 1, keys); break;
        }
    }
}

template <int NB, int MAXT, bool RK_REGS, bool SEARCH>
cudaError_t set_smem_attr()
{
    const size_t bytes = aestt::kTableBytes + (SEARCH ? sizeof(uint64_t) * aesrt::kSearchMaxReqs : 0);
    return cudaFuncSetAttribute(batch_ttable_kernel<NB, MAXT, RK_REGS, SEARCH>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <bool SEARCH>
cudaError_t set_smem_attrs()
{
    cudaError_t e;
    if ((e = set_smem_attr<1, kRegsMaxThreads, true, SEARCH>()) ||
        (e = set_smem_attr<2, kRegsMaxThreads, true, SEARCH>()) ||
        (e = set_smem_attr<4, kRegsMaxThreads, true, SEARCH>()) || (e = set_smem_attr<1, 1024, false, SEARCH>()) ||
        (e = set_smem_attr<2, 1024, false, SEARCH>()) || (e = set_smem_attr<4, 1024, false, SEARCH>()))
        return e;
    return cudaSuccess;
}

// Launch the T-table kernel for shape s (nb and the CTA size pick the
// instantiation).
template <bool SEARCH>
cudaError_t launch_ttable(int ctas, const aesrt::BatchShape &s, size_t smem, cudaStream_t stream,
                          const BatchReq *reqs, const uint32_t *map, int nreq, uint64_t total,
                          unsigned long long *counter, const uint32_t *te0, uint32_t tg, TileOrder order)
{
#define AES_BATCH_LAUNCH(NB, MAXT, REGS)                                                                   \
    batch_ttable_kernel<NB, MAXT, REGS, SEARCH><<<ctas, s.threads, smem, stream>>>(reqs, map, nreq, total, \
                                                                                   counter, te0, tg, order)
    const bool regs = s.threads <= kRegsMaxThreads;
    switch (s.nb) {
    case 1:
        if (regs)
            AES_BATCH_LAUNCH(1, kRegsMaxThreads, true);
        else
            AES_BATCH_LAUNCH(1, 1024, false);
        break;
    case 4:
        if (regs)
            AES_BATCH_LAUNCH(4, kRegsMaxThreads, true);
        else
            AES_BATCH_LAUNCH(4, 1024, false);
        break;
    default:
        if (regs)
            AES_BATCH_LAUNCH(2, kRegsMaxThreads, true);
        else
            AES_BATCH_LAUNCH(2, 1024, false);
        break;
    }
#undef AES_BATCH_LAUNCH
    return cudaGetLastError();
}

int g_bs_ctas_per_sm = 1;  // resident bitsliced batch CTAs per SM (set with the attributes)

}  // namespace

namespace aesrt {

cudaError_t batch_set_attributes()
{
    cudaError_t e;
    if ((e = set_smem_attrs<false>()) || (e = set_smem_attrs<true>()))
        return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_bitslice_kernel, kBsThreads, 0)))
        return e;
    g_bs_ctas_per_sm = per_sm > 0 ? per_sm : 1;
    return cudaSuccess;
}

cudaError_t launch_batch_search(const BatchReq *reqs, int n, uint64_t total_tiles, unsigned long long *counter,
                                const uint32_t *te0, const BatchShape &s, int nsm, cudaStream_t stream)
{
    if (n < 1 || n > kSearchMaxReqs || s.variant != AES_VARIANT_TTABLE)
        return cudaErrorInvalidValue;
    int ctas = s.ctas > 0 ? std::min(s.ctas, nsm) : nsm;
    if ((uint64_t)ctas > total_tiles)
        ctas = (int)total_tiles;
    const size_t smem = aestt::kTableBytes + sizeof(uint64_t) * (size_t)n;
    return launch_ttable<true>(ctas, s, smem, stream, reqs, nullptr, n, total_tiles, counter, te0,
                               (uint32_t)(s.tile_blocks / 256), TileOrder{1, 0});
}

static uint64_t gcd64(uint64_t a, uint64_t b)
{
    while (b) {
        const uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

static TileOrder make_order(uint64_t total, uint32_t seed)
{
    TileOrder o{1, 0};
    if (!seed || total < 2)
        return o;
    uint64_t x = seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    for (int tries = 0; tries < 64; ++tries) {
        x ^= x >> 29;
        x *= 0xBF58476D1CE4E5B9ull;
        x ^= x >> 32;
        const uint64_t a = 1 + x % (total - 1);
        if (gcd64(a, total) == 1 && a != 1) {
            o.a = a;
            break;
        }
    }
    o.b = (x >> 7) % total;
    return o;
}

// Host-side preparation shared by aes_ctr_batch and the graph plans.
struct BatchTables {
    std::vector<BatchReq> reqs;
    std::vector<uint32_t> tile_req;
    uint64_t total_tiles = 0;
    int64_t bytes = 0;
};

int validate_batch_shape(BatchShape &s)
{
    if (s.variant == AES_VARIANT_AUTO)
        s.variant = AES_VARIANT_TTABLE;
    if (s.variant == AES_VARIANT_BITSLICE) {
        if (s.threads != kBsThreads)
            return AES_EINVAL;  // one instantiation: 128-thread CTAs
    } else if (s.variant != AES_VARIANT_TTABLE) {
        return AES_EINVAL;
    }
    if (s.nb != 1 && s.nb != 2 && s.nb != 4)
        return AES_EINVAL;
    if (s.threads < 32 || s.threads > 1024 || (s.threads & 31))
        return AES_EINVAL;
    if (s.tile_blocks < 256 || s.tile_blocks % 256 || s.tile_blocks > (1 << 22))
        return AES_EINVAL;
    if (s.ctas < 0)
        return AES_EINVAL;
    return AES_OK;
}

static BatchShape pick_batch_shape(const DeviceState &st, const aes_batch_opts_t *opts)
{
    BatchShape s = st.batch_tuned;
    if (opts) {
        if (opts->variant && opts->variant != s.variant) {
            // another variant than the tuned one: start from its defaults
            s = opts->variant == AES_VARIANT_BITSLICE ? BatchShape{AES_VARIANT_BITSLICE, kBsThreads, 2048, 0, 1}
                                                      : BatchShape{opts->variant, 512, 2048, 0, 2};
        }
        if (opts->threads)
            s.threads = opts->threads;
        if (opts->tile_blocks)
            s.tile_blocks = opts->tile_blocks;
        if (opts->ctas)
            s.ctas = opts->ctas;
        if (opts->blocks_per_thread)
            s.nb = opts->blocks_per_thread;
    }
    return s;
}

static int build_tables(const aes_desc_t *descs, int n, int dev, const BatchShape &s, BatchTables &bt)
{
    bt.reqs.resize((size_t)n);
    uint64_t tiles = 0;
    for (int i = 0; i < n; ++i) {
        const aes_desc_t &d = descs[i];
        if (!d.ctx)
            return AES_EINVAL;
        if (d.ctx->device != dev)
            return AES_EINVAL;
        BatchReq &r = bt.reqs[(size_t)i];
        std::memset(&r, 0, sizeof(r));
        r.len = d.len;
        iv_halves(d.iv, &r.iv_hi, &r.iv_lo);
        r.rk = reinterpret_cast<const uint4 *>(d.ctx->d_rk);
        r.nr = (uint32_t)d.ctx->nr;
        r.tile_begin = tiles;
        if (d.len) {
            const void *din = nullptr;
            void *dout = nullptr;
            int rc = check_payload(d.in, d.out, d.len, dev, &din, &dout);
            if (rc)
                return rc;
            r.in = static_cast<const uint4 *>(din);
            r.out = static_cast<uint4 *>(dout);
            tiles += tiles_of(d.len, d.iv[15], s.tile_blocks);
            bt.bytes += (int64_t)d.len;
        }
    }
    if (tiles > 0xffffffffull)
        return AES_ETOOBIG;
    bt.total_tiles = tiles;
    bt.tile_req.resize((size_t)tiles);
    for (int i = 0; i < n; ++i) {
        const BatchReq &r = bt.reqs[(size_t)i];
        const uint64_t k = r.len ? tiles_of(r.len, (uint32_t)(r.iv_lo & 255u), s.tile_blocks) : 0;
        for (uint64_t t = 0; t < k; ++t)
            bt.tile_req[(size_t)(r.tile_begin + t)] = (uint32_t)i;
    }
    return AES_OK;
}

// Device image: [reqs][tile map][counter], each part 256-byte aligned.
struct DeviceImage {
    size_t off_map = 0, off_counter = 0, bytes = 0;
};

static DeviceImage image_layout(const BatchTables &bt)
{
    DeviceImage im;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    im.off_map = up(bt.reqs.size() * sizeof(BatchReq));
    im.off_counter = up(im.off_map + bt.tile_req.size() * sizeof(uint32_t));
    im.bytes = im.off_counter + 256;
    return im;
}

cudaError_t launch_batch_image(uint8_t *img, const DeviceImage &im, const BatchTables &bt,
                               const uint32_t *te0, const BatchShape &s, int nsm, uint32_t seed,
                               cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(img + im.off_counter, 0, sizeof(unsigned long long), stream);
    if (e)
        return e;
    // persistent CTAs: as many as are resident at once (one T-table CTA
    // per SM: its tables take 128 KiB of shared memory)
    const int resident = s.variant == AES_VARIANT_BITSLICE ? nsm * g_bs_ctas_per_sm : nsm;
    int ctas = s.ctas > 0 ? std::min(s.ctas, resident) : resident;
    if ((uint64_t)ctas > bt.total_tiles)
        ctas = (int)bt.total_tiles;
    const TileOrder order = make_order(bt.total_tiles, seed);
    const BatchReq *reqs = reinterpret_cast<const BatchReq *>(img);
    const uint32_t *map = reinterpret_cast<const uint32_t *>(img + im.off_map);
    unsigned long long *counter = reinterpret_cast<unsigned long long *>(img + im.off_counter);
    const uint32_t tg = (uint32_t)(s.tile_blocks / 256);
    if (s.variant == AES_VARIANT_BITSLICE) {
        batch_bitslice_kernel<<<ctas, kBsThreads, 0, stream>>>(reqs, map, bt.total_tiles, counter, tg, order);
        return cudaGetLastError();
    }
    return launch_ttable<false>(ctas, s, aestt::kTableBytes, stream, reqs, map, (int)bt.reqs.size(),
                                bt.total_tiles, counter, te0, tg, order);
}

}  // namespace aesrt

using namespace aesrt;

struct aes_batch_plan_s {
    int device;
    BatchTables bt;
    DeviceImage im;
    uint8_t *img = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

int aes_ctr_batch_ex(const aes_desc_t *descs, int n, void *stream, const aes_batch_opts_t *opts)
{
    if (n < 0 || (n > 0 && !descs))
        return AES_EINVAL;
    if (n > AES_BATCH_MAX)
        return AES_ETOOBIG;
    if (n == 0)
        return AES_OK;
    DeviceState *st = nullptr;
    int rc = device_state(&st);
    if (rc)
        return rc;
    BatchShape s = pick_batch_shape(*st, opts);
    if ((rc = validate_batch_shape(s)))
        return rc;
    BatchTables bt;
    if ((rc = build_tables(descs, n, st->device, s, bt)))
        return rc;
    if (bt.total_tiles == 0)
        return AES_OK;
    const DeviceImage im = image_layout(bt);
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    uint8_t *img = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&img), im.bytes, cs);
    if (e)
        return e == cudaErrorMemoryAllocation ? AES_ENOMEM : cuda_fail(e, "cudaMallocAsync");
    // Pageable sources: each copy has finished reading the host vector when
    // cudaMemcpyAsync returns, so bt may be destroyed afterwards.
    e = cudaMemcpyAsync(img, bt.reqs.data(), bt.reqs.size() * sizeof(BatchReq),
                        cudaMemcpyHostToDevice, cs);
    if (!e)
        e = cudaMemcpyAsync(img + im.off_map, bt.tile_req.data(), bt.tile_req.size() * sizeof(uint32_t),
                            cudaMemcpyHostToDevice, cs);
    if (!e)
        e = launch_batch_image(img, im, bt, st->te0, s, st->nsm, opts ? opts->tile_order_seed : 0, cs);
    cudaError_t e2 = cudaFreeAsync(img, cs);
    if (e)
        return cuda_fail(e, "aes_ctr_batch");
    if (e2)
        return cuda_fail(e2, "cudaFreeAsync");
    return AES_OK;
}

int aes_ctr_batch(const aes_desc_t *descs, int n, void *stream)
{
    return aes_ctr_batch_ex(descs, n, stream, nullptr);
}

int aes_batch_plan_create(aes_batch_plan_t *out, const aes_desc_t *descs, int n,
                          const aes_batch_opts_t *opts)
{
    if (!out)
        return AES_EINVAL;
    *out = nullptr;
    if (n < 1 || !descs)
        return AES_EINVAL;
    if (n > AES_BATCH_MAX)
        return AES_ETOOBIG;
    DeviceState *st = nullptr;
    int rc = device_state(&st);
    if (rc)
        return rc;
    BatchShape s = pick_batch_shape(*st, opts);
    if ((rc = validate_batch_shape(s)))
        return rc;
    aes_batch_plan_s *plan = new (std::nothrow) aes_batch_plan_s();
    if (!plan)
        return AES_ENOMEM;
    plan->device = st->device;
    if ((rc = build_tables(descs, n, st->device, s, plan->bt))) {
        delete plan;
        return rc;
    }
    plan->im = image_layout(plan->bt);
    cudaError_t e = cudaMalloc(&plan->img, plan->im.bytes);
    if (e) {
        delete plan;
        return e == cudaErrorMemoryAllocation ? AES_ENOMEM : cuda_fail(e, "cudaMalloc(plan)");
    }
    e = cudaMemcpyAsync(plan->img, plan->bt.reqs.data(), plan->bt.reqs.size() * sizeof(BatchReq),
                        cudaMemcpyHostToDevice, st->setup);
    if (!e && !plan->bt.tile_req.empty())
        e = cudaMemcpyAsync(plan->img + plan->im.off_map, plan->bt.tile_req.data(),
                            plan->bt.tile_req.size() * sizeof(uint32_t), cudaMemcpyHostToDevice,
                            st->setup);
    if (!e)
        e = cudaStreamSynchronize(st->setup);
    // Capture counter reset + persistent kernel on a private stream.
    cudaStream_t cap = nullptr;
    if (!e)
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (!e && plan->bt.total_tiles > 0) {
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (!e) {
            cudaError_t le = launch_batch_image(plan->img, plan->im, plan->bt, st->te0, s, st->nsm,
                                                opts ? opts->tile_order_seed : 0, cap);
            e = cudaStreamEndCapture(cap, &plan->graph);
            if (!e)
                e = le;
        }
        if (!e)
            e = cudaGraphInstantiate(&plan->exec, plan->graph, 0);
    }
    if (cap)
        cudaStreamDestroy(cap);
    if (e) {
        if (plan->exec)
            cudaGraphExecDestroy(plan->exec);
        if (plan->graph)
            cudaGraphDestroy(plan->graph);
        cudaFree(plan->img);
        delete plan;
        return cuda_fail(e, "aes_batch_plan_create");
    }
    *out = plan;
    return AES_OK;
}

int aes_batch_plan_launch(aes_batch_plan_t plan, void *stream)
{
    if (!plan)
        return AES_EINVAL;
    if (!plan->exec)
        return AES_OK;  // nothing to encrypt (all lengths zero)
    cudaError_t e = cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(stream));
    return e ? cuda_fail(e, "cudaGraphLaunch") : AES_OK;
}

int64_t aes_batch_plan_bytes(aes_batch_plan_t plan) { return plan ? plan->bt.bytes : AES_EINVAL; }

int aes_batch_plan_destroy(aes_batch_plan_t plan)
{
    if (!plan)
        return AES_OK;
    if (plan->exec)
        cudaGraphExecDestroy(plan->exec);
    if (plan->graph)
        cudaGraphDestroy(plan->graph);
    cudaFree(plan->img);
    delete plan;
    return AES_OK;
}

}  // extern "C"
