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
// A nonzero `order` enables a test aid: tile t is processed as tile
// (a*t + b) mod T for a host-chosen a coprime to T (a permutation), so tiles
// complete in a scrambled order; results must not change.
#include "../../include/aesoffload.h"
#include "internal.h"
#include "runtime.h"
#include "common.cuh"
#include "aes_ttable.cuh"
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

template <int NB, int MAXT, bool RK_REGS>
__global__ void __launch_bounds__(MAXT, 1)
    batch_ttable_kernel(const BatchReq *__restrict__ reqs, const uint32_t *__restrict__ tile_req,
                        uint64_t total_tiles, unsigned long long *__restrict__ counter,
                        const uint32_t *__restrict__ te0, uint32_t tile_groups, TileOrder order)
{
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ uint4 s_rk[RK_REGS ? 1 : MAXT / 32][15];  // round keys of each warp's current tile
    aestt::fill_tables(smem, te0);
    __syncthreads();
    const aestt::Lanes ln;
    const uint32_t lane = threadIdx.x & 31u;
    uint4 *w_rk = s_rk[RK_REGS ? 0 : threadIdx.x >> 5];
    const bool permuted = order.a != 1 || order.b != 0;
    // Every warp claims tiles on its own: no CTA-wide barrier per tile.
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0)
            t = atomicAdd(counter, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= total_tiles)
            break;
        if (permuted)
            t = (order.a * t + order.b) % total_tiles;
        const BatchReq rq = reqs[__ldg(tile_req + t)];
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

}  // namespace

namespace aesrt {

constexpr size_t kBatchSmem = aestt::kTableBytes;

cudaError_t batch_set_attributes()
{
    cudaError_t e = cudaFuncSetAttribute(batch_ttable_kernel<2, kRegsMaxThreads, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem);
    if (!e)
        e = cudaFuncSetAttribute(batch_ttable_kernel<2, 1024, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kBatchSmem);
    return e;
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

static int validate_batch_shape(BatchShape &s)
{
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
        if (opts->threads)
            s.threads = opts->threads;
        if (opts->tile_blocks)
            s.tile_blocks = opts->tile_blocks;
        if (opts->ctas)
            s.ctas = opts->ctas;
        if (opts->variant)
            s.variant = opts->variant;
    }
    return s;
}

// Tiles of a request: whole counter groups, tile_blocks / 256 per tile.
static uint64_t tiles_of(uint64_t len, uint32_t iv_low_byte, int tile_blocks)
{
    const uint64_t nb = (len + 15) / 16;
    if (!nb)
        return 0;
    const uint64_t groups = ((iv_low_byte + nb - 1) >> 8) + 1;
    const uint64_t per = (uint64_t)tile_blocks / 256u;
    return (groups + per - 1) / per;
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
    int ctas = s.ctas > 0 ? std::min(s.ctas, nsm) : nsm;
    if ((uint64_t)ctas > bt.total_tiles)
        ctas = (int)bt.total_tiles;
    const TileOrder order = make_order(bt.total_tiles, seed);
    const BatchReq *reqs = reinterpret_cast<const BatchReq *>(img);
    const uint32_t *map = reinterpret_cast<const uint32_t *>(img + im.off_map);
    unsigned long long *counter = reinterpret_cast<unsigned long long *>(img + im.off_counter);
    const uint32_t tg = (uint32_t)(s.tile_blocks / 256);
    if (s.threads <= kRegsMaxThreads)
        batch_ttable_kernel<2, kRegsMaxThreads, true>
            <<<ctas, s.threads, kBatchSmem, stream>>>(reqs, map, bt.total_tiles, counter, te0, tg, order);
    else
        batch_ttable_kernel<2, 1024, false>
            <<<ctas, s.threads, kBatchSmem, stream>>>(reqs, map, bt.total_tiles, counter, te0, tg, order);
    return cudaGetLastError();
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
