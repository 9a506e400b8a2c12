// server.cu -- served mode: a resident kernel polls a request queue in pinned,
// mapped host memory, so a request costs no kernel launch.
//
// The paper reroutes an offload through a server's own concurrency: submit
// the work to an executor, suspend the request, resume it on completion
// (Sec. 3), detecting completion by polling (Sec. 6 setup).  Here "submit" is
// offload_submit writing a descriptor and a queue entry, "suspend" is the
// ticket it returns at once, and "resume" is offload_poll observing the
// request's completion flag, which the GPU raises itself.
//
// Host -> device (all in pinned mapped memory):
//   descs[d]   request descriptor in slot d (pointers, length, IV, key slot, generation)
//   queue[i]   entry of request sequence number s at i = s mod Q: {tag = s + 1, d}; the tag
//              is stored last with release semantics
//   stop       set by offload_server_destroy
// Device -> host:
//   done[d]    (generation << 2) | status, stored with st.release.sys once the last tile
//              of the request in slot d is written (status 1 = OK, 2 = rejected)
//   kstatus    exit reasons of the resident CTAs (bit mask)
// Device-only state:
//   cursor     seq (28 bits) | slot d (16 bits) | next tile (20 bits) of the request
//              being cut into tiles; CTAs claim tiles with one atomicAdd
//   adv        sequence number an elected CTA is advancing the cursor to
//   recs[d]    validated copy of descs[d] with its tile count and a count of finished tiles
//
// Requests are taken in submission order, but their tiles run on every
// resident CTA at once, so requests that arrive while others are on the GPU
// start as soon as a CTA frees up (continuous batching).  Every wait on the
// device is bounded: a CTA with no work for idle_timeout exits (the host
// relaunches the kernel on the next submit or poll), and the stop flag ends
// all waits.
#include "../../include/aesoffload.h"
#include "internal.h"
#include "runtime.h"
#include "common.cuh"
#include "aes_ttable.cuh"
#include "tile.cuh"

#include <algorithm>
#include <chrono>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

namespace {

constexpr uint32_t kSeqMask = (1u << 28) - 1;
constexpr uint32_t kTileBits = 20;
constexpr uint32_t kMaxTiles = (1u << kTileBits) - 8192;  // headroom for exhausted claims
constexpr int kMaxSlots = 65535;
constexpr uint32_t kExitStop = 1, kExitIdle = 2, kExitError = 4;

struct HostDesc {  // 64 bytes, host-written
    uint64_t in, out, len, iv_hi, iv_lo, gen;
    uint32_t key_slot, flags;  // flags bit 0: the output is pinned host memory
    uint64_t pad1;
};
static_assert(sizeof(HostDesc) == 64, "HostDesc layout");

struct QEntry {
    uint64_t tag;   // sequence number + 1, stored last
    uint32_t desc;  // slot index
    uint32_t pad;
};

struct SrvRec {  // device-only, 128 bytes
    aesrt::BatchReq rq;
    unsigned long long seq_ntiles;  // (seq << 20) | ntiles, written after the rest
    unsigned long long gen;
    unsigned int done_tiles;
    unsigned int pad[11];
};
static_assert(sizeof(SrvRec) == 128, "SrvRec layout");

struct SrvParams {
    unsigned long long *cursor;
    unsigned long long *adv;
    SrvRec *recs;
    const uint4 *keys;          // max_keys x 15 round keys
    const int *key_nr;          // max_keys; 0 = unregistered
    const QEntry *queue;        // mapped
    const HostDesc *descs;      // mapped
    unsigned long long *done;   // mapped
    const unsigned int *stop;   // mapped
    unsigned int *kstatus;      // mapped
    const uint32_t *te0;
    uint32_t qmask, max_keys, tile_groups, nslots;
    uint64_t idle_ns, max_len;
};

__device__ __forceinline__ uint64_t gtime()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint64_t ld_acquire_sys(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t ld_relaxed_gpu(const unsigned long long *p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_gpu(unsigned long long *p, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_sys(unsigned long long *p, uint64_t v)
{
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_volatile(const unsigned int *p)
{
    return *reinterpret_cast<const volatile unsigned int *>(p);
}
__device__ __forceinline__ uint64_t ld_volatile64(const uint64_t *p)
{
    return *reinterpret_cast<const volatile uint64_t *>(p);
}

// Elected advancer: wait for request nseq = seq + 1 in the queue, validate
// and copy it into recs[d], then move the cursor to it.  Returns 0 or an
// exit code (after handing the advancer role back).
__device__ uint32_t advance(const SrvParams &p, uint32_t seq, uint64_t &last_work)
{
    const uint32_t nseq = (seq + 1) & kSeqMask;
    const uint32_t idx = nseq & p.qmask;
    const uint32_t want = (nseq + 1) & kSeqMask;
    for (;;) {
        const uint64_t tag = ld_acquire_sys(&p.queue[idx].tag);
        if ((uint32_t)(tag & kSeqMask) == want)
            break;
        uint32_t r = 0;
        if (ld_volatile(p.stop))
            r = kExitStop;
        else if (gtime() - last_work > p.idle_ns)
            r = kExitIdle;
        if (r) {
            atomicCAS(p.adv, (unsigned long long)nseq, (unsigned long long)seq);
            return r;
        }
        __nanosleep(128);
    }
    const uint32_t d = ld_volatile(&p.queue[idx].desc);
    if (d >= p.nslots)
        return kExitError;  // the host never writes such an entry
    const HostDesc *hd = p.descs + d;
    const uint64_t in = ld_volatile64(&hd->in), out = ld_volatile64(&hd->out);
    const uint64_t len = ld_volatile64(&hd->len), gen = ld_volatile64(&hd->gen);
    const uint32_t ks = ld_volatile(&hd->key_slot);
    int nr = 0;
    if (ks < p.max_keys)
        nr = __ldcg(p.key_nr + ks);
    bool ok = (nr == 10 || nr == 12 || nr == 14) && len <= p.max_len;
    if (ok && len)
        ok = in && out && !((in | out) & 15u);
    uint32_t ntiles = 0;
    const uint64_t iv_lo = ld_volatile64(&hd->iv_lo);
    if (ok && len) {
        // tiles are runs of tile_groups whole 256-block counter groups
        const uint64_t nb = (len + 15) >> 4;
        const uint64_t groups = (((iv_lo & 255u) + nb - 1) >> 8) + 1;
        ntiles = (uint32_t)((groups + p.tile_groups - 1) / p.tile_groups);
    }
    SrvRec *rec = p.recs + d;
    rec->rq.in = reinterpret_cast<const uint4 *>(in);
    rec->rq.out = reinterpret_cast<uint4 *>(out);
    rec->rq.len = len;
    rec->rq.iv_hi = ld_volatile64(&hd->iv_hi);
    rec->rq.iv_lo = iv_lo;
    rec->rq.rk = p.keys + 15u * (ok ? ks : 0u);
    rec->rq.nr = (uint32_t)nr;
    rec->rq.pad = ld_volatile(&hd->flags);
    rec->gen = gen;
    rec->done_tiles = 0;
    __threadfence();
    st_relaxed_gpu(&rec->seq_ntiles, ((uint64_t)nseq << kTileBits) | ntiles);
    __threadfence();
    unsigned long long cur = ld_relaxed_gpu(p.cursor);
    const unsigned long long nv = ((unsigned long long)nseq << 36) | ((unsigned long long)d << kTileBits);
    for (uint32_t it = 0;; ++it) {
        if ((uint32_t)(cur >> 36) != seq || it > (1u << 24))
            return kExitError;  // only the elected advancer moves the sequence number
        const unsigned long long old = atomicCAS(p.cursor, cur, nv);
        if (old == cur)
            break;
        cur = old;
    }
    if (ntiles == 0) {
        __threadfence_system();
        st_release_sys(p.done + d, (gen << 2) | (ok ? 1u : 2u));
    }
    last_work = gtime();
    return 0;
}

// Claim the next tile (thread 0 of a CTA).  Returns 0 with *d, *t set, or an
// exit code.
__device__ uint32_t acquire(const SrvParams &p, uint64_t &last_work, uint32_t *d_out, uint32_t *t_out)
{
    for (;;) {
        if (ld_volatile(p.stop))
            return kExitStop;
        const unsigned long long v = atomicAdd(p.cursor, 1ull);
        const uint32_t seq = (uint32_t)(v >> 36);
        const uint32_t d = (uint32_t)(v >> kTileBits) & 0xffffu;
        const uint32_t t = (uint32_t)v & ((1u << kTileBits) - 1);
        if (d < p.nslots) {
            const uint64_t sn = ld_relaxed_gpu(&p.recs[d].seq_ntiles);
            if ((uint32_t)(sn >> kTileBits) == seq && t < (uint32_t)(sn & ((1u << kTileBits) - 1))) {
                *d_out = d;
                *t_out = t;
                return 0;
            }
        }
        // The current request has no tiles left: advance, or wait for the
        // CTA that does.
        if (atomicCAS(p.adv, (unsigned long long)seq, (unsigned long long)((seq + 1) & kSeqMask)) == seq) {
            const uint32_t r = advance(p, seq, last_work);
            if (r)
                return r;
        } else {
            for (;;) {
                if ((uint32_t)(ld_relaxed_gpu(p.cursor) >> 36) != seq)
                    break;
                if ((uint32_t)ld_relaxed_gpu(p.adv) == seq)
                    break;  // the advancer gave up its role: compete for it again
                if (ld_volatile(p.stop))
                    return kExitStop;
                if (gtime() - last_work > p.idle_ns)
                    return kExitIdle;
                __nanosleep(128);
            }
        }
    }
}

__global__ void __launch_bounds__(512, 1) server_kernel(const __grid_constant__ SrvParams p)
{
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ uint4 s_rk[15];
    __shared__ int s_cmd;
    __shared__ uint32_t s_tile;
    aestt::fill_tables(smem, p.te0);
    const aestt::Lanes ln;
    uint64_t last_work = gtime();  // used by thread 0
    // Thread 0 claims a tile for the whole CTA (so at most one poller per
    // CTA touches the cursor); a tile is tile_groups counter groups, one per
    // warp by default, so the per-tile barrier waits for no straggler.
    for (;;) {
        if (threadIdx.x == 0) {
            uint32_t d = 0, t = 0;
            const uint32_t r = acquire(p, last_work, &d, &t);
            s_cmd = r ? -(int)r : (int)d;
            s_tile = t;
        }
        __syncthreads();  // also publishes the tables on the first pass
        const int cmd = s_cmd;
        if (cmd < 0) {
            if (threadIdx.x == 0)
                atomicOr_system(p.kstatus, (unsigned int)(-cmd));
            break;
        }
        SrvRec *rec = p.recs + cmd;
        aesrt::BatchReq rq;
        {
            const uint4 *src = reinterpret_cast<const uint4 *>(&rec->rq);
            uint4 *dst = reinterpret_cast<uint4 *>(&rq);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                dst[i] = __ldcg(src + i);
        }
        if (threadIdx.x <= rq.nr)
            s_rk[threadIdx.x] = __ldcg(rq.rk + threadIdx.x);
        const uint32_t tile = s_tile;
        __syncthreads();
        uint64_t first, last;
        aestile::tile_blocks_of(tile, p.tile_groups, rq.iv_lo & 255u, (rq.len + 15) >> 4, &first, &last);
        switch (rq.nr) {
        case 10: aestile::run_tile<10, 2>(rq, first, last, smem, ln, s_rk); break;
        case 12: aestile::run_tile<12, 2>(rq, first, last, smem, ln, s_rk); break;
        default: aestile::run_tile<14, 2>(rq, first, last, smem, ln, s_rk); break;
        }
        // Order this thread's output stores before the tile is counted: at
        // system scope when the output lives in host memory, else GPU scope
        // (the completing thread's system-scope release covers the rest).
        if (rq.pad & 1u)
            __threadfence_system();
        else
            __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            const uint32_t ntiles = (uint32_t)(ld_relaxed_gpu(&rec->seq_ntiles) & ((1u << kTileBits) - 1));
            const uint64_t gen = __ldcg(&rec->gen);
            const unsigned int prev = atomicAdd(&rec->done_tiles, 1u);
            if (prev + 1 == ntiles) {
                __threadfence_system();
                st_release_sys(p.done + cmd, (gen << 2) | 1u);
            }
            last_work = gtime();
        }
    }
}

}  // namespace

using namespace aesrt;

struct offload_server_s {
    int device = -1;
    int slots = 0, max_keys = 0, ctas = 0, threads = 0, tile_blocks = 0;
    uint32_t qsize = 0;
    uint64_t budget = 0, max_len = 0, idle_ns = 0;
    // mapped host memory
    HostDesc *descs = nullptr;
    QEntry *queue = nullptr;
    unsigned long long *done = nullptr;
    unsigned int *ctrl = nullptr;  // [0] stop, [1] kernel exit status
    // device memory
    uint8_t *dmem = nullptr;
    SrvParams params{};
    cudaStream_t stream = nullptr;
    cudaStream_t setup = nullptr;
    // host bookkeeping
    std::mutex mu;                 // free list, key table, launches
    std::vector<uint32_t> free_slots;
    std::vector<uint64_t> gen;     // per slot, current generation
    std::vector<uint64_t> bytes;   // per slot, budget charged
    std::unique_ptr<std::atomic<uint64_t>[]> live;  // per slot, live ticket (0 = free)
    std::vector<int> key_used;
    std::atomic<uint64_t> next_seq{1};
    std::atomic<uint64_t> inflight{0};
    std::atomic<bool> stopping{false};
    std::atomic<int> running{0};
    std::atomic<uint64_t> n_sub{0}, n_done{0}, n_again{0}, n_err{0}, n_relaunch{0}, n_bytes{0};
    uint32_t last_status = 0;
};

namespace {

int launch_resident(offload_server_s *s)
{
    s->ctrl[1] = 0;
    server_kernel<<<s->ctas, s->threads, aestt::kTableBytes, s->stream>>>(s->params);
    cudaError_t e = cudaGetLastError();
    if (e)
        return cuda_fail(e, "server_kernel launch");
    s->running.store(1);
    return AES_OK;
}

// Relaunch the resident kernel if every CTA has exited (idle timeout).
int ensure_running(offload_server_s *s)
{
    if (s->stopping.load())
        return AES_ESTOPPED;
    cudaError_t q = cudaStreamQuery(s->stream);
    if (q == cudaErrorNotReady)
        return AES_OK;
    std::lock_guard<std::mutex> lk(s->mu);
    q = cudaStreamQuery(s->stream);
    if (q == cudaErrorNotReady)
        return AES_OK;
    if (q != cudaSuccess)
        return cuda_fail(q, "resident kernel");
    s->last_status = s->ctrl[1];
    s->running.store(0);
    if (s->last_status & kExitError)
        return AES_ECUDA;
    s->n_relaunch.fetch_add(1);
    return launch_resident(s);
}

void release_slot(offload_server_s *s, uint32_t d)
{
    s->inflight.fetch_sub(s->bytes[d]);
    std::lock_guard<std::mutex> lk(s->mu);
    s->free_slots.push_back(d);
}

}  // namespace

extern "C" {

int offload_server_create(offload_server_t *out, const offload_cfg_t *cfg)
{
    if (!out)
        return AES_EINVAL;
    *out = nullptr;
    DeviceState *st = nullptr;
    int rc = device_state(&st);
    if (rc)
        return rc;
    offload_cfg_t c{};
    if (cfg)
        c = *cfg;
    const int slots = c.slots ? c.slots : 1024;
    const int max_keys = c.max_keys ? c.max_keys : 64;
    const int ctas = c.ctas ? c.ctas : std::max(1, st->nsm - 4);
    const int threads = c.threads ? c.threads : 512;
    const int tile_blocks = c.tile_blocks ? c.tile_blocks : 256 * (threads / 32);  // one group per warp
    if (slots < 1 || slots > kMaxSlots || max_keys < 1 || max_keys > (1 << 20) || ctas < 1 ||
        ctas > st->nsm || threads < 32 || threads > 512 || (threads & 31) || tile_blocks < 256 ||
        tile_blocks % 256 || tile_blocks > (1 << 22))
        return AES_EINVAL;
    offload_server_s *s = new (std::nothrow) offload_server_s();
    if (!s)
        return AES_ENOMEM;
    s->device = st->device;
    s->slots = slots;
    s->max_keys = max_keys;
    s->ctas = ctas;
    s->threads = threads;
    s->tile_blocks = tile_blocks;
    s->budget = c.hbm_budget;
    s->idle_ns = 1000ull * (c.idle_timeout_us ? c.idle_timeout_us : 200000u);
    s->max_len = std::min<uint64_t>(16ull << 30, ((uint64_t)kMaxTiles - 1) * (uint64_t)tile_blocks * 16u);
    uint32_t q = 1;
    while (q < (uint32_t)slots)
        q <<= 1;
    s->qsize = q;
    s->free_slots.reserve(slots);
    for (int i = slots - 1; i >= 0; --i)
        s->free_slots.push_back((uint32_t)i);
    s->gen.assign(slots, 0);
    s->bytes.assign(slots, 0);
    s->live.reset(new std::atomic<uint64_t>[slots]);
    for (int i = 0; i < slots; ++i)
        s->live[i].store(0);
    s->key_used.assign(max_keys, 0);

    cudaError_t e = cudaSuccess;
    auto fail = [&](const char *where) {
        if (s->stream)
            cudaStreamDestroy(s->stream);
        if (s->setup)
            cudaStreamDestroy(s->setup);
        cudaFree(s->dmem);
        cudaFreeHost(s->descs);
        cudaFreeHost(s->queue);
        cudaFreeHost(s->done);
        cudaFreeHost(s->ctrl);
        delete s;
        return e == cudaErrorMemoryAllocation ? AES_ENOMEM : cuda_fail(e, where);
    };
    const unsigned flags = cudaHostAllocMapped | cudaHostAllocPortable;
    if ((e = cudaHostAlloc(reinterpret_cast<void **>(&s->descs), sizeof(HostDesc) * slots, flags)))
        return fail("cudaHostAlloc(descs)");
    if ((e = cudaHostAlloc(reinterpret_cast<void **>(&s->queue), sizeof(QEntry) * q, flags)))
        return fail("cudaHostAlloc(queue)");
    if ((e = cudaHostAlloc(reinterpret_cast<void **>(&s->done), sizeof(unsigned long long) * slots, flags)))
        return fail("cudaHostAlloc(done)");
    if ((e = cudaHostAlloc(reinterpret_cast<void **>(&s->ctrl), 64, flags)))
        return fail("cudaHostAlloc(ctrl)");
    std::memset(s->descs, 0, sizeof(HostDesc) * slots);
    std::memset(s->queue, 0, sizeof(QEntry) * q);
    std::memset(s->done, 0, sizeof(unsigned long long) * slots);
    std::memset(s->ctrl, 0, 64);
    // device: [cursor, adv][recs][keys][key_nr]
    const size_t off_recs = 256;
    const size_t off_keys = off_recs + sizeof(SrvRec) * (size_t)slots;
    const size_t off_nr = off_keys + 240 * (size_t)max_keys;
    const size_t dbytes = off_nr + sizeof(int) * (size_t)max_keys;
    if ((e = cudaMalloc(&s->dmem, dbytes)))
        return fail("cudaMalloc(server)");
    if ((e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)))
        return fail("cudaStreamCreate");
    if ((e = cudaStreamCreateWithFlags(&s->setup, cudaStreamNonBlocking)))
        return fail("cudaStreamCreate");
    if ((e = cudaMemsetAsync(s->dmem, 0, dbytes, s->setup)) || (e = cudaStreamSynchronize(s->setup)))
        return fail("cudaMemset(server)");
    SrvParams &P = s->params;
    P.cursor = reinterpret_cast<unsigned long long *>(s->dmem);
    P.adv = reinterpret_cast<unsigned long long *>(s->dmem + 8);
    P.recs = reinterpret_cast<SrvRec *>(s->dmem + off_recs);
    P.keys = reinterpret_cast<const uint4 *>(s->dmem + off_keys);
    P.key_nr = reinterpret_cast<const int *>(s->dmem + off_nr);
    void *dp = nullptr;
    if ((e = cudaHostGetDevicePointer(&dp, s->queue, 0)))
        return fail("cudaHostGetDevicePointer");
    P.queue = static_cast<const QEntry *>(dp);
    if ((e = cudaHostGetDevicePointer(&dp, s->descs, 0)))
        return fail("cudaHostGetDevicePointer");
    P.descs = static_cast<const HostDesc *>(dp);
    if ((e = cudaHostGetDevicePointer(&dp, s->done, 0)))
        return fail("cudaHostGetDevicePointer");
    P.done = static_cast<unsigned long long *>(dp);
    if ((e = cudaHostGetDevicePointer(&dp, s->ctrl, 0)))
        return fail("cudaHostGetDevicePointer");
    P.stop = static_cast<const unsigned int *>(dp);
    P.kstatus = static_cast<unsigned int *>(dp) + 1;
    P.te0 = st->te0;
    P.qmask = q - 1;
    P.max_keys = (uint32_t)max_keys;
    P.tile_groups = (uint32_t)(tile_blocks / 256);
    P.nslots = (uint32_t)slots;
    P.idle_ns = s->idle_ns;
    P.max_len = s->max_len;
    if ((e = cudaFuncSetAttribute(server_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)aestt::kTableBytes)))
        return fail("cudaFuncSetAttribute(server)");
    rc = launch_resident(s);
    if (rc) {
        e = cudaErrorLaunchFailure;
        return fail("server launch");
    }
    *out = s;
    return AES_OK;
}

int offload_key_register(offload_server_t s, const uint8_t *key, int bits, int *slot_out)
{
    if (!s || !key || !slot_out)
        return AES_EINVAL;
    if (bits != 128 && bits != 192 && bits != 256)
        return AES_EKEYBITS;
    DeviceState *st = nullptr;
    int rc = device_state(&st);
    if (rc)
        return rc;
    std::lock_guard<std::mutex> lk(s->mu);
    int slot = -1;
    for (int i = 0; i < s->max_keys; ++i)
        if (!s->key_used[i]) {
            slot = i;
            break;
        }
    if (slot < 0)
        return AES_ETOOBIG;
    uint8_t *stage = nullptr;
    cudaError_t e = cudaMalloc(&stage, 64);
    if (e)
        return e == cudaErrorMemoryAllocation ? AES_ENOMEM : cuda_fail(e, "cudaMalloc(key stage)");
    uint8_t h[64] = {0};
    std::memcpy(h, key, bits / 8);
    const int32_t b = bits;
    std::memcpy(h + 32, &b, 4);
    const int nr = bits / 32 + 6;
    uint32_t *w = reinterpret_cast<uint32_t *>(const_cast<uint4 *>(s->params.keys + 15u * slot));
    e = cudaMemcpyAsync(stage, h, 64, cudaMemcpyHostToDevice, s->setup);
    if (!e)
        e = launch_key_expand(stage, reinterpret_cast<const int32_t *>(stage + 32), st->te0, w, 1, s->setup);
    if (!e)
        e = cudaMemcpyAsync(const_cast<int *>(s->params.key_nr) + slot, &nr, sizeof(int),
                            cudaMemcpyHostToDevice, s->setup);
    if (!e)
        e = cudaStreamSynchronize(s->setup);
    cudaFree(stage);
    if (e)
        return cuda_fail(e, "offload_key_register");
    s->key_used[slot] = 1;
    *slot_out = slot;
    return AES_OK;
}

int offload_submit(offload_server_t s, int key_slot, const uint8_t *iv, const void *in, void *out,
                   size_t len, uint64_t *ticket)
{
    if (!s || !iv || !ticket)
        return AES_EINVAL;
    if (s->stopping.load())
        return AES_ESTOPPED;
    if (key_slot < 0 || key_slot >= s->max_keys || !s->key_used[key_slot])
        return AES_EINVAL;
    if (len > s->max_len)
        return AES_ETOOBIG;
    const void *din = nullptr;
    void *dout = nullptr;
    bool out_host = false;
    if (len) {
        int rc = check_payload(in, out, len, s->device, &din, &dout, &out_host);
        if (rc)
            return rc;
    }
    const uint64_t charge = len == 0 ? 0 : (in == out ? (uint64_t)len : 2ull * len);
    if (s->budget && charge > s->budget)
        return AES_ETOOBIG;
    // admission: budget, then a free slot
    if (s->budget) {
        uint64_t cur = s->inflight.load();
        do {
            if (cur + charge > s->budget) {
                s->n_again.fetch_add(1);
                return AES_EAGAIN;
            }
        } while (!s->inflight.compare_exchange_weak(cur, cur + charge));
    } else {
        s->inflight.fetch_add(charge);
    }
    uint32_t d;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->free_slots.empty()) {
            s->inflight.fetch_sub(charge);
            s->n_again.fetch_add(1);
            return AES_EAGAIN;
        }
        d = s->free_slots.back();
        s->free_slots.pop_back();
    }
    const uint64_t gen = ++s->gen[d];
    s->bytes[d] = charge;
    HostDesc &hd = s->descs[d];
    hd.in = (uint64_t)(uintptr_t)din;
    hd.out = (uint64_t)(uintptr_t)dout;
    hd.len = len;
    iv_halves(iv, &hd.iv_hi, &hd.iv_lo);
    hd.gen = gen;
    hd.key_slot = (uint32_t)key_slot;
    hd.flags = out_host ? 1u : 0u;
    const uint64_t tk = (gen << 16) | d;
    s->live[d].store(tk);
    const uint64_t seq = s->next_seq.fetch_add(1);
    QEntry &qe = s->queue[seq & (s->qsize - 1)];
    qe.desc = d;
    __atomic_store_n(&qe.tag, seq + 1, __ATOMIC_RELEASE);
    s->n_sub.fetch_add(1);
    *ticket = tk;
    const int rc = ensure_running(s);
    return rc == AES_ESTOPPED ? AES_OK : rc;
}

int offload_poll(offload_server_t s, uint64_t ticket)
{
    if (!s)
        return AES_EINVAL;
    const uint32_t d = (uint32_t)(ticket & 0xffffu);
    const uint64_t gen = ticket >> 16;
    if ((int)d >= s->slots || gen == 0 || s->live[d].load() != ticket)
        return AES_EINVAL;
    const uint64_t v = __atomic_load_n(&s->done[d], __ATOMIC_ACQUIRE);
    if ((v >> 2) != gen) {
        if (s->stopping.load())
            return AES_ESTOPPED;
        const int rc = ensure_running(s);
        return rc ? rc : AES_PENDING;
    }
    uint64_t expect = ticket;
    if (!s->live[d].compare_exchange_strong(expect, 0))
        return AES_EINVAL;  // another thread released it first
    const uint32_t status = (uint32_t)(v & 3u);
    const uint64_t nbytes = s->descs[d].len;
    release_slot(s, d);
    if (status != 1) {
        s->n_err.fetch_add(1);
        return AES_EDESC;
    }
    s->n_done.fetch_add(1);
    s->n_bytes.fetch_add(nbytes);
    return AES_OK;
}

int offload_wait(offload_server_t s, uint64_t ticket, uint64_t timeout_us)
{
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const int rc = offload_poll(s, ticket);
        if (rc != AES_PENDING)
            return rc;
        const auto us = std::chrono::duration_cast<std::chrono::microseconds>(
                            std::chrono::steady_clock::now() - t0).count();
        if ((uint64_t)us >= timeout_us)
            return AES_ETIMEOUT;
    }
}

int offload_server_stats(offload_server_t s, offload_stats_t *out)
{
    if (!s || !out)
        return AES_EINVAL;
    out->submitted = s->n_sub.load();
    out->completed = s->n_done.load();
    out->rejected_eagain = s->n_again.load();
    out->device_errors = s->n_err.load();
    out->relaunches = s->n_relaunch.load();
    out->bytes_completed = s->n_bytes.load();
    const cudaError_t q = cudaStreamQuery(s->stream);
    out->running = q == cudaErrorNotReady ? 1 : 0;
    out->kernel_status = out->running ? s->last_status : s->ctrl[1];
    return AES_OK;
}

int offload_server_destroy(offload_server_t s)
{
    if (!s)
        return AES_OK;
    s->stopping.store(true);
    __atomic_store_n(&s->ctrl[0], 1u, __ATOMIC_RELEASE);
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t q = cudaStreamQuery(s->stream);
        if (q != cudaErrorNotReady)
            break;
        if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(5))
            return AES_ETIMEOUT;  // leak rather than free under a running kernel
        std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
    cudaStreamSynchronize(s->setup);
    cudaStreamDestroy(s->stream);
    cudaStreamDestroy(s->setup);
    cudaFree(s->dmem);
    cudaFreeHost(s->descs);
    cudaFreeHost(s->queue);
    cudaFreeHost(s->done);
    cudaFreeHost(s->ctrl);
    delete s;
    return AES_OK;
}

}  // extern "C"
