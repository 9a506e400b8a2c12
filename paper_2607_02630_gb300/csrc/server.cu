// server.cu -- served mode: a resident kernel polls a request queue in pinned,
// mapped host memory, so a request costs no kernel launch.
//
// The paper reroutes an offload through a server's own concurrency: submit
// the work to an executor, suspend the request, resume it on completion
// (Sec. 3), detecting completion by polling (Sec. 6 setup).  Here "submit" is
// offload_submit writing a queue entry, "suspend" is the ticket it returns at
// once, and "resume" is offload_poll observing the request's completion flag,
// which the GPU raises itself.
//
// Host -> device (pinned mapped memory):
//   queue[d]   body of the request in descriptor slot d (64 bytes): payload
//              pointers, length, IV, key slot, generation, flags
//   order[i]   ((s + 1) << 16) | d for request sequence number s at
//              i = s mod Q, stored (release) after the body: one load gives
//              the device a request's slot, and the body stays put until the
//              request completes
//   stop       set by offload_server_destroy
// Device -> host:
//   done[d]    (generation << 2) | status, stored with st.release.sys once the last tile
//              of the request in slot d is written (status 1 = OK, 2 = rejected)
//   kstatus    exit reasons of the resident CTAs (bit mask)
// Device-only state:
//   cursor     seq (28 bits) | slot d (16 bits) | next tile (20 bits) of the request
//              being cut into tiles; tiles are claimed with atomicAdd
//   adv        sequence number an elected CTA is advancing the cursor to
//   disp       next sequence number to dispatch (validate into recs)
//   disp_ring  (seq, slot, tile count) of the last 64 dispatched requests,
//              written once their records are complete
//   recs[d]    validated copy of the request in slot d, its tile count and a count of
//              finished tiles
//
// Each resident CTA is warp-specialised: warp 0 is the agent, the others are
// workers.  The agent alone touches the global cursor: it claims tiles in
// batches (as many as its workers are waiting for, plus a prefetch) and hands
// them to the workers through a ring in shared memory.  Requests are
// dispatched ahead of the cursor, in order, up to 4 per round trip over the
// host link (tags read together, claimed with one CAS on disp).  When a claim
// takes a request's last tiles, or a claim finds none left, that agent (one,
// elected through adv) moves the cursor to the next request as soon as its
// dispatch-ring entry is published, and dispatches what is queued behind it.
// A tile is tile_groups counter groups of one request and is encrypted by one
// worker warp, so a request is spread over many SMs at once and requests that
// arrive while others are on the GPU start as soon as an agent asks for work
// (continuous batching).  Every wait on the device is bounded: an agent with
// no new work for idle_timeout exits and its workers follow once the ring is
// drained (the host relaunches the kernel on the next submit or poll), and
// the stop flag ends every wait.
//
// claim_mode 1 replaces the global cursor with a claim word per request
// record: agents walk the dispatched requests in order on their own, so
// several requests are cut into tiles at once (cursor then holds `low`, the
// oldest request that may have unclaimed tiles).  The protocol -- layouts,
// dispatch, both claim modes, the agent loop, the agent-worker ring and
// completion -- is in served_protocol.cuh, which also compiles for host
// threads; this file holds the kernel (the workers' tile loop) and the host
// side.
#include "../../include/aesoffload.h"
#include "internal.h"
#include "runtime.h"
#include "common.cuh"
#include "aes_ttable.cuh"
#include "tile.cuh"
#include "served_protocol.cuh"

#include <algorithm>
#include <chrono>
#include <cstddef>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

namespace {

using namespace srvp;

// Round keys in registers, read through L2 (coherent): the resident kernel
// outlives key registrations, and adjacent 240-byte key slots share cache
// lines, so a non-coherent (read-only path) copy of a line could predate a
// key registered after it was cached.
template <int NR>
struct RkRegsL2 {
    uint4 w[NR + 1];
    __device__ __forceinline__ explicit RkRegsL2(const uint4 *g)
    {
#pragma unroll
        for (int r = 0; r <= NR; ++r)
            w[r] = __ldcg(g + r);
    }
    __device__ __forceinline__ uint4 get(int r) const { return w[r]; }
};

// Part `part` of `parts` of the single counter group [first, last) (or the
// whole tile when parts == 1) of a request, done by the calling warp alone,
// with the request's round keys in registers.
// (stamp: trace builds record when the keys have arrived)
template <int NR, int NB>
__device__ __forceinline__ void run_part_regs(const aesrt::BatchReq &rq, uint64_t first, uint64_t last,
                                              uint32_t part, uint32_t parts, const uint8_t *smem,
                                              const aestt::Lanes &ln, const SrvParams &p, uint32_t seq, bool stamp)
{
    const RkRegsL2<NR> rk(rq.rk);
#ifdef SRV_TRACE
    if (stamp) {  // a move that reads the last round key waits for it, then the stamp
        uint32_t sink;
        asm volatile("mov.b32 %0, %1;" : "=r"(sink) : "r"(rk.get(NR).x));
        trace(p, seq, kTrKeysLoaded);
    }
#else
    (void)p;
    (void)seq;
    (void)stamp;
#endif
    aestile::xor_range<NR, NB>(rq.in, rq.out, rq.len, rq.iv_hi, rq.iv_lo, first, last, part, parts, parts, smem,
                               ln, rk);
}

template <bool PER_REQ>
__global__ void __launch_bounds__(512, 1) server_kernel(const __grid_constant__ SrvParams p)
{
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ Ring ring;
    if (threadIdx.x == 0)
        ring_init(ring);
    aestt::fill_tables(smem, p.te0);
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    if (warp == 0) {
        if (lane == 0) {
            agent<PER_REQ>(p, ring);
            if (ring.exit_code)
                atomicOr_system(p.kstatus, ring.exit_code);
        }
        return;  // no CTA-wide barrier follows
    }
    const aestt::Lanes ln;
    uint32_t cur_d = ~0u, cur_seq = ~0u, tg = 1, tp = 1;
    uint64_t gen = 0;
    aesrt::BatchReq rq;
    for (;;) {
        uint32_t d = 0, t = 0, seq = 0, nt = 0;
        if (!ring_pop_warp(ring, &d, &t, &seq, &nt))
            break;
        if (lane == 0 && t == 0)
            trace(p, seq, kTrFirstPop);
        SrvRec *rec = p.recs + d;
        if (d != cur_d || seq != cur_seq) {  // a new request for this warp: load it and its keys
            // the request (64 bytes), then seq_ntiles/gen and the tile shape:
            // one 128-byte line, six independent loads
            const uint4 *src = reinterpret_cast<const uint4 *>(&rec->rq);
            uint4 *dst = reinterpret_cast<uint4 *>(&rq);
            uint4 w[6];
#pragma unroll
            for (int i = 0; i < 6; ++i)
                w[i] = __ldcg(src + i);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                dst[i] = w[i];
            static_assert(offsetof(SrvRec, gen) == 72 && offsetof(SrvRec, tile_groups) == 80 &&
                              offsetof(SrvRec, tile_parts) == 84,
                          "record words read as uint4 4 and 5");
            gen = ((uint64_t)w[4].w << 32) | w[4].z;
            tg = w[5].x;
            tp = w[5].y;
            __syncwarp();
#ifdef SRV_TRACE
            if (lane == 0 && t == 0) {  // a move that reads the record waits for it, then the stamp
                uint64_t sink;
                asm volatile("mov.b64 %0, %1;" : "=l"(sink) : "l"(rq.len));
                trace(p, seq, kTrRecLoaded);
            }
#endif
            cur_d = d;
            cur_seq = seq;
        }
        if (rq.pad & kFlagEmulated) {
            // emulated offload: hold this warp for rq.len ns (at most kMaxEmulatedNs)
            if (lane == 0) {
                const uint64_t t0 = gtime();
                for (;;) {
                    const int64_t el = since(t0);
                    if (el >= (int64_t)rq.len || el < 0)  // done, or the timer stepped back
                        break;
                    __nanosleep(256);
                }
            }
            __syncwarp();
        } else {
            uint64_t first, last;
            const uint32_t part = t % tp;
            aestile::tile_blocks_of(t / tp, tg, rq.iv_lo & 255u, (rq.len + 15) >> 4, &first, &last);
            switch (rq.nr) {
            case 10: run_part_regs<10, 2>(rq, first, last, part, tp, smem, ln, p, seq, lane == 0 && t == 0); break;
            case 12: run_part_regs<12, 2>(rq, first, last, part, tp, smem, ln, p, seq, lane == 0 && t == 0); break;
            default: run_part_regs<14, 2>(rq, first, last, part, tp, smem, ln, p, seq, lane == 0 && t == 0); break;
            }
        }
        // Order the tile's output stores before it is counted: a warp
        // barrier gathers every lane's stores under lane 0, whose
        // acquire-release add publishes them (GPU scope) to the worker that
        // raises the completion word with a system-scope release.  Outputs
        // in host memory are fenced at system scope by every lane first.
        if (rq.pad & kFlagHostOut)
            __threadfence_system();
        __syncwarp();
        if (lane == 0 && t == 0)
            trace(p, seq, kTrFirstTileDone);
        if (lane == 0)
            tile_finished(p, d, nt, seq, gen);
    }
}

}  // namespace

using namespace aesrt;

struct offload_server_s {
    int device = -1;
    int slots = 0, max_keys = 0, ctas = 0, threads = 0, tile_blocks = 0;
    int claim_mode = 0;  // 0: global cursor, 1: per-request claims
    int trace_requests = 0;
    unsigned long long *trace = nullptr;  // device stamp buffer (trace builds)
    uint32_t qsize = 0;
    uint64_t budget = 0, max_len = 0, idle_ns = 0;
    // mapped host memory
    QEntry *queue = nullptr;       // one body per descriptor slot
    uint64_t *order = nullptr;     // qsize order words
    unsigned long long *done = nullptr;
    unsigned int *ctrl = nullptr;  // [0] stop, [1] kernel exit status
    // device memory
    uint8_t *dmem = nullptr;
    uint8_t *key_stage = nullptr;  // 64 bytes in dmem: key + bits for one registration (under mu)
    SrvParams params{};
    cudaStream_t stream = nullptr;
    cudaStream_t setup = nullptr;
    // host bookkeeping
    std::mutex mu;                 // free list, key table, launches
    std::vector<uint32_t> free_slots;
    std::vector<uint64_t> gen;     // per slot, current generation
    std::vector<uint64_t> bytes;   // per slot, budget charged
    std::vector<uint64_t> lens;    // per slot, payload length
    std::unique_ptr<std::atomic<uint64_t>[]> live;  // per slot, live ticket (0 = free)
    std::vector<int> key_used;
    std::vector<uint8_t> key_nr;   // per key slot, Nr of its key (sent with each request)
    std::atomic<uint64_t> next_seq{1};
    std::atomic<uint64_t> inflight{0};
    std::atomic<bool> stopping{false};
    std::atomic<uint64_t> n_sub{0}, n_done{0}, n_again{0}, n_err{0}, n_relaunch{0}, n_bytes{0};
    uint32_t last_status = 0;
    std::atomic<int64_t> next_query_ns{0};  // when the kernel's stream is queried next
};

namespace {

int launch_resident(offload_server_s *s)
{
    s->ctrl[1] = 0;
    if (s->claim_mode)
        server_kernel<true><<<s->ctas, s->threads, aestt::kTableBytes, s->stream>>>(s->params);
    else
        server_kernel<false><<<s->ctas, s->threads, aestt::kTableBytes, s->stream>>>(s->params);
    cudaError_t e = cudaGetLastError();
    if (e)
        return cuda_fail(e, "server_kernel launch");
    return AES_OK;
}

// Relaunch the resident kernel if every CTA has exited (idle timeout).
int ensure_running(offload_server_s *s)
{
    if (s->stopping.load())
        return AES_ESTOPPED;
    // CTAs raise their exit reason in the mapped status word before they
    // end, so while it is clear the kernel is running -- unless it died on
    // a fault, which only a stream query shows: query at most every 1 ms.
    const int64_t now = std::chrono::duration_cast<std::chrono::nanoseconds>(
                            std::chrono::steady_clock::now().time_since_epoch()).count();
    if (__atomic_load_n(&s->ctrl[1], __ATOMIC_ACQUIRE) == 0) {
        int64_t next = s->next_query_ns.load();
        if (now < next || !s->next_query_ns.compare_exchange_strong(next, now + 1000000))
            return AES_OK;
    }
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

// Admission (HBM budget, then a free slot), the body of one request in its
// slot and, stored last with release semantics, its order word.  Submitters
// may race: if the order word of seq s is not stored yet, the device waits
// at s, so every later request stays in flight holding a slot and s +
// qsize cannot be admitted before that word has been read.
int enqueue(offload_server_s *s, uint32_t key_slot, uint64_t iv_hi, uint64_t iv_lo, const void *din, void *dout,
            uint64_t len, uint32_t flags, uint64_t charge, uint64_t *ticket)
{
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
    s->lens[d] = flags & kFlagEmulated ? 0 : len;
    const uint64_t tk = (gen << 16) | d;
    s->live[d].store(tk);
    // The body goes to the request's own slot, which it holds until it
    // completes.  Its order word reuses the one of seq - qsize: a slot is
    // admitted only while fewer than `slots` requests are in flight and the
    // device reads order words in sequence order, so that word (qsize >=
    // slots) has been read already.
    const uint64_t seq = s->next_seq.fetch_add(1);
    QEntry &qe = s->queue[d];
    qe.in = (uint64_t)(uintptr_t)din;
    qe.out = (uint64_t)(uintptr_t)dout;
    qe.len = len;
    qe.iv_hi = iv_hi;
    qe.iv_lo = iv_lo;
    qe.gen = gen;
    qe.key_slot = key_slot | (uint32_t)s->key_nr[key_slot] << 24;
    qe.desc = (uint16_t)d;
    qe.flags = (uint16_t)flags;
    qe.tag = seq + 1;
    __atomic_store_n(&s->order[seq & (s->qsize - 1)], ((seq + 1) << 16) | d, __ATOMIC_RELEASE);
    s->n_sub.fetch_add(1);
    *ticket = tk;
    const int rc = ensure_running(s);
    return rc == AES_ESTOPPED ? AES_OK : rc;
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
    const int tile_blocks = c.tile_blocks;  // 0: chosen per request
    // warp 0 of each CTA is the agent, so at least one worker warp is needed
    if (slots < 1 || slots > kMaxSlots || max_keys < 1 || max_keys > (1 << 20) || ctas < 1 ||
        ctas > st->nsm || threads < 64 || threads > 32 * kMaxWarps || (threads & 31) ||
        !(tile_blocks == 0 || tile_blocks == 64 || tile_blocks == 128 ||
          (tile_blocks >= 256 && tile_blocks % 256 == 0)) ||
        tile_blocks > (1 << 22) || c.claim_mode < 0 || c.claim_mode > 1 || c.trace_requests < 0 ||
        c.trace_requests > (1 << 20) || (c.trace_requests & (c.trace_requests - 1)))
        return AES_EINVAL;
#ifndef SRV_TRACE
    if (c.trace_requests)
        return AES_EINVAL;  // this build has no stamps to record
#endif
    offload_server_s *s = new (std::nothrow) offload_server_s();
    if (!s)
        return AES_ENOMEM;
    s->device = st->device;
    s->slots = slots;
    s->max_keys = max_keys;
    s->ctas = ctas;
    s->threads = threads;
    s->tile_blocks = tile_blocks;
    s->claim_mode = c.claim_mode;
    s->trace_requests = c.trace_requests;
    s->budget = c.hbm_budget;
    s->idle_ns = 1000ull * (c.idle_timeout_us ? c.idle_timeout_us : 200000u);
    // tiles of at least 64 blocks (1024 adaptive for long requests) keep the tile count < kMaxTiles
    s->max_len = std::min<uint64_t>(16ull << 30, ((uint64_t)kMaxTiles - 1) *
                                                   (uint64_t)(tile_blocks ? tile_blocks : 1024) * 16u);
    uint32_t q = 1;
    while (q < (uint32_t)slots)
        q <<= 1;
    s->qsize = q;
    s->free_slots.reserve(slots);
    for (int i = slots - 1; i >= 0; --i)
        s->free_slots.push_back((uint32_t)i);
    s->gen.assign(slots, 0);
    s->bytes.assign(slots, 0);
    s->lens.assign(slots, 0);
    s->live.reset(new std::atomic<uint64_t>[slots]);
    for (int i = 0; i < slots; ++i)
        s->live[i].store(0);
    s->key_used.assign(max_keys, 0);
    s->key_nr.assign(max_keys, 0);

    cudaError_t e = cudaSuccess;
    auto fail = [&](const char *where) {
        if (s->stream)
            cudaStreamDestroy(s->stream);
        if (s->setup)
            cudaStreamDestroy(s->setup);
        cudaFree(s->dmem);
        cudaFree(s->trace);
        cudaFreeHost(s->queue);
        cudaFreeHost(s->order);
        cudaFreeHost(s->done);
        cudaFreeHost(s->ctrl);
        delete s;
        return e == cudaErrorMemoryAllocation ? AES_ENOMEM : cuda_fail(e, where);
    };
    const unsigned flags = cudaHostAllocMapped | cudaHostAllocPortable;
    if ((e = cudaHostAlloc(reinterpret_cast<void **>(&s->queue), sizeof(QEntry) * (size_t)slots, flags)))
        return fail("cudaHostAlloc(queue)");
    if ((e = cudaHostAlloc(reinterpret_cast<void **>(&s->order), sizeof(uint64_t) * q, flags)))
        return fail("cudaHostAlloc(order)");
    if ((e = cudaHostAlloc(reinterpret_cast<void **>(&s->done), sizeof(unsigned long long) * slots, flags)))
        return fail("cudaHostAlloc(done)");
    if ((e = cudaHostAlloc(reinterpret_cast<void **>(&s->ctrl), 64, flags)))
        return fail("cudaHostAlloc(ctrl)");
    std::memset(s->queue, 0, sizeof(QEntry) * (size_t)slots);
    std::memset(s->order, 0, sizeof(uint64_t) * q);
    std::memset(s->done, 0, sizeof(unsigned long long) * slots);
    std::memset(s->ctrl, 0, 64);
    // device: cursor, adv and disp each on a 4 KiB page of their own (every
    // agent polls them), then disp_ring, recs, keys and the key staging area
    // (registration allocates nothing: cudaFree would wait for the resident
    // kernel to exit)
    const size_t off_adv = 4096, off_disp = 8192, off_slots = 12288;
    const size_t off_recs = 16384;
    static_assert(8 * kDispRing <= 4096, "disp_ring fits in its page");
    const size_t off_keys = off_recs + sizeof(SrvRec) * (size_t)slots;
    const size_t off_stage = (off_keys + 240 * (size_t)max_keys + 255) / 256 * 256;
    const size_t dbytes = off_stage + 64;
    if ((e = cudaMalloc(&s->dmem, dbytes)))
        return fail("cudaMalloc(server)");
    if ((e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)))
        return fail("cudaStreamCreate");
    if ((e = cudaStreamCreateWithFlags(&s->setup, cudaStreamNonBlocking)))
        return fail("cudaStreamCreate");
    const unsigned long long first_seq = 1;  // request sequence numbers start at 1
    // per-request claims: the cursor word is low, the oldest request that
    // may have unclaimed tiles, and starts at the first sequence number
    if ((e = cudaMemsetAsync(s->dmem, 0, dbytes, s->setup)) ||
        (e = cudaMemcpyAsync(s->dmem + off_disp, &first_seq, 8, cudaMemcpyHostToDevice, s->setup)) ||
        (s->claim_mode && (e = cudaMemcpyAsync(s->dmem, &first_seq, 8, cudaMemcpyHostToDevice, s->setup))) ||
        (e = cudaStreamSynchronize(s->setup)))
        return fail("cudaMemset(server)");
    SrvParams &P = s->params;
    P.cursor = reinterpret_cast<unsigned long long *>(s->dmem);
    P.adv = reinterpret_cast<unsigned long long *>(s->dmem + off_adv);
    P.disp = reinterpret_cast<unsigned long long *>(s->dmem + off_disp);
    P.disp_ring = reinterpret_cast<unsigned long long *>(s->dmem + off_slots);
    P.recs = reinterpret_cast<SrvRec *>(s->dmem + off_recs);
    P.keys = reinterpret_cast<const uint4 *>(s->dmem + off_keys);
    s->key_stage = s->dmem + off_stage;
    if (s->trace_requests) {
        const size_t tb = sizeof(unsigned long long) * kTracePoints * (size_t)s->trace_requests;
        if ((e = cudaMalloc(reinterpret_cast<void **>(&s->trace), tb)) ||
            (e = cudaMemsetAsync(s->trace, 0, tb, s->setup)) || (e = cudaStreamSynchronize(s->setup)))
            return fail("trace buffer");
        P.trace = s->trace;
        P.trace_mask = (uint32_t)s->trace_requests - 1;
    }
    void *dp = nullptr;
    if ((e = cudaHostGetDevicePointer(&dp, s->queue, 0)))
        return fail("cudaHostGetDevicePointer");
    P.queue = static_cast<const QEntry *>(dp);
    if ((e = cudaHostGetDevicePointer(&dp, s->order, 0)))
        return fail("cudaHostGetDevicePointer");
    P.order = static_cast<const uint64_t *>(dp);
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
    P.tile_blocks = (uint32_t)tile_blocks;
    P.nslots = (uint32_t)slots;
    P.nctas = (uint32_t)ctas;
    P.idle_ns = s->idle_ns;
    P.max_len = s->max_len;
    if ((e = cudaFuncSetAttribute(server_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)aestt::kTableBytes)) ||
        (e = cudaFuncSetAttribute(server_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
    uint8_t *stage = s->key_stage;
    uint8_t h[64] = {0};
    std::memcpy(h, key, bits / 8);
    const int32_t b = bits;
    std::memcpy(h + 32, &b, 4);
    const int nr = bits / 32 + 6;
    uint32_t *w = reinterpret_cast<uint32_t *>(const_cast<uint4 *>(s->params.keys + 15u * slot));
    cudaError_t e = cudaMemcpyAsync(stage, h, 64, cudaMemcpyHostToDevice, s->setup);
    if (!e)
        e = launch_key_expand(stage, reinterpret_cast<const int32_t *>(stage + 32), st->te0, w, 1, s->setup);
    if (!e)
        e = cudaStreamSynchronize(s->setup);
    if (e)
        return cuda_fail(e, "offload_key_register");
    s->key_nr[slot] = (uint8_t)nr;
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
    uint64_t iv_hi = 0, iv_lo = 0;
    iv_halves(iv, &iv_hi, &iv_lo);
    return enqueue(s, (uint32_t)key_slot, iv_hi, iv_lo, din, dout, len, out_host ? kFlagHostOut : 0u, charge,
                   ticket);
}

int offload_submit_emulated(offload_server_t s, uint64_t duration_ns, uint64_t *ticket)
{
    if (!s || !ticket || duration_ns > kMaxEmulatedNs)
        return AES_EINVAL;
    if (s->stopping.load())
        return AES_ESTOPPED;
    return enqueue(s, 0, 0, 0, nullptr, nullptr, duration_ns, kFlagEmulated, 0, ticket);
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
    const uint64_t nbytes = s->lens[d];
    release_slot(s, d);
    if (status != 1) {
        s->n_err.fetch_add(1);
        return AES_EDESC;
    }
    s->n_done.fetch_add(1);
    s->n_bytes.fetch_add(nbytes);
    return AES_OK;
}

int offload_poll_many(offload_server_t s, const uint64_t *tickets, int n, int *status, uint64_t timeout_us)
{
    if (!s || n < 0 || (n > 0 && (!tickets || !status)))
        return AES_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        int done = 0;
        for (int i = 0; i < n; ++i) {
            status[i] = offload_poll(s, tickets[i]);
            done += status[i] != AES_PENDING;
        }
        if (done || n == 0)
            return done;
        const auto us = std::chrono::duration_cast<std::chrono::microseconds>(
                            std::chrono::steady_clock::now() - t0).count();
        if ((uint64_t)us >= timeout_us)
            return 0;
    }
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

int offload_server_trace(offload_server_t s, uint64_t *out, size_t max_words)
{
    static_assert(kTracePoints == AES_TRACE_POINTS, "trace points");
    if (!s || !out || !s->trace)
        return AES_EINVAL;
    size_t n = (size_t)kTracePoints * (size_t)s->trace_requests;
    if (n > max_words)
        n = max_words;
    cudaError_t e = cudaMemcpyAsync(out, s->trace, n * sizeof(uint64_t), cudaMemcpyDeviceToHost, s->setup);
    if (!e)
        e = cudaStreamSynchronize(s->setup);
    if (e)
        return cuda_fail(e, "offload_server_trace");
    return (int)n;
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
    out->kernel_status = __atomic_load_n(&s->ctrl[1], __ATOMIC_ACQUIRE);
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
    cudaFree(s->trace);
    cudaFreeHost(s->queue);
    cudaFreeHost(s->order);
    cudaFreeHost(s->done);
    cudaFreeHost(s->ctrl);
    delete s;
    return AES_OK;
}

}  // extern "C"
