// served_protocol.cuh -- the request protocol of the served kernel: queue
// entry and record layouts, dispatch of queued requests into device
// records, the two ways agents claim tiles (one global cursor moved from
// request to request; per-request claim words), and the completion of a
// request's last tile.
//
// The same source compiles for the device (nvcc: PTX memory operations at
// the scopes the protocol needs) and for the host (GCC atomics on plain
// memory).  Host threads standing in for the resident CTAs can then run the
// protocol's logic -- every tile claimed once, every request completed once,
// slot reuse, idle exits and relaunches -- without a GPU.  A host run checks
// logic only: CPUs order memory differently from the GPU.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "internal.h"

#ifdef __CUDACC__
#define SRV_INLINE __device__ __forceinline__
#define SRV_NOINLINE __device__ __noinline__
#define SRV_FN __device__
#else
#include <atomic>
#include <chrono>
#include <cstring>
#include <thread>
#include <vector>
#define SRV_INLINE inline
#define SRV_NOINLINE inline
#define SRV_FN inline
#endif

namespace srvp {

constexpr uint32_t kSeqMask = (1u << 28) - 1;
constexpr uint32_t kTileBits = 20;
constexpr uint32_t kTileMask = (1u << kTileBits) - 1;
constexpr uint32_t kMaxTiles = (1u << kTileBits) - 16384;  // headroom for batched exhausted claims
constexpr int kMaxSlots = 65535;
constexpr uint32_t kExitStop = 1, kExitIdle = 2, kExitError = 4;
constexpr uint32_t kNotReady = 8;  // advance(): next request not ready (not an exit reason)
constexpr uint32_t kFlagHostOut = 1;   // QEntry.flags: the output is pinned host memory
constexpr uint32_t kFlagEmulated = 2;  // QEntry.flags: emulated offload, len = duration in ns
constexpr uint64_t kMaxEmulatedNs = 10000000;
constexpr int kMaxWarps = 16;   // CTA of at most 512 threads (128 registers each: round keys in registers)
constexpr uint32_t kRing = 64;  // >= workers + prefetch
// Tiles an agent keeps queued for its workers.  A deep queue rides through
// the microseconds the global cursor needs to move from one request to the
// next (8 MiB AES-256 stream: 440 GB/s with 1 queued tile, 664 with 16).
constexpr uint32_t kPrefetch = 16;
constexpr uint32_t kMaxClaim = 4;    // tiles per claim: spreads a request over many SMs
// After an agent has claimed its fair share of a request (its tiles / the
// CTA count, rounded up) it leaves the rest to other CTAs for up to this long
// (ns), unless the cursor moves on: otherwise the first agents to see a new
// request queue its tiles behind their own busy workers while other SMs sit
// idle (one 1 MiB request: 512 tiles finished in 2-3 rounds on ~35 SMs).
constexpr uint32_t kShareHoldNs = 2000;
constexpr uint32_t kLookahead = 8;   // requests validated ahead of the cursor
constexpr uint32_t kDispRing = 64;   // > kLookahead
constexpr uint32_t kDispatchBatch = 4;  // queue entries read per round trip over the host link
// Time limit of an idle worker's suspended wait for its ring slot (ns): the
// wait ends early when the slot is filled; at the limit the worker looks at
// the agent's exit code and waits again.
constexpr uint32_t kWaitHintNs = 2000;
// Per-request claims (claim_mode 1): a request's claim word holds its
// sequence number above a 36-bit tile counter, so claims that overshoot the
// tile count never reach the sequence bits; disp carries a busy bit while
// one agent dispatches.
constexpr uint32_t kClaimShift = 36;
constexpr uint64_t kClaimTileMask = (1ull << kClaimShift) - 1;
constexpr uint64_t kDispBusy = 1ull << 40;

struct QEntry {  // 64 bytes, host-written into the request's slot before its order word
    uint64_t tag;  // sequence number + 1 (informational)
    uint64_t in, out, len, iv_hi, iv_lo, gen;
    uint32_t key_slot;  // key slot (bits 0..23) | Nr of its key (bits 24..31; 0 = not registered)
    uint16_t desc;   // slot index d
    uint16_t flags;  // kFlagHostOut, kFlagEmulated
};
static_assert(sizeof(QEntry) == 64, "QEntry layout");

struct SrvRec {  // device-only, 128 bytes
    aesrt::BatchReq rq;             // rq.pad holds the flags
    unsigned long long seq_ntiles;  // (seq << 20) | ntiles, written after the rest
    unsigned long long gen;
    unsigned int tile_groups;       // this request's tile: tile_groups groups, or
    unsigned int tile_parts;        // 1/tile_parts of one group
    unsigned int done_tiles;
    unsigned int pad0;
    unsigned long long claim;       // per-request claims: (seq << 36) | next tile
    unsigned int pad[6];
};
static_assert(offsetof(SrvRec, tile_groups) % 8 == 0, "tile shape words are 8-byte aligned");
static_assert(offsetof(SrvRec, claim) % 8 == 0, "claim word is 8-byte aligned");
static_assert(sizeof(SrvRec) == 128, "SrvRec layout");

struct SrvParams {
    unsigned long long *cursor;
    unsigned long long *adv;
    unsigned long long *disp;      // next sequence number to dispatch (validate into recs)
    unsigned long long *disp_ring; // kDispRing: ring_entry() of dispatched request s at s % kDispRing
    SrvRec *recs;
    const uint4 *keys;          // max_keys x 15 round keys
    const QEntry *queue;        // mapped: the body of the request in slot d at queue[d]
    const uint64_t *order;      // mapped: order[s & qmask] = ((s + 1) << 16) | d, stored after the body
    unsigned long long *done;   // mapped
    const unsigned int *stop;   // mapped
    unsigned int *kstatus;      // mapped
    const uint32_t *te0;
    uint32_t qmask, max_keys, tile_blocks, nslots;  // tile_blocks 0 = chosen per request
    uint32_t nctas;             // resident CTAs (the fair share of a request is its tiles / nctas)
    uint64_t idle_ns, max_len;
    unsigned long long *trace;  // trace builds: kTracePoints stamps per request (null: off)
    uint32_t trace_mask;        // requests kept in the trace buffer - 1 (a power of two - 1)
};

// ---- memory operations ----------------------------------------------------
#ifdef __CUDACC__
SRV_INLINE uint64_t gtime()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
SRV_INLINE void ld_volatile_v2(const uint64_t *p, uint64_t &a, uint64_t &b)
{
    asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}
SRV_INLINE uint64_t ld_relaxed_gpu(const unsigned long long *p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
SRV_INLINE void st_relaxed_gpu(unsigned long long *p, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
SRV_INLINE void st_release_sys(unsigned long long *p, uint64_t v)
{
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
SRV_INLINE uint32_t ld_volatile(const unsigned int *p)
{
    return *reinterpret_cast<const volatile unsigned int *>(p);
}
SRV_INLINE uint64_t ld_relaxed_sys(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.relaxed.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
SRV_INLINE uint64_t ld_acquire_sys(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
SRV_INLINE void fence_acq_rel_sys() { asm volatile("fence.acq_rel.sys;" ::: "memory"); }
SRV_INLINE void fence_gpu() { __threadfence(); }
SRV_INLINE void fence_sys() { __threadfence_system(); }
SRV_INLINE void nap(unsigned ns) { __nanosleep(ns); }
template <class T>
SRV_INLINE T ld_cg(const T *p)
{
    return __ldcg(p);
}
SRV_INLINE unsigned long long atom_add(unsigned long long *p, unsigned long long v) { return atomicAdd(p, v); }
SRV_INLINE unsigned int atom_add(unsigned int *p, unsigned int v) { return atomicAdd(p, v); }
// add with acquire-release semantics at GPU scope: the caller's earlier
// stores (and those it has observed) are ordered before the add, and the
// adds of other threads that precede it in the word's order before what
// follows it
SRV_INLINE unsigned int atom_add_acq_rel(unsigned int *p, unsigned int v)
{
    unsigned int old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
SRV_INLINE unsigned long long atom_cas(unsigned long long *p, unsigned long long c, unsigned long long v)
{
    return atomicCAS(p, c, v);
}
SRV_INLINE unsigned long long atom_exch(unsigned long long *p, unsigned long long v) { return atomicExch(p, v); }
#else
// Host build, for threads that stand in for CTAs.  By default loads
// acquire, stores release and read-modify-writes are acq_rel: stronger than
// the device's relaxed operations plus fences, so a run checks the
// protocol's logic (and a thread sanitizer, which does not model fences,
// reports no false races).  Two switches make runs harsher:
//  * chaos_period() = n > 0: each protocol memory operation yields the
//    thread with probability 1/n, for finer interleavings;
//  * weak_stores() = true: stores wait in a per-thread buffer and become
//    visible later and out of order (per address in program order), all at
//    once at the thread's next fence, release store or wait, and one at a
//    time with probability 1/2 at each store and load.  A thread's loads see
//    its own buffered stores first; a read-modify-write first makes the
//    thread's buffered stores to its address visible.  This is closer to the
//    device's relaxed stores than any CPU, so fence placement is exercised.
inline int &chaos_period()
{
    static int n = 0;
    return n;
}
inline bool &weak_stores()
{
    static bool w = false;
    return w;
}
inline uint64_t host_rand()
{
    thread_local uint64_t x = 0x9E3779B97F4A7C15ull ^ (uint64_t)(uintptr_t)&x;
    x ^= x << 13;
    x ^= x >> 7;
    x ^= x << 17;
    return x;
}
inline void chaos()
{
    const int n = chaos_period();
    if (n > 0 && host_rand() % (uint64_t)n == 0)
        std::this_thread::yield();
}
struct PendingStore {
    void *p;
    uint64_t v;
    int size;
};
inline std::vector<PendingStore> &store_buf()
{
    thread_local std::vector<PendingStore> b;
    return b;
}
inline void put(const PendingStore &s)
{
    switch (s.size) {
    case 1: __atomic_store_n(static_cast<uint8_t *>(s.p), (uint8_t)s.v, __ATOMIC_RELEASE); break;
    case 2: __atomic_store_n(static_cast<uint16_t *>(s.p), (uint16_t)s.v, __ATOMIC_RELEASE); break;
    case 4: __atomic_store_n(static_cast<uint32_t *>(s.p), (uint32_t)s.v, __ATOMIC_RELEASE); break;
    default: __atomic_store_n(static_cast<uint64_t *>(s.p), s.v, __ATOMIC_RELEASE); break;
    }
}
// every buffered store of this thread becomes visible (fence, release, exit)
inline void drain_stores()
{
    auto &b = store_buf();
    for (const auto &s : b)
        put(s);
    b.clear();
}
inline void drain_address(const void *p)
{
    auto &b = store_buf();
    size_t w = 0;
    for (size_t i = 0; i < b.size(); ++i) {
        if (b[i].p == p)
            put(b[i]);
        else
            b[w++] = b[i];
    }
    b.resize(w);
}
inline void drain_one_maybe()
{
    auto &b = store_buf();
    if (b.empty() || (host_rand() & 1))
        return;
    size_t i = (size_t)(host_rand() % b.size());
    for (size_t j = 0; j < i; ++j)  // per address, program order
        if (b[j].p == b[i].p) {
            i = j;
            break;
        }
    put(b[i]);
    b.erase(b.begin() + (std::ptrdiff_t)i);
}
template <class T>
inline void st_weak(T *p, T v)
{
    chaos();
    if (!weak_stores()) {
        __atomic_store_n(p, v, __ATOMIC_RELEASE);
        return;
    }
    uint64_t u = 0;
    std::memcpy(&u, &v, sizeof(T));
    store_buf().push_back(PendingStore{(void *)p, u, (int)sizeof(T)});
    drain_one_maybe();
}
template <class T>
inline T ld_weak(const T *p)
{
    chaos();
    if (weak_stores()) {
        const auto &b = store_buf();
        for (size_t i = b.size(); i-- > 0;)
            if (b[i].p == p) {
                T v;
                std::memcpy(&v, &b[i].v, sizeof(T));
                return v;
            }
        drain_one_maybe();
    }
    return __atomic_load_n(p, __ATOMIC_ACQUIRE);
}
inline uint64_t gtime()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}
inline void ld_volatile_v2(const uint64_t *p, uint64_t &a, uint64_t &b)
{
    a = ld_weak(p);
    b = ld_weak(p + 1);
}
inline uint64_t ld_relaxed_gpu(const unsigned long long *p) { return ld_weak(p); }
inline void st_relaxed_gpu(unsigned long long *p, uint64_t v) { st_weak(p, (unsigned long long)v); }
inline void st_release_sys(unsigned long long *p, uint64_t v)
{
    chaos();
    drain_stores();
    __atomic_store_n(p, v, __ATOMIC_RELEASE);
}
inline uint32_t ld_volatile(const unsigned int *p) { return ld_weak(p); }
inline uint64_t ld_relaxed_sys(const uint64_t *p) { return ld_weak(p); }
inline uint64_t ld_acquire_sys(const uint64_t *p) { return ld_weak(p); }
inline void fence_acq_rel_sys()
{
    drain_stores();
    __atomic_thread_fence(__ATOMIC_ACQ_REL);
}
inline void fence_gpu()
{
    drain_stores();
    __atomic_thread_fence(__ATOMIC_SEQ_CST);
}
inline void fence_sys()
{
    drain_stores();
    __atomic_thread_fence(__ATOMIC_SEQ_CST);
}
inline void nap(unsigned)
{
    drain_stores();  // a waiting thread's stores reach memory (forward progress)
    std::this_thread::yield();
}
template <class T>
inline T ld_cg(const T *p)
{
    return ld_weak(p);
}
inline unsigned long long atom_add(unsigned long long *p, unsigned long long v)
{
    chaos();
    drain_address(p);
    return __atomic_fetch_add(p, v, __ATOMIC_ACQ_REL);
}
inline unsigned int atom_add(unsigned int *p, unsigned int v)
{
    chaos();
    drain_address(p);
    return __atomic_fetch_add(p, v, __ATOMIC_ACQ_REL);
}
inline unsigned int atom_add_acq_rel(unsigned int *p, unsigned int v)
{
    chaos();
    drain_stores();  // a release: every earlier store of this thread is visible first
    return __atomic_fetch_add(p, v, __ATOMIC_ACQ_REL);
}
inline unsigned long long atom_cas(unsigned long long *p, unsigned long long c, unsigned long long v)
{
    chaos();
    drain_address(p);
    __atomic_compare_exchange_n(p, &c, v, false, __ATOMIC_ACQ_REL, __ATOMIC_ACQUIRE);
    return c;
}
inline unsigned long long atom_exch(unsigned long long *p, unsigned long long v)
{
    chaos();
    drain_address(p);
    return __atomic_exchange_n(p, v, __ATOMIC_ACQ_REL);
}
#endif

// Plain and volatile accesses to records and to the CTA's shared ring, and
// the CTA-scope fence (on the host, weak stores and a drain).
#ifdef __CUDACC__
template <class T>
SRV_INLINE void st_field(T *p, T v)
{
    *p = v;
}
template <class T>
SRV_INLINE T ld_field(const T *p)
{
    return *p;
}
SRV_INLINE uint32_t ld_vol(const volatile unsigned int *p) { return *p; }
SRV_INLINE void st_vol(volatile unsigned int *p, uint32_t v) { *p = v; }
SRV_INLINE void fence_cta() { __threadfence_block(); }
#define SRV_STAT(field) ((void)0)
#else
template <class T>
inline void st_field(T *p, T v)
{
    st_weak(p, v);
}
template <class T>
inline T ld_field(const T *p)
{
    return ld_weak(p);
}
inline uint32_t ld_vol(const volatile unsigned int *p) { return ld_weak(const_cast<const unsigned int *>(p)); }
inline void st_vol(volatile unsigned int *p, uint32_t v) { st_weak(const_cast<unsigned int *>(p), (unsigned int)v); }
inline void fence_cta()
{
    drain_stores();
    __atomic_thread_fence(__ATOMIC_SEQ_CST);
}
// How often host runs take the protocol's rare paths.
struct HostStats {
    std::atomic<uint64_t> stale_claim_retries{0}, recycled_claims{0}, low_repairs{0};
};
inline HostStats &host_stats()
{
    static HostStats s;
    return s;
}
#define SRV_STAT(field) (::srvp::host_stats().field.fetch_add(1, std::memory_order_relaxed))
#endif

// ---- tracing (builds with -DSRV_TRACE) -------------------------------------
// Per-request timer stamps of the protocol's steps, for latency breakdowns:
// request seq's stamps sit at trace[(seq & trace_mask) * kTracePoints + point].
// Other builds compile the stamps out, so the kernels are unchanged.
enum TracePoint : uint32_t {
    kTrDispatch = 0,    // a dispatcher has claimed the request (its order word seen)
    kTrPublished,       // its record is complete and its ring entry about to be stored
    kTrFirstClaim,      // an agent claimed its first tile (tile 0)
    kTrFirstPop,        // a worker took tile 0 from its CTA's ring
    kTrRecLoaded,       // that worker has the request's record
    kTrKeysLoaded,      // that worker has its round keys in registers
    kTrFirstTileDone,   // tile 0 is encrypted and stored
    kTrDone,            // the last tile's worker raised the completion word
    kTracePoints
};
#ifdef SRV_TRACE
SRV_INLINE void trace(const SrvParams &p, uint32_t seq, uint32_t point)
{
    if (p.trace)
        p.trace[(size_t)(seq & p.trace_mask) * kTracePoints + point] = gtime();
}
#else
SRV_INLINE void trace(const SrvParams &, uint32_t, uint32_t) {}
#endif

// Nanoseconds since t0, as a signed count: a timer that steps back reads as
// negative (not idle) instead of wrapping to a huge unsigned difference.
SRV_INLINE int64_t since(uint64_t t0)
{
    return (int64_t)(gtime() - t0);
}

// The stop flag lives in host memory (one NVLink-C2C round trip per read),
// so spinning loops look at it at most every 50 us.
struct StopCheck {
    uint64_t next = 0;
    SRV_INLINE bool operator()(const unsigned int *flag)
    {
        const uint64_t now = gtime();
        const int64_t ahead = (int64_t)(next - now);
        if (ahead > 0 && ahead <= 50000)  // read within the last 50 us (and the timer did not step back)
            return false;
        next = now + 50000;
        return ld_volatile(flag) != 0;
    }
};

// Entry of the dispatch ring for request k: sequence number (28 bits), slot
// d (16 bits; 0xffff marks a queue entry the host never writes) and tile
// count (20 bits).  It is stored after the request's record is complete, so
// an entry that carries k is all the advancer needs to move the cursor.
SRV_INLINE uint64_t ring_entry(uint32_t k, uint32_t d, uint32_t ntiles)
{
    return ((uint64_t)k << 36) | ((uint64_t)d << kTileBits) | ntiles;
}

// Order words k0 .. k0 + n - 1 into ow (0 past n).  Word k0 is read last,
// with acquire semantics: the loads after it (the request's body) are
// ordered after it, so dispatching one request needs no fence; the other
// words are relaxed loads issued before it, all in flight together.  The
// host stores each order word with release semantics after the body.
// Measured on GB300 with one 1 MiB request in flight: 19.3 -> 16.0 us from
// submit to the poll that sees completion, against relaxed loads and a
// system-scope fence; the host's new order word is also seen sooner.
SRV_INLINE void load_order_words(const SrvParams &p, uint32_t k0, uint32_t n, uint64_t (&ow)[kDispatchBatch])
{
#pragma unroll
    for (uint32_t i = 1; i < kDispatchBatch; ++i)
        ow[i] = i >= n ? 0 : ld_relaxed_sys(p.order + ((k0 + i) & p.qmask));
    ow[0] = n ? ld_acquire_sys(p.order + (k0 & p.qmask)) : 0;
}

// Dispatch, in sequence order, up to n_max requests starting at k0 (the
// value of disp the caller saw) whose queue entries are present: their tags
// are read in one round trip over the host link and the requests claimed
// with one CAS on disp (one dispatcher per request); then the entries are
// read (after an acquire load of the first order word, and a system-scope
// fence when more than one request was found) and validated into recs[d], and finally their dispatch-ring entries are
// published.  A request without tiles is completed here.  Returns the number
// of requests dispatched (0: k0 not queued yet, or someone else took it) and,
// in *first, the ring entry of request k0.
// PER_REQ (claim_mode 1): the caller holds the dispatch lock (disp = k0 |
// kDispBusy), so there is no CAS here, and each record's claim word is set
// with its tile count.
// pre_ow (optional): the order words of k0 .. k0 + kDispatchBatch - 1,
// already loaded by the caller with load_order_words, e.g. by the
// advancer's polling loop, so a request seen there costs no second read of
// its order word.
template <bool PER_REQ>
SRV_NOINLINE uint32_t dispatch(const SrvParams &p, uint32_t k0, uint32_t n_max, uint64_t *first = nullptr,
                               const uint64_t *pre_ow = nullptr)
{
    // The order words name each request's slot; its body sits in the slot,
    // which the request holds until it completes, so the body cannot change
    // between these reads and the body reads below, however long they take.
    uint32_t m = 0;
    uint64_t ow[kDispatchBatch];
    if (pre_ow) {
#pragma unroll
        for (uint32_t i = 0; i < kDispatchBatch; ++i)
            ow[i] = i >= n_max ? 0 : pre_ow[i];
    } else {
        load_order_words(p, k0, n_max, ow);
    }
#pragma unroll
    for (uint32_t i = 0; i < kDispatchBatch; ++i)
        if (m == i && i < n_max && (uint32_t)((ow[i] >> 16) & kSeqMask) == ((k0 + i + 1) & kSeqMask))
            m = i + 1;
    if (m == 0)
        return 0;
#ifdef SRV_TRACE
    const uint64_t t_seen = gtime();
#endif
    if (m > 1)  // words 1.. were relaxed loads: order their bodies after them
        fence_acq_rel_sys();
    // The bodies are read before the requests are claimed (CAS on disp), so
    // the host-link reads and the claim in L2 are in flight together; a
    // dispatcher that loses the claim drops what it read.
    uint64_t x[kDispatchBatch][7];
#pragma unroll
    for (uint32_t i = 0; i < kDispatchBatch; ++i) {
        if (i < m && (uint32_t)(ow[i] & 0xffffu) < p.nslots) {
            const uint64_t *e = reinterpret_cast<const uint64_t *>(p.queue + (ow[i] & 0xffffu));
            uint64_t unused;
            ld_volatile_v2(e + 0, unused, x[i][0]);
            ld_volatile_v2(e + 2, x[i][1], x[i][2]);
            ld_volatile_v2(e + 4, x[i][3], x[i][4]);
            ld_volatile_v2(e + 6, x[i][5], x[i][6]);
            (void)unused;
        }
    }
    if (!PER_REQ && atom_cas(p.disp, (unsigned long long)k0, (unsigned long long)((k0 + m) & kSeqMask)) != k0)
        return 0;
#ifdef SRV_TRACE
    for (uint32_t i = 0; i < m; ++i)
        if (p.trace)
            p.trace[(size_t)(((k0 + i) & kSeqMask) & p.trace_mask) * kTracePoints + kTrDispatch] = t_seen;
#endif
    uint64_t ent[kDispatchBatch] = {};
    uint32_t done_word[kDispatchBatch] = {};  // status for a request completed here, else 0
#pragma unroll
    for (uint32_t i = 0; i < kDispatchBatch; ++i) {
        if (i >= m)
            continue;
        const uint32_t k = (k0 + i) & kSeqMask;
        const uint64_t in = x[i][0], out = x[i][1], len = x[i][2], iv_hi = x[i][3], iv_lo = x[i][4];
        const uint32_t ks = (uint32_t)x[i][6] & 0xffffffu;
        const uint32_t key_nr = ((uint32_t)x[i][6] >> 24) & 0xffu;  // the host's record of the key's Nr
        const uint32_t d = (uint32_t)(ow[i] & 0xffffu);
        const uint32_t flags = (uint32_t)(x[i][6] >> 48);
        done_word[i] = 0;
        if (d >= p.nslots) {  // the host never writes such an entry; the advancer stops on it
            ent[i] = ring_entry(k, 0xffffu, 0);
            continue;
        }
        int nr = ks < p.max_keys ? (int)key_nr : 0;
        bool ok = (nr == 10 || nr == 12 || nr == 14) && len <= p.max_len;
        if (ok && len)
            ok = in && out && !((in | out) & 15u);
        uint32_t ntiles = 0, tg = 1, tp = 1;
        const bool emulated = (flags & kFlagEmulated) != 0;
        if (emulated) {  // one tile that holds a worker warp for len ns; no key, no payload
            ok = len <= kMaxEmulatedNs;
            ntiles = ok ? 1u : 0u;
            nr = 0;
        } else if (ok && len) {
            // tiles are runs of tg whole 256-block counter groups, or (tp > 1)
            // equal parts of one group.  Unless fixed by the server config, a
            // request is cut into about 512 tiles of 64..1024 blocks: short
            // requests spread over many warps, long ones keep claims rare.
            const uint64_t nb = (len + 15) >> 4;
            const uint64_t groups = (((iv_lo & 255u) + nb - 1) >> 8) + 1;
            uint32_t tb = p.tile_blocks;
            if (!tb) {
                tb = 64;
                while (tb < 1024 && (uint64_t)tb * 512 < nb)
                    tb <<= 1;
            }
            if (tb >= 256)
                tg = tb / 256;
            else
                tp = 256 / tb;
            ntiles = (uint32_t)((groups + tg - 1) / tg * tp);
        }
        SrvRec *rec = p.recs + d;
        st_field(&rec->rq.in, reinterpret_cast<const uint4 *>(in));
        st_field(&rec->rq.out, reinterpret_cast<uint4 *>(out));
        st_field(&rec->rq.len, len);
        st_field(&rec->rq.iv_hi, iv_hi);
        st_field(&rec->rq.iv_lo, iv_lo);
        st_field(&rec->rq.rk, p.keys + 15u * (ok && !emulated ? ks : 0u));
        st_field(&rec->rq.nr, (uint32_t)nr);
        st_field(&rec->rq.pad, flags);
        st_field(&rec->gen, (unsigned long long)x[i][5]);
        st_field(&rec->done_tiles, 0u);
        st_field(&rec->tile_groups, tg);
        st_field(&rec->tile_parts, tp);
        ent[i] = ring_entry(k, d, ntiles);
        // with the record: a claim finds it once it has seen the ring entry
        // (global cursor) or the claim word (per-request claims) below
        st_relaxed_gpu(&rec->seq_ntiles, ((uint64_t)k << kTileBits) | ntiles);
        if (ntiles == 0)
            done_word[i] = ok ? 1u : 2u;
    }
    // One fence: the ring entries (and with per-request claims the claim
    // words) follow the records.  Nothing reads a record's seq_ntiles for
    // request k before it has seen k's ring entry or claim word: the cursor
    // names k only after the advancer has read k's ring entry.
    fence_gpu();
    if (PER_REQ) {
        // A claimer that sees the ring entry before the claim word retries
        // (it reads an older sequence number there).
#pragma unroll
        for (uint32_t i = 0; i < kDispatchBatch; ++i) {
            const uint32_t d = (uint32_t)(ent[i] >> kTileBits) & 0xffffu;
            if (i < m && d != 0xffffu)
                st_relaxed_gpu(&p.recs[d].claim, (ent[i] >> 36) << kClaimShift);
        }
    }
    for (uint32_t i = 0; i < m; ++i)  // before the ring entries: no claim can precede it
        trace(p, (k0 + i) & kSeqMask, kTrPublished);
#pragma unroll
    for (uint32_t i = 0; i < kDispatchBatch; ++i)
        if (i < m)
            st_relaxed_gpu(p.disp_ring + ((k0 + i) % kDispRing), ent[i]);
#pragma unroll
    for (uint32_t i = 0; i < kDispatchBatch; ++i) {
        if (i < m && done_word[i]) {
            const uint32_t d = (uint32_t)(ent[i] >> kTileBits) & 0xffffu;
            fence_sys();
            trace(p, (k0 + i) & kSeqMask, kTrDone);
            st_release_sys(p.done + d, (x[i][5] << 2) | done_word[i]);
        }
    }
    if (first)
        *first = ent[0];
    return m;
}

SRV_INLINE void dispatch_ahead(const SrvParams &p, uint32_t nseq)
{
    const uint32_t k = (uint32_t)ld_relaxed_gpu(p.disp);
    const uint32_t ahead = (k - nseq) & kSeqMask;
    if (ahead <= kLookahead)
        dispatch<false>(p, k, kLookahead + 1 - ahead);
}

// What an agent remembers between global-cursor claims, to save round trips
// to L2: the (sequence, slot) of its last successful claim with that
// request's seq_ntiles word (valid while its claims keep landing on the same
// request; dropped after any failed claim), and a cursor value it has just
// seen move to a new request, whose seq_ntiles it loads alongside its next
// claim instead of after it.
struct ClaimCache {
    uint64_t key = ~0ull;  // (seq << 16) | slot of the cached seq_ntiles
    uint64_t sn = 0;
    uint64_t seen = ~0ull; // (seq << 16) | slot the cursor was seen to name
    uint32_t lookahead = 0;  // nonzero: validate requests ahead of this sequence number once the claimed tiles are queued
};

// Elected advancer (adv has been moved from seq to seq + 1): move the cursor
// to request seq + 1 once its dispatch-ring entry is published (dispatching
// it, with what is queued behind it, if it is next in line), step over
// requests without tiles, and dispatch up to kLookahead requests ahead.
// With block == false the role is handed back at once (kNotReady) when the
// next request is not ready.  With reserve > 0 the cursor move itself claims
// the new request's first `reserve` tiles for the caller: *got is set to
// their count (0 if it moved to no request with tiles) with the request's
// slot, sequence number and tile count in *rd, *rseq, *rnt.  Returns 0,
// kNotReady or an exit code (after handing the role back).
SRV_NOINLINE uint32_t advance(const SrvParams &p, uint32_t seq, uint64_t &last_work, StopCheck &stop, bool block,
                              ClaimCache &cache, uint32_t reserve = 0, uint32_t *got = nullptr,
                              uint32_t *rd = nullptr, uint32_t *rseq = nullptr, uint32_t *rnt = nullptr)
{
    if (got)
        *got = 0;
    for (;;) {
        const uint32_t nseq = (seq + 1) & kSeqMask;
        uint64_t e = 0;
        for (uint32_t round = 0;; ++round) {
            // The ring entry and the dispatch word in L2; from the second
            // round on (waiting for a request: polling), the next order words
            // over the host link in the same round of loads.  Under load the
            // entry is usually published already, and the first round finds
            // it without a host-link round trip.
            e = ld_relaxed_gpu(p.disp_ring + (nseq % kDispRing));
            const uint32_t dsp = (uint32_t)ld_relaxed_gpu(p.disp);
            uint64_t ow[kDispatchBatch];
            if (round)
                load_order_words(p, nseq, kDispatchBatch, ow);
            if ((uint32_t)(e >> 36) == nseq)
                break;  // dispatched and published
            if (dsp == nseq && dispatch<false>(p, nseq, kLookahead + 1, &e, round ? ow : nullptr))
                break;  // dispatched it here: e is its ring entry
            uint32_t r = 0;
            if (!block)
                r = kNotReady;
            else if (stop(p.stop))
                r = kExitStop;
            else if (since(last_work) > (int64_t)p.idle_ns)
                r = kExitIdle;
            if (r) {
                atom_cas(p.adv, (unsigned long long)nseq, (unsigned long long)seq);
                return r;
            }
            nap(32);
        }
        const uint32_t d = (uint32_t)(e >> kTileBits) & 0xffffu;
        if (d >= p.nslots)
            return kExitError;
        const uint32_t nt = (uint32_t)(e & kTileMask);
        // Only the elected advancer changes the sequence number; claims that
        // raced with it only added to the tile count of the old request.  The
        // ring entry carries the request's tile count, so the caller's first
        // claim (made by this very store when reserving) needs no record read.
        const uint32_t take = reserve && nt ? reserve : 0u;
        atom_exch(p.cursor, ((unsigned long long)nseq << 36) | ((unsigned long long)d << kTileBits) | take);
        cache.key = ((uint64_t)nseq << 16) | d;
        cache.sn = ((uint64_t)nseq << kTileBits) | nt;
        last_work = gtime();
        if (take) {
            // the caller queues its tiles first; the look-ahead dispatch
            // (a round trip over the host link) waits until they are queued
            *got = take < nt ? take : nt;
            *rd = d;
            *rseq = nseq;
            *rnt = nt;
            trace(p, nseq, kTrFirstClaim);
            cache.lookahead = nseq | 0x80000000u;
            return 0;
        }
        dispatch_ahead(p, nseq);
        if (nt)
            return 0;
        // nothing to claim in nseq: step over it, unless another agent
        // (which saw the empty request) already took that role
        if (atom_cas(p.adv, (unsigned long long)nseq, (unsigned long long)((nseq + 1) & kSeqMask)) != nseq)
            return 0;
        seq = nseq;
    }
}

// Claim up to `want` tiles of the current request (the agent of a CTA).
// Returns 0 with the tiles [*t0, *t1) of slot *d and its sequence number, or
// an exit code.
// idle_workers: this CTA's workers wait for tiles, so an agent that moves
// the cursor takes the new request's first tiles in the same store (the
// one-in-flight case); with work still queued it leaves them to the others.
SRV_FN uint32_t claim(const SrvParams &p, uint64_t &last_work, StopCheck &stop, uint32_t want, bool idle_workers,
                      uint32_t *d_out, uint32_t *seq_out, uint32_t *t0, uint32_t *t1, uint32_t *nt_out,
                      ClaimCache &cache)
{
    for (;;) {
        if (stop(p.stop))
            return kExitStop;
        // the record word of a request the cursor was just seen to name is
        // loaded together with the claim (both in flight at once)
        uint64_t sn_seen = 0;
        const uint64_t seen = cache.seen;
        if (seen != ~0ull && (uint32_t)(seen & 0xffffu) < p.nslots)
            sn_seen = ld_relaxed_gpu(&p.recs[seen & 0xffffu].seq_ntiles);
        cache.seen = ~0ull;
        const unsigned long long v = atom_add(p.cursor, (unsigned long long)want);
        const uint32_t seq = (uint32_t)(v >> 36);
        const uint32_t d = (uint32_t)(v >> kTileBits) & 0xffffu;
        const uint32_t t = (uint32_t)v & kTileMask;
        if (d < p.nslots) {
            const uint64_t key = ((uint64_t)seq << 16) | d;
            const uint64_t sn = key == cache.key ? cache.sn
                                : key == seen    ? sn_seen
                                                 : ld_relaxed_gpu(&p.recs[d].seq_ntiles);
            const uint32_t nt = (uint32_t)(sn & kTileMask);
            if ((uint32_t)(sn >> kTileBits) == seq && t < nt) {
                cache.key = key;
                cache.sn = sn;
                *d_out = d;
                *seq_out = seq;
                *t0 = t;
                *t1 = t + want < nt ? t + want : nt;
                *nt_out = nt;
                last_work = gtime();
                if (t == 0)
                    trace(p, seq, kTrFirstClaim);
                return 0;
            }
        }
        cache.key = ~0ull;  // a failed claim: never reuse an older request's word
        // The current request has no tiles left: advance (claiming the next
        // request's first tiles in the same store), or wait for the CTA that
        // does.
        if (atom_cas(p.adv, (unsigned long long)seq, (unsigned long long)((seq + 1) & kSeqMask)) == seq) {
            uint32_t got = 0, rd = 0, rseq = 0, rnt = 0;
            const uint32_t r = advance(p, seq, last_work, stop, true, cache, idle_workers ? want : 0u, &got, &rd,
                                       &rseq, &rnt);
            if (r)
                return r;
            if (got) {
                *d_out = rd;
                *seq_out = rseq;
                *t0 = 0;
                *t1 = got;
                *nt_out = rnt;
                return 0;
            }
        } else {
            for (uint32_t spin = 0;; ++spin) {
                const uint64_t c = ld_relaxed_gpu(p.cursor);
                if ((uint32_t)(c >> 36) != seq) {
                    // the server is working even if this CTA's claims keep
                    // losing: idle means no new request anywhere, so a CTA
                    // does not exit under light load while others serve
                    last_work = gtime();
                    cache.seen = (c >> kTileBits) & ((1ull << 44) - 1);  // (seq << 16) | slot
                    break;
                }
                if ((spin & 7) == 7 && (uint32_t)ld_relaxed_gpu(p.adv) == seq)
                    break;  // the advancer gave up its role: compete for it again
                if (stop(p.stop))
                    return kExitStop;
                if (since(last_work) > (int64_t)p.idle_ns)
                    return kExitIdle;
                nap(100);
            }
        }
    }
}

// ---- per-request claims (claim_mode 1) ----------------------------------
// No global cursor: every agent walks the dispatched requests in sequence
// order on its own (`cur`) and claims tiles with atomicAdd on the claim
// word of the request it stands on.  `low` (the cursor word) is the oldest
// request that may still have unclaimed tiles; it bounds dispatch (the
// dispatch ring keeps the entries of requests low .. low + kDispRing - 1)
// and lets agents that fell behind jump forward.  Several requests are cut
// into tiles at once, and no agent waits for another to move a cursor.

// a is ahead of b (by less than half the sequence space)
SRV_INLINE bool seq_after(uint32_t a, uint32_t b)
{
    const uint32_t d = (a - b) & kSeqMask;
    return d != 0 && d < (kSeqMask >> 1);
}

// Request s has no unclaimed tiles (s must be >= low, so its ring entry is
// not overwritten yet).  A slot already holding a newer request means s was
// completed and reaped.
SRV_FN bool exhausted(const SrvParams &p, uint32_t s)
{
    const uint64_t e = ld_relaxed_gpu(p.disp_ring + s % kDispRing);
    if ((uint32_t)(e >> 36) != s)
        return false;  // not dispatched yet
    const uint32_t d = (uint32_t)(e >> kTileBits) & 0xffffu;
    const uint32_t nt = (uint32_t)e & kTileMask;
    if (d >= p.nslots)
        return false;  // a claimer meets it and stops the kernel
    if (nt == 0)
        return true;
    const uint64_t v = ld_relaxed_gpu(&p.recs[d].claim);
    const uint32_t vs = (uint32_t)(v >> kClaimShift);
    if (vs == s)
        return (v & kClaimTileMask) >= nt;
    return seq_after(vs, s);  // newer: s was reaped; older: s's claim word not seen yet
}

// Request s has no unclaimed tiles any more (the caller took its last ones,
// or it has none): move low from s to s + 1, and on over every following
// request that is exhausted too.  A failed CAS means low is not s (behind
// it: whoever moves low to s goes on from there, and waiting agents repeat
// the check; ahead: nothing to do).  The fences order the claim word
// accesses against the CAS on low (the caller's last claim, then its CAS;
// another agent's CAS, then its look at the claim word), so that one of the
// two sees the other.
SRV_FN void help_low(const SrvParams &p, uint32_t s)
{
    fence_gpu();
    for (uint32_t i = 0; i < kDispRing; ++i) {
        const uint32_t n = (s + 1) & kSeqMask;
        if (atom_cas(p.cursor, (unsigned long long)s, (unsigned long long)n) != s)
            return;
        fence_gpu();
        s = n;
        if (!exhausted(p, s))
            return;
    }
}

// Take the dispatch lock at k0 (the value of disp the caller saw) and
// dispatch up to kDispatchBatch queued requests, no further than the ring
// allows past low.  Returns the number dispatched.
SRV_FN uint32_t try_dispatch(const SrvParams &p, uint32_t k0, uint32_t low)
{
    const uint32_t used = (k0 - low) & kSeqMask;
    if (used >= kDispRing)
        return 0;
    const uint32_t room = kDispRing - used;
    const uint32_t n = room < kDispatchBatch ? room : kDispatchBatch;
    if (atom_cas(p.disp, (unsigned long long)k0, (unsigned long long)k0 | kDispBusy) != k0)
        return 0;
    const uint32_t m = dispatch<true>(p, k0, n);
    atom_exch(p.disp, (unsigned long long)((k0 + m) & kSeqMask));
    return m;
}

// Dispatch ahead of an agent standing on request cur while fewer than
// kLookahead requests are validated ahead of it.
SRV_FN void lookahead(const SrvParams &p, uint32_t cur)
{
    const uint64_t k = ld_relaxed_gpu(p.disp);
    if (k & kDispBusy)
        return;
    if ((((uint32_t)k - cur) & kSeqMask) > kLookahead)
        return;
    try_dispatch(p, (uint32_t)k, (uint32_t)ld_relaxed_gpu(p.cursor));
}

// Claim up to `want` tiles (per-request claims).  Same results as claim().
SRV_FN uint32_t claim_pr(const SrvParams &p, uint32_t &cur, uint64_t &last_work, StopCheck &stop,
                             uint32_t want, uint32_t *d_out, uint32_t *seq_out, uint32_t *t0, uint32_t *t1,
                             uint32_t *nt_out)
{
    uint32_t seen_low = (uint32_t)ld_relaxed_gpu(p.cursor);
    uint32_t backoff = 32;
    for (;;) {
        if (stop(p.stop))
            return kExitStop;
        const uint32_t low = (uint32_t)ld_relaxed_gpu(p.cursor);
        if (low != seen_low) {  // the server is making progress
            seen_low = low;
            last_work = gtime();
        }
        if (seq_after(low, cur))
            cur = low;
        const uint64_t e = ld_relaxed_gpu(p.disp_ring + cur % kDispRing);
        const uint32_t es = (uint32_t)(e >> 36);
        if (es == cur) {
            const uint32_t d = (uint32_t)(e >> kTileBits) & 0xffffu;
            const uint32_t nt = (uint32_t)e & kTileMask;
            if (d >= p.nslots)
                return kExitError;  // the host never writes such an entry
            if (nt) {
                const uint64_t v = atom_add(&p.recs[d].claim, (unsigned long long)want);
                const uint32_t vs = (uint32_t)(v >> kClaimShift);
                const uint64_t t = v & kClaimTileMask;
                if (vs == cur && t < nt) {
                    *d_out = d;
                    *seq_out = cur;
                    *t0 = (uint32_t)t;
                    *t1 = t + want < nt ? (uint32_t)t + want : nt;
                    *nt_out = nt;
                    last_work = gtime();
                    if (t == 0)
                        trace(p, cur, kTrFirstClaim);
                    if (t + want >= nt) {  // took the request's last tiles
                        help_low(p, cur);
                        cur = (cur + 1) & kSeqMask;
                    }
                    return 0;
                }
                if (vs != cur && !seq_after(vs, cur)) {
                    SRV_STAT(stale_claim_retries);
                    continue;  // cur's claim word not seen yet (it precedes the ring entry): retry
                }
                if (vs != cur) {
                    // The slot was reaped and reused: this claim landed on the
                    // newer request vs, whose record is complete (its claim
                    // word is set after it); keep the tiles if it has them.
                    fence_gpu();
                    const uint64_t sn = ld_relaxed_gpu(&p.recs[d].seq_ntiles);
                    const uint32_t nt2 = (uint32_t)(sn & kTileMask);
                    if ((uint32_t)(sn >> kTileBits) == vs && t < nt2) {
                        *d_out = d;
                        *seq_out = vs;
                        *t0 = (uint32_t)t;
                        *t1 = t + want < nt2 ? (uint32_t)t + want : nt2;
                        *nt_out = nt2;
                        last_work = gtime();
                        if (t == 0)
                            trace(p, vs, kTrFirstClaim);
                        SRV_STAT(recycled_claims);
                        return 0;
                    }
                }
            }
            // cur has no tiles left.  Moving low on is the job of the agent
            // that took the last tiles (above); a request without tiles has
            // none, so its visitors do it, once low has reached it.
            if (nt == 0 && (uint32_t)ld_relaxed_gpu(p.cursor) == cur)
                help_low(p, cur);
            cur = (cur + 1) & kSeqMask;
            backoff = 32;
            continue;
        }
        if (seq_after(es, cur)) {  // the ring moved past cur: it was exhausted long ago
            cur = (cur + 1) & kSeqMask;
            continue;
        }
        // cur is not dispatched yet: dispatch it if it is next in line
        const uint64_t k = ld_relaxed_gpu(p.disp);
        if (k == cur && try_dispatch(p, cur, low)) {
            last_work = gtime();
            continue;
        }
        if (exhausted(p, low)) {  // repair: low stopped on a request that is exhausted
            SRV_STAT(low_repairs);
            help_low(p, low);
        }
        if (since(last_work) > (int64_t)p.idle_ns)
            return kExitIdle;
        nap(backoff);
        backoff = backoff < 256 ? 2 * backoff : 256;
    }
}


// ---- the agent's steps (one per resident CTA) ------------------------------

// Claim up to `want` tiles for the agent's workers, by either protocol.
// adv_after: (global cursor) this claim took its request's last tiles, so
// the cursor is moved on once they are queued (lease_queued).
template <bool PER_REQ>
SRV_INLINE uint32_t agent_claim(const SrvParams &p, uint32_t &cur, uint64_t &last_work, StopCheck &stop,
                                uint32_t want, bool idle_workers, uint32_t *d, uint32_t *seq, uint32_t *t0,
                                uint32_t *t1, uint32_t *nt, bool &adv_after, ClaimCache &cache)
{
    const uint32_t code = PER_REQ ? claim_pr(p, cur, last_work, stop, want, d, seq, t0, t1, nt)
                                  : claim(p, last_work, stop, want, idle_workers, d, seq, t0, t1, nt, cache);
    adv_after = !PER_REQ && code == 0 && *t1 == *nt;
    return code;
}

// The tiles of the agent's last claim (of request lseq) are queued for its
// workers.  Per-request claims: validate requests ahead.  Global cursor: if
// the claim took the request's last tiles, move the cursor on now instead of
// waiting for a claim to fail (without waiting, if the next request is not
// ready).  Returns 0 or an exit code.
template <bool PER_REQ>
SRV_INLINE uint32_t lease_queued(const SrvParams &p, uint32_t cur, uint32_t lseq, bool &adv_after,
                                 uint64_t &last_work, StopCheck &stop, ClaimCache &cache)
{
    if (PER_REQ) {
        lookahead(p, cur);
        return 0;
    }
    if (cache.lookahead) {  // the advancer's look-ahead, postponed until its tiles were queued
        dispatch_ahead(p, cache.lookahead & 0x7fffffffu);
        cache.lookahead = 0;
    }
    if (!adv_after)
        return 0;
    adv_after = false;
    if (atom_cas(p.adv, (unsigned long long)lseq, (unsigned long long)((lseq + 1) & kSeqMask)) == lseq) {
        const uint32_t r = advance(p, lseq, last_work, stop, false, cache);
        if (r && r != kNotReady)
            return r;
    }
    return 0;
}

// A worker finished one tile of request seq (in slot d, ntiles tiles,
// generation gen); the worker finishing the last one raises the request's
// completion word in host memory.  Ordering: each worker's tile stores come
// before its acquire-release add on done_tiles (the worker's lane 0 adds
// after a warp barrier over the tile's stores; for host-memory outputs the
// warp has also fenced at system scope); the last add acquires every
// earlier one, and the completion word is stored with system-scope release,
// so a host that sees the word sees every tile's output.
SRV_INLINE void tile_finished(const SrvParams &p, uint32_t d, uint32_t ntiles, uint32_t seq, uint64_t gen)
{
    SrvRec *rec = p.recs + d;
    const unsigned int prev = atom_add_acq_rel(&rec->done_tiles, 1u);
    if (prev + 1 == ntiles) {
        trace(p, seq, kTrDone);
        st_release_sys(p.done + d, (gen << 2) | 1u);
    }
    (void)seq;
}


// ---- the CTA: agent and worker warps, joined by a ring in shared memory ----
// The agent (warp 0, lane 0) claims tiles and pushes them; each worker warp
// reserves the next position (atomicAdd on head) and waits for the agent to
// fill it.  A slot is refilled only once the worker that read its previous
// item has marked it read.  On the GPU each slot has an mbarrier whose phase
// completes when the agent fills it, so waiting workers are suspended in
// mbarrier.try_wait instead of polling shared memory (a polling warp takes
// issue slots and shared-memory cycles from the warps that encrypt: with 14
// idle workers polling, the one encrypting ran 3.5x slower); host builds
// poll.
//
// The worker that reserved a position writes (position << 8) | its warp into
// the slot's owner word, so the agent can see on which SM partition (warp %
// 4) each waiting worker runs: when the next waiting worker's partition
// already runs a tile of the same lease and a later waiting worker's does
// not, the agent fills the position with an empty item (the worker reserves
// again) and gives the tile to the later one.  The tiles of one claim then
// run on different partitions instead of sharing one partition's issue slot
// (two tiles on one partition take 1.6x as long, three 2.2x).  Under load no
// worker waits and the agent fills in order.
struct Ring {
#ifdef __CUDACC__
    unsigned long long full[kRing];  // mbarrier per slot, expected arrivals 1 (device builds)
#endif
    unsigned int head;               // positions reserved by workers (atomicAdd)
    volatile unsigned int tail;      // positions filled by the agent
    volatile unsigned int exit_code; // set by the agent after its last push
    uint32_t d[kRing], t[kRing], seq[kRing], nt[kRing];  // nt == 0: an empty item
    volatile unsigned int read_mark[kRing];  // position + 1 of the last item read from each slot
    volatile unsigned int owner[kRing];      // (position << 8) | warp of the worker that reserved it
};
constexpr uint32_t kPartitions = 4;  // warp w of an SM runs on partition w % 4

#ifdef __CUDACC__
SRV_INLINE uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
// The agent filled `slot`: complete the slot's current phase (release: the
// item's fields are visible to the worker whose wait sees the phase end).
SRV_INLINE void ring_signal(Ring &ring, uint32_t slot)
{
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&ring.full[slot]))
                 : "memory");
}
// Wait (suspended, up to about hint_ns) for the phase of `slot` with the
// given parity to complete; true once it has (acquire).
SRV_INLINE bool ring_try_wait(Ring &ring, uint32_t slot, uint32_t parity, uint32_t hint_ns)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred P1;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 P1, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, P1;\n}"
        : "=r"(ok)
        : "r"(smem_addr(&ring.full[slot])), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}
#else
inline void ring_signal(Ring &, uint32_t) {}
#endif

// The ring's counters, set by one thread before the agent and the workers
// start (and its barriers initialised on the GPU).
SRV_INLINE void ring_init(Ring &ring)
{
    ring.head = 0;
    ring.tail = 0;
    ring.exit_code = 0;
    for (uint32_t i = 0; i < kRing; ++i) {
        ring.read_mark[i] = 0;
        ring.owner[i] = ~0u;
    }
#ifdef __CUDACC__
    for (uint32_t i = 0; i < kRing; ++i)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&ring.full[i])) : "memory");
#endif
}

// How many items the agent may add now: slots whose previous item has been
// read, up to kPrefetch queued beyond the waiting workers.  *waiting:
// workers waiting for an item.
SRV_INLINE uint32_t ring_room(Ring &ring, uint32_t *waiting)
{
    const uint32_t head = ld_vol(reinterpret_cast<volatile unsigned int *>(&ring.head));
    const uint32_t tail = ld_vol(&ring.tail);
    const int32_t queued = (int32_t)(tail - head);
    *waiting = queued < 0 ? (uint32_t)(-queued) : 0u;
    const uint32_t want = queued < (int32_t)kPrefetch ? (uint32_t)((int32_t)kPrefetch - queued) : 0u;
    uint32_t r = 0;
    while (r < want && r < 2 * kMaxClaim &&
           (tail + r < kRing || ld_vol(&ring.read_mark[(tail + r) % kRing]) == tail + r - kRing + 1))
        ++r;
    return r;
}

// The partition of the worker waiting at position pos, or kPartitions when
// unknown (its owner word is not written yet).
SRV_INLINE uint32_t ring_owner_partition(Ring &ring, uint32_t pos)
{
    const uint32_t o = ld_vol(&ring.owner[pos % kRing]);
    return (o >> 8) == (pos & 0xffffffu) ? (o & 0xffu) % kPartitions : kPartitions;
}

// Queue tiles [lt, lend) of a lease into up to `room` positions: the items'
// fields (empty items where a waiting worker's partition already runs a tile
// of this lease and a later waiting worker's is free; `used` holds the
// lease's partitions), one CTA fence, the new tail, then each filled slot's
// barrier.  Returns the number of tiles queued.  The partitions of the
// workers waiting in the positions to fill are read once, all at a time,
// into 4-bit fields of one word, since the placement looks at each several
// times.
SRV_INLINE uint32_t push_lease(Ring &ring, uint32_t room, uint32_t d, uint32_t seq, uint32_t lt, uint32_t lend,
                               uint32_t nt, uint32_t &used)
{
    static_assert(2 * kMaxClaim * 4 <= 32 && kPartitions < 16, "one 4-bit partition field per position");
    const uint32_t tail = ld_vol(&ring.tail);
    const uint32_t head = ld_vol(reinterpret_cast<volatile unsigned int *>(&ring.head));
    const int32_t waiting = (int32_t)(head - tail);  // workers wait at tail .. head - 1
    uint32_t nw = waiting <= 0 ? 0u : (uint32_t)waiting < room ? (uint32_t)waiting : room;
    nw = nw < 2 * kMaxClaim ? nw : 2 * kMaxClaim;  // ring_room never offers more
    uint32_t parts = 0;
    for (uint32_t i = 0; i < nw; ++i)
        parts |= ring_owner_partition(ring, tail + i) << (4 * i);
    uint32_t filled = 0, tiles = 0;
    while (filled < room && lt + tiles < lend) {
        const uint32_t pos = tail + filled;
        const uint32_t slot = pos % kRing;
        bool skip = false;
        if (filled < nw) {  // a worker waits at pos
            const uint32_t part = (parts >> (4 * filled)) & 15u;
            if (part < kPartitions && ((used >> part) & 1u)) {
                for (uint32_t q = filled + 1; q < nw; ++q) {
                    const uint32_t pq = (parts >> (4 * q)) & 15u;
                    if (pq < kPartitions && !((used >> pq) & 1u)) {
                        skip = true;
                        break;
                    }
                }
            }
            if (!skip && part < kPartitions)
                used |= 1u << part;
        }
        st_field(&ring.d[slot], d);
        st_field(&ring.t[slot], lt + tiles);
        st_field(&ring.seq[slot], seq);
        st_field(&ring.nt[slot], skip ? 0u : nt);
        ++filled;
        if (!skip)
            ++tiles;
    }
    if (filled) {
        fence_cta();
        st_vol(&ring.tail, tail + filled);
        for (uint32_t i = 0; i < filled; ++i)
            ring_signal(ring, (tail + i) % kRing);
    }
    return tiles;
}

// Agent warp, lane 0: keep the ring up to kPrefetch items ahead of the
// workers.  PER_REQ selects per-request claims (claim_mode 1) over the
// global cursor.
template <bool PER_REQ>
SRV_NOINLINE void agent(const SrvParams &p, Ring &ring)
{
    uint64_t last_work = gtime();
    StopCheck stop;
    ClaimCache cache;
    uint32_t cur = PER_REQ ? (uint32_t)ld_relaxed_gpu(p.cursor) : 0u;  // request this agent stands on
    uint32_t ld = 0, lseq = 0, lt = 0, lend = 0, lnt = 0;  // current lease: tiles [lt, lend) of slot ld
    uint32_t lparts = 0;                                  // partitions running the current lease's tiles
    bool adv_after = false;                               // the lease ends its request
    uint32_t code = 0;
    uint32_t backoff = 32;  // ns; a spinning agent would take shared-memory cycles from its workers
    // global cursor: the request this agent last claimed from, how many of its
    // tiles it took, its fair share and when the share was reached
    uint32_t fs_seq = ~0u, fs_taken = 0, fs_share = ~0u, fs_nt = 0;
    uint64_t fs_full_at = 0;
    for (;;) {
        uint32_t waiting = 0;
        const uint32_t room = ring_room(ring, &waiting);
        if (!room) {  // full
            if (stop(p.stop)) {
                code = kExitStop;
                break;
            }
            nap(backoff);
            backoff = backoff < 256 ? 2 * backoff : 256;
            continue;
        }
        if (lt >= lend) {
            if (!PER_REQ && fs_taken >= fs_share) {
                // this CTA holds its share of request fs_seq: while the cursor is
                // still on it with tiles left, give the other CTAs kShareHoldNs
                const uint64_t cv = ld_relaxed_gpu(p.cursor);
                if ((uint32_t)(cv >> 36) == fs_seq && ((uint32_t)cv & kTileMask) < fs_nt &&
                    since(fs_full_at) < (int64_t)kShareHoldNs) {
                    if (stop(p.stop)) {
                        code = kExitStop;
                        break;
                    }
                    nap(64);
                    continue;
                }
                fs_share = ~0u;  // hold over: claim as usual
            }
            const uint32_t want = waiting + kPrefetch < kMaxClaim ? waiting + kPrefetch : kMaxClaim;
            code = agent_claim<PER_REQ>(p, cur, last_work, stop, want, waiting > 0, &ld, &lseq, &lt, &lend, &lnt,
                                        adv_after, cache);
            if (code)
                break;
            lparts = 0;
            if (!PER_REQ) {
                if (lseq != fs_seq) {
                    fs_seq = lseq;
                    fs_taken = 0;
                    fs_nt = lnt;
                    fs_share = p.nctas ? (lnt + p.nctas - 1) / p.nctas : ~0u;
                }
                fs_taken += lend - lt;
                if (fs_taken >= fs_share)
                    fs_full_at = gtime();
            }
        }
        // the room seen before the claim is still available: only the agent fills
        lt += push_lease(ring, room, ld, lseq, lt, lend, lnt, lparts);
        backoff = 32;
        if (lt >= lend) {  // the whole lease is queued
            code = lease_queued<PER_REQ>(p, cur, lseq, adv_after, last_work, stop, cache);
            if (code)
                break;
        }
    }
    fence_cta();
    st_vol(&ring.exit_code, code);
}

// A worker's lane 0 (host builds): take the next position and wait for the
// agent to fill it.  Returns false when the agent has exited without filling
// it (its last pushes are taken first).
SRV_INLINE bool ring_pop(Ring &ring, uint32_t warp, uint32_t *d, uint32_t *t, uint32_t *seq, uint32_t *nt)
{
again:
    const uint32_t pos = atom_add(&ring.head, 1u);
    st_vol(&ring.owner[pos % kRing], (pos << 8) | warp);
    for (uint32_t spin = 0;; ++spin) {
        if ((int32_t)(ld_vol(&ring.tail) - pos) > 0)
            break;
        if (spin > 4)
            nap(64);
        if (ld_vol(&ring.exit_code)) {
            fence_cta();
            if ((int32_t)(ld_vol(&ring.tail) - pos) <= 0)
                return false;
            break;
        }
    }
    fence_cta();
    *d = ld_field(&ring.d[pos % kRing]);
    *t = ld_field(&ring.t[pos % kRing]);
    *seq = ld_field(&ring.seq[pos % kRing]);
    *nt = ld_field(&ring.nt[pos % kRing]);
    fence_cta();
    st_vol(&ring.read_mark[pos % kRing], pos + 1);
    if (*nt == 0)
        goto again;  // an empty item: the tile went to another partition
    return true;
}

#ifdef __CUDACC__
// The same step for a whole worker warp on the GPU: lane 0 reserves the
// position; the warp waits suspended on the slot's mbarrier for the phase of
// this lap (position / kRing) -- at most 15 workers wait beyond the filled
// positions and kRing = 64, so the slot's previous lap is always filled
// before anyone waits for this one, and the parity names this lap alone.
// The wait is re-armed every ~2 us to look at the agent's exit code.
SRV_INLINE bool ring_pop_warp(Ring &ring, uint32_t *d, uint32_t *t, uint32_t *seq, uint32_t *nt)
{
    const uint32_t lane = threadIdx.x & 31u;
again:
    uint32_t pos = 0;
    if (lane == 0) {
        pos = atomicAdd(&ring.head, 1u);
        st_vol(&ring.owner[pos % kRing], (pos << 8) | (threadIdx.x >> 5));
    }
    pos = __shfl_sync(0xffffffffu, pos, 0);
    const uint32_t slot = pos % kRing, parity = (pos / kRing) & 1u;
    for (;;) {
        const bool full = __shfl_sync(0xffffffffu, (uint32_t)ring_try_wait(ring, slot, parity, kWaitHintNs), 0) != 0;
        if (full)
            break;
        if (ld_vol(&ring.exit_code)) {
            __threadfence_block();
            if ((int32_t)(ld_vol(&ring.tail) - pos) <= 0)
                return false;  // the agent has left; this position was never filled
        }
    }
    *d = ring.d[slot];
    *t = ring.t[slot];
    *seq = ring.seq[slot];
    *nt = ring.nt[slot];
    __syncwarp();
    if (lane == 0) {
        __threadfence_block();
        st_vol(&ring.read_mark[slot], pos + 1);
    }
    if (*nt == 0)
        goto again;  // an empty item: the tile went to another partition
    return true;
}
#endif

}  // namespace srvp
