// conflict.cpp -- the page-protection conflict detector for rerouted handlers.
//
// Rerouting lets a handler park at its offload while the server runs others,
// which removes the run-to-completion atomicity that a single-threaded
// server's unlocked shared aggregates (counters, batch queues, caches) rely
// on: an unlocked read-modify-write that spans the offload loses updates
// when handlers overlap.  The paper's transparent detector write-protects
// the shared-state pages, snapshots a version clock when a handler parks at
// its offload, and treats a write fault on a page modified during the park
// as a conflict; under enforcement it serializes only the conflicting
// handlers (Sec. 5, "A transparent conflict detector").
//
// cdet_run() measures that detector on a synthetic server: `handlers`
// cooperative handlers (ucontext fibers on the calling thread, one event
// loop) serve `requests` requests; request i reads shared counter
// c(i) (one of `counters`, `counters_per_page` to a page), parks at an
// offload, and writes the counter back incremented.  The paper sorts the
// shared state of offload-adjacent servers into four patterns, of which
// only this unlocked shared aggregate is hazardous under overlap; the
// other three are selectable too (`pattern`), to check that the detector
// stays silent on them: the counter is only read; each handler (one per
// connection) updates a counter of its own; the application holds a lock
// from the read to the write.  Modes:
//   UNPROTECTED  overlap, nothing guards the counters (updates get lost);
//   LOCK         one coarse lock held from the read to the write, i.e.
//                across the offload (serializes the offloads it protects);
//   DETECT       overlap, the detector counts conflicts but lets them be;
//   ENFORCE      overlap, a conflicting handler is restarted and re-run
//                serialized: its offload is waited for without yielding.
// The offload is a host timer of offload_ns, or, with a server, the served
// path: an emulated offload of offload_ns (offload_submit_emulated) or a real
// AES-CTR request of `bytes` from a per-handler buffer.
//
// Detector mechanics: the shared region is mapped PROT_READ.  A write faults
// into on_fault(), which (for the running handler f and page p) reports a
// conflict when f has parked since its request started and p's version is
// newer than f's snapshot, and otherwise stamps p with the next clock value
// and unprotects it.  Pages a handler unprotected are protected again before
// any other handler runs (when it parks, restarts or finishes a request), so
// every handler's first write to a page after someone else's is seen.  A
// restart is a siglongjmp from the fault handler to the request's start,
// taken on the handler's own stack; it suits handlers whose writes before
// the conflicting one may be repeated (true of the workload here).
#include "../../include/aesoffload.h"

#include <chrono>
#include <csetjmp>
#include <csignal>
#include <cstdint>
#include <cstring>
#include <sys/mman.h>
#include <ucontext.h>
#include <unistd.h>
#include <vector>

namespace {

using clk = std::chrono::steady_clock;

constexpr size_t kStack = 256 * 1024;

struct Fiber {
    ucontext_t ctx;
    void *stack = nullptr;
    sigjmp_buf restart;
    int id = 0;
    bool done = false;
    bool parked = false;        // waiting for its offload
    bool serialized = false;    // re-running after a conflict: no parking
    bool snap_valid = false;    // has parked during the current request
    uint64_t snapshot = 0;      // version clock when it last parked
    uint64_t ticket = 0;        // offload in flight (server)
    uint64_t reads = 0;         // CDET_PATTERN_READONLY: reads completed
    clk::time_point deadline;   // offload in flight (host timer)
    int dirty_lo = 0, dirty_hi = -1;  // pages this handler unprotected: within [lo, hi]
};

struct Run {
    cdet_run_cfg_t cfg;
    long page = 4096;
    uint8_t *region = nullptr;
    size_t region_bytes = 0;
    int npages = 0;
    std::vector<uint64_t> page_version;
    uint64_t clock = 0;
    std::vector<Fiber> fibers;
    Fiber *current = nullptr;
    ucontext_t sched;
    int next_request = 0;
    bool lock_held = false;
    uint64_t conflicts = 0, restarts = 0;
    int error = 0;
    bool detector = false;
};

Run *g_run = nullptr;  // the run in progress (one at a time per process)
struct sigaction g_prev_segv;

uint64_t *counter_ptr(Run &r, int c)
{
    const int per = r.cfg.counters_per_page;
    const int pg = c / per, slot = c % per;
    return reinterpret_cast<uint64_t *>(r.region + (size_t)pg * (size_t)r.page + 64u * (size_t)slot);
}

// Only the running handler's pages are ever writable (every other page is
// read-only whenever another handler runs), so one call over the range that
// spans its unprotected pages restores the invariant, however many they are.
void protect_dirty(Run &r, Fiber &f)
{
    if (f.dirty_hi >= f.dirty_lo)
        mprotect(r.region + (size_t)f.dirty_lo * (size_t)r.page,
                 (size_t)(f.dirty_hi - f.dirty_lo + 1) * (size_t)r.page, PROT_READ);
    f.dirty_lo = 0;
    f.dirty_hi = -1;
}

void on_fault(int sig, siginfo_t *si, void *uc)
{
    Run *r = g_run;
    uint8_t *a = static_cast<uint8_t *>(si->si_addr);
    if (!r || !r->detector || a < r->region || a >= r->region + r->region_bytes || !r->current) {
        // not ours: fall back to the previous action and let the access fault again
        sigaction(SIGSEGV, &g_prev_segv, nullptr);
        (void)sig;
        (void)uc;
        return;
    }
    Fiber &f = *r->current;
    const int p = (int)((size_t)(a - r->region) / (size_t)r->page);
    if (f.snap_valid && r->page_version[(size_t)p] > f.snapshot) {
        ++r->conflicts;
        if (r->cfg.mode == CDET_ENFORCE) {
            ++r->restarts;
            siglongjmp(f.restart, 1);
        }
    }
    r->page_version[(size_t)p] = ++r->clock;
    mprotect(r->region + (size_t)p * (size_t)r->page, (size_t)r->page, PROT_READ | PROT_WRITE);
    if (f.dirty_hi < f.dirty_lo) {
        f.dirty_lo = p;
        f.dirty_hi = p;
    } else {
        f.dirty_lo = p < f.dirty_lo ? p : f.dirty_lo;
        f.dirty_hi = p > f.dirty_hi ? p : f.dirty_hi;
    }
}

bool offload_done(Run &r, Fiber &f)
{
    if (!r.cfg.srv)
        return clk::now() >= f.deadline;
    const int rc = offload_poll(r.cfg.srv, f.ticket);
    if (rc == AES_PENDING)
        return false;
    if (rc != AES_OK && !r.error)
        r.error = rc;
    return true;
}

bool offload_start(Run &r, Fiber &f, int req)
{
    if (!r.cfg.srv) {
        f.deadline = clk::now() + std::chrono::nanoseconds(r.cfg.offload_ns);
        return true;
    }
    for (;;) {
        int rc;
        if (r.cfg.bytes) {
            uint8_t iv[16] = {};
            std::memcpy(iv, &req, sizeof(req));
            const size_t stride = (r.cfg.bytes + 255) / 256 * 256;
            const uint8_t *in = static_cast<const uint8_t *>(r.cfg.buf_in) + stride * (size_t)f.id;
            uint8_t *out = static_cast<uint8_t *>(r.cfg.buf_out) + stride * (size_t)f.id;
            rc = offload_submit(r.cfg.srv, r.cfg.key_slot, iv, in, out, r.cfg.bytes, &f.ticket);
        } else {
            rc = offload_submit_emulated(r.cfg.srv, r.cfg.offload_ns, &f.ticket);
        }
        if (rc == AES_OK)
            return true;
        if (rc != AES_EAGAIN) {
            if (!r.error)
                r.error = rc;
            return false;
        }
    }
}

// The offload of the running handler: park (the event loop runs others)
// unless the handler is serialized, in which case wait for it here.
void offload(Run &r, Fiber &f, int req)
{
    if (!offload_start(r, f, req))
        return;
    if (f.serialized) {
        while (!offload_done(r, f)) {
        }
        return;
    }
    protect_dirty(r, f);
    f.snapshot = r.clock;
    f.snap_valid = true;
    f.parked = true;
    swapcontext(&f.ctx, &r.sched);  // resumed by the loop once the offload is done
}

void acquire_lock(Run &r, Fiber &f)
{
    while (r.lock_held)
        swapcontext(&f.ctx, &r.sched);  // yield; the loop resumes runnable handlers
    r.lock_held = true;
}

void release_lock(Run &r)
{
    r.lock_held = false;
}

// One request: read a counter, offload, write it back incremented.
void serve(Run &r, Fiber &f, int req)
{
    // counter of request req: a mixed hash (splitmix64 finaliser), so that
    // requests in flight together pick counters independently
    uint64_t h = (uint64_t)req + 0x9E3779B97F4A7C15ull;
    h = (h ^ (h >> 30)) * 0xBF58476D1CE4E5B9ull;
    h = (h ^ (h >> 27)) * 0x94D049BB133111EBull;
    h ^= h >> 31;
    const int pattern = r.cfg.pattern;
    const int c = pattern == CDET_PATTERN_PER_CONN ? f.id : (int)(h % (uint64_t)r.cfg.counters);
    const bool locked = r.cfg.mode == CDET_LOCK || pattern == CDET_PATTERN_LOCKED;
    f.serialized = false;
    if (sigsetjmp(f.restart, 1)) {
        // restarted after a conflict (the stale write faulted before it
        // landed): re-run serialized, so no other handler interleaves
        protect_dirty(r, f);
        f.serialized = true;
    }
    f.snap_valid = false;
    if (locked)
        acquire_lock(r, f);
    volatile uint64_t *ctr = counter_ptr(r, c);
    const uint64_t v = *ctr;  // read
    offload(r, f, req);       // park
    if (pattern == CDET_PATTERN_READONLY)
        ++f.reads;
    else
        *ctr = v + 1;         // write (may fault)
    if (locked)
        release_lock(r);
    protect_dirty(r, f);
    f.snap_valid = false;
}

void fiber_main(unsigned lo, unsigned hi)
{
    Fiber *f = reinterpret_cast<Fiber *>(((uintptr_t)hi << 32) | (uintptr_t)lo);
    Run &r = *g_run;
    for (;;) {
        if (r.error || r.next_request >= r.cfg.requests)
            break;
        const int req = r.next_request++;
        serve(r, *f, req);
    }
    f->done = true;
    swapcontext(&f->ctx, &r.sched);
}

}  // namespace

extern "C" {

int cdet_run(const cdet_run_cfg_t *cfg, cdet_run_result_t *res)
{
    if (!cfg || !res || cfg->handlers < 1 || cfg->handlers > 4096 || cfg->requests < 0 || cfg->counters < 1 ||
        cfg->counters_per_page < 1 || cfg->counters_per_page > 64 || cfg->mode < CDET_UNPROTECTED ||
        cfg->mode > CDET_ENFORCE || (cfg->bytes && (!cfg->srv || !cfg->buf_in || !cfg->buf_out)) ||
        cfg->pattern < CDET_PATTERN_SHARED || cfg->pattern > CDET_PATTERN_LOCKED ||
        (cfg->pattern == CDET_PATTERN_PER_CONN && cfg->counters < cfg->handlers))
        return AES_EINVAL;
    if (g_run)
        return AES_EINVAL;  // one run at a time
    Run r;
    r.cfg = *cfg;
    r.page = sysconf(_SC_PAGESIZE);
    r.npages = (cfg->counters + cfg->counters_per_page - 1) / cfg->counters_per_page;
    r.region_bytes = (size_t)r.npages * (size_t)r.page;
    r.detector = cfg->mode == CDET_DETECT || cfg->mode == CDET_ENFORCE;
    void *m = mmap(nullptr, r.region_bytes, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (m == MAP_FAILED)
        return AES_ENOMEM;
    r.region = static_cast<uint8_t *>(m);
    r.page_version.assign((size_t)r.npages, 0);
    r.fibers.resize((size_t)cfg->handlers);
    for (int i = 0; i < cfg->handlers; ++i) {
        Fiber &f = r.fibers[(size_t)i];
        f.id = i;
        f.stack = mmap(nullptr, kStack, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
        if (f.stack == MAP_FAILED) {
            f.stack = nullptr;
            r.error = AES_ENOMEM;
        }
    }
    struct sigaction sa {};
    if (!r.error && r.detector) {
        sa.sa_sigaction = on_fault;
        sa.sa_flags = SA_SIGINFO;
        sigemptyset(&sa.sa_mask);
        if (sigaction(SIGSEGV, &sa, &g_prev_segv) != 0)
            r.error = AES_EINVAL;
        else
            mprotect(r.region, r.region_bytes, PROT_READ);
    }
    g_run = &r;
    const clk::time_point t0 = clk::now();
    if (!r.error) {
        for (auto &f : r.fibers) {
            getcontext(&f.ctx);
            f.ctx.uc_stack.ss_sp = f.stack;
            f.ctx.uc_stack.ss_size = kStack;
            f.ctx.uc_link = &r.sched;
            const uintptr_t fp = reinterpret_cast<uintptr_t>(&f);
            makecontext(&f.ctx, reinterpret_cast<void (*)()>(fiber_main), 2, (unsigned)(fp & 0xffffffffu),
                        (unsigned)(fp >> 32));
        }
        // the event loop: run every handler that can make progress
        int alive = cfg->handlers;
        while (alive > 0) {
            alive = 0;
            for (auto &f : r.fibers) {
                if (f.done)
                    continue;
                ++alive;
                if (f.parked) {
                    if (!offload_done(r, f))
                        continue;
                    f.parked = false;
                }
                r.current = &f;
                swapcontext(&r.sched, &f.ctx);
                r.current = nullptr;
            }
        }
    }
    const double elapsed = std::chrono::duration<double>(clk::now() - t0).count();
    uint64_t total = 0;
    if (r.detector)
        mprotect(r.region, r.region_bytes, PROT_READ | PROT_WRITE);
    for (int c = 0; c < cfg->counters; ++c)
        total += *counter_ptr(r, c);
    for (auto &f : r.fibers)
        total += f.reads;
    if (r.detector && !r.error)
        sigaction(SIGSEGV, &g_prev_segv, nullptr);
    g_run = nullptr;
    for (auto &f : r.fibers)
        if (f.stack)
            munmap(f.stack, kStack);
    munmap(r.region, r.region_bytes);
    res->final_count = total;
    res->lost_updates = (uint64_t)cfg->requests - total;
    res->conflicts = r.conflicts;
    res->restarts = r.restarts;
    res->elapsed_s = elapsed;
    return r.error;
}

}  // extern "C"
