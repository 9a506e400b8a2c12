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
//
// With cfg.store_mode == CDET_STORES_EMULATE (the default) the pages are
// never unprotected: the fault
// handler performs the store itself through a writable alias of the region
// (see "store emulation" below), so every write faults and a page also
// records which handler stamped it (a handler's own later writes are no
// conflict).
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
    bool finished = false;      // its completion was reaped on its behalf (finished_rc)
    int finished_rc = 0;
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
    std::vector<int> page_writer;  // handler whose write stamped the page (-1 none)
    uint8_t *alias = nullptr;      // writable second mapping of the region (store emulation)
    uint64_t emulated = 0, protect_calls = 0;
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
    if (f.dirty_hi >= f.dirty_lo) {
        mprotect(r.region + (size_t)f.dirty_lo * (size_t)r.page,
                 (size_t)(f.dirty_hi - f.dirty_lo + 1) * (size_t)r.page, PROT_READ);
        ++r.protect_calls;
    }
    f.dirty_lo = 0;
    f.dirty_hi = -1;
}

// ---- store emulation (cfg.store_mode == CDET_STORES_EMULATE) -------------
// The shared pages stay read-only for the whole run.  The fault handler
// performs the faulting store itself, through a second, writable mapping
// of the same memory, and steps the program counter past it.  A guarded
// write then costs one fault and no protection change; a protection change
// is the expensive part in a process that shares its page tables with a GPU.
// Decoded are the plain general-register stores a compiler emits for an
// aggregate update:
//   x86-64: MOV r/m8|16|32|64, r and MOV r/m, imm (opcodes 88 / 89 and
//   C6 / C7 with ModRM.reg 0; optional 66 and REX prefixes);
//   AArch64: STR / STUR / STTR of 8..64-bit general registers (immediate
//   unsigned offset, unscaled, pre- and post-index with base write-back,
//   register offset).
// Anything else (vector, pair, atomic and exclusive stores) falls back to
// unprotecting the page.
struct Store {
    uint64_t value = 0;
    int size = 0;        // bytes stored
    int len = 0;         // instruction bytes
    int wb_reg = -1;     // AArch64 base register written back (31 = SP), -1 none
    int64_t wb_delta = 0;
};

#if defined(__x86_64__)
int x86_greg(int n)
{
    static const int map[16] = {REG_RAX, REG_RCX, REG_RDX, REG_RBX, REG_RSP, REG_RBP, REG_RSI, REG_RDI,
                                REG_R8,  REG_R9,  REG_R10, REG_R11, REG_R12, REG_R13, REG_R14, REG_R15};
    return map[n & 15];
}

bool decode_store(const ucontext_t *uc, Store *st)
{
    const greg_t *g = uc->uc_mcontext.gregs;
    const uint8_t *ip = reinterpret_cast<const uint8_t *>(g[REG_RIP]);
    int i = 0;
    bool op16 = false;
    if (ip[i] == 0x66) {
        op16 = true;
        ++i;
    }
    uint8_t rex = 0;
    if ((ip[i] & 0xF0) == 0x40)
        rex = ip[i++];
    const uint8_t op = ip[i++];
    if (op != 0x88 && op != 0x89 && op != 0xC6 && op != 0xC7)
        return false;
    const uint8_t modrm = ip[i++];
    const int mod = modrm >> 6, rm = modrm & 7, reg = (modrm >> 3) & 7;
    if (mod == 3)
        return false;  // register destination: not a store
    if ((op == 0xC6 || op == 0xC7) && reg != 0)
        return false;  // C6 / C7 with another ModRM.reg are not MOV
    if (rm == 4) {     // SIB byte; base 101 with mod 00 means disp32 and no base
        const uint8_t sib = ip[i++];
        if (mod == 0 && (sib & 7) == 5)
            i += 4;
    } else if (mod == 0 && rm == 5) {
        i += 4;  // RIP-relative disp32
    }
    if (mod == 1)
        i += 1;
    else if (mod == 2)
        i += 4;
    if (op == 0xC6 || op == 0xC7) {  // the immediate follows the address bytes
        st->size = op == 0xC6 ? 1 : ((rex & 8) ? 8 : (op16 ? 2 : 4));
        const int isz = st->size == 8 ? 4 : st->size;  // imm32, sign-extended for 64-bit stores
        int64_t imm = 0;
        if (isz == 1)
            imm = (int8_t)ip[i];
        else if (isz == 2)
            imm = (int16_t)(ip[i] | (ip[i + 1] << 8));
        else
            imm = (int32_t)((uint32_t)ip[i] | ((uint32_t)ip[i + 1] << 8) | ((uint32_t)ip[i + 2] << 16) |
                            ((uint32_t)ip[i + 3] << 24));
        i += isz;
        st->value = (uint64_t)imm;
    } else if (op == 0x88) {
        st->size = 1;
        if (!rex && reg >= 4)  // AH, CH, DH, BH
            st->value = (uint64_t)g[x86_greg(reg - 4)] >> 8;
        else
            st->value = (uint64_t)g[x86_greg(reg | ((rex & 4) ? 8 : 0))];
    } else {
        st->size = (rex & 8) ? 8 : (op16 ? 2 : 4);
        st->value = (uint64_t)g[x86_greg(reg | ((rex & 4) ? 8 : 0))];
    }
    st->len = i;
    return true;
}

void retire_store(ucontext_t *uc, const Store &st)
{
    uc->uc_mcontext.gregs[REG_RIP] += st.len;
}
#elif defined(__aarch64__)
bool decode_store(const ucontext_t *uc, Store *st)
{
    const uint32_t insn = *reinterpret_cast<const uint32_t *>(uc->uc_mcontext.pc);
    const int rt = (int)(insn & 31), rn = (int)((insn >> 5) & 31);
    if ((insn & 0x3FC00000u) == 0x39000000u) {
        // STR (immediate, unsigned offset): size 111 0 01 00 imm12 Rn Rt
    } else if ((insn & 0x3FE00000u) == 0x38000000u) {
        // STUR / STR post-index / STTR / STR pre-index: size 111 0 00 00 0 imm9 idx Rn Rt
        const uint32_t idx = (insn >> 10) & 3;
        if (idx == 1 || idx == 3) {
            st->wb_reg = rn;
            st->wb_delta = (int64_t)((int32_t)(insn << 11) >> 23);  // imm9, sign-extended
        }
    } else if ((insn & 0x3FE00C00u) == 0x38200800u) {
        // STR (register offset): size 111 0 00 00 1 Rm option S 10 Rn Rt
    } else {
        return false;
    }
    st->size = 1 << (insn >> 30);
    st->value = rt == 31 ? 0 : (uint64_t)uc->uc_mcontext.regs[rt];  // register 31 is XZR here
    st->len = 4;
    return true;
}

void retire_store(ucontext_t *uc, const Store &st)
{
    if (st.wb_reg == 31)
        uc->uc_mcontext.sp += (uint64_t)st.wb_delta;
    else if (st.wb_reg >= 0)
        uc->uc_mcontext.regs[st.wb_reg] += (uint64_t)st.wb_delta;
    uc->uc_mcontext.pc += (uint64_t)st.len;
}
#else
bool decode_store(const ucontext_t *, Store *) { return false; }
void retire_store(ucontext_t *, const Store &) {}
#endif

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
    // a conflict: the page changed during this handler's park, by another
    // handler (with store emulation every write faults, the handler's own
    // later writes included)
    if (f.snap_valid && r->page_version[(size_t)p] > f.snapshot && r->page_writer[(size_t)p] != f.id) {
        ++r->conflicts;
        if (r->cfg.mode == CDET_ENFORCE) {
            ++r->restarts;
            siglongjmp(f.restart, 1);
        }
    }
    r->page_version[(size_t)p] = ++r->clock;
    r->page_writer[(size_t)p] = f.id;
    Store st;
    ucontext_t *ctx = static_cast<ucontext_t *>(uc);
    if (r->alias && decode_store(ctx, &st) &&
        (size_t)(a - r->region) % (size_t)r->page + (size_t)st.size <= (size_t)r->page) {
        std::memcpy(r->alias + (a - r->region), &st.value, (size_t)st.size);  // little-endian: the low bytes
        retire_store(ctx, st);
        ++r->emulated;
        return;
    }
    mprotect(r->region + (size_t)p * (size_t)r->page, (size_t)r->page, PROT_READ | PROT_WRITE);
    ++r->protect_calls;
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
    int rc;
    if (f.finished) {
        f.finished = false;
        rc = f.finished_rc;
    } else {
        rc = offload_poll(r.cfg.srv, f.ticket);
    }
    if (rc == AES_PENDING)
        return false;
    if (rc != AES_OK && !r.error)
        r.error = rc;
    return true;
}

// Reap, on their behalf, the completed offloads of other parked handlers:
// their slots are freed without any other handler running, so a handler
// waiting for a slot (or a serialized one) keeps its place in the order.
void reap_others(Run &r, Fiber &self)
{
    for (auto &g : r.fibers) {
        if (&g == &self || !g.parked || g.finished)
            continue;
        const int rc = offload_poll(r.cfg.srv, g.ticket);
        if (rc != AES_PENDING) {
            g.finished = true;
            g.finished_rc = rc;
        }
    }
}

bool offload_start(Run &r, Fiber &f, int req)
{
    if (!r.cfg.srv) {
        f.deadline = clk::now() + std::chrono::nanoseconds(r.cfg.offload_ns);
        return true;
    }
    const clk::time_point t0 = clk::now();
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
        if (rc == AES_EAGAIN && clk::now() - t0 > std::chrono::seconds(30))
            rc = AES_ETIMEOUT;  // no slot freed: the server is stuck
        if (rc != AES_EAGAIN) {
            if (!r.error)
                r.error = rc;
            return false;
        }
        // Every slot is held (more handlers than server slots): the holders
        // are parked handlers, whose completions only the event loop would
        // reap, and it cannot run while this handler waits here.
        reap_others(r, f);
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
        (cfg->store_mode != CDET_STORES_EMULATE && cfg->store_mode != CDET_STORES_UNPROTECT) ||
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
    void *m = MAP_FAILED;
    if (r.detector && cfg->store_mode == CDET_STORES_EMULATE) {
        // one memory object mapped twice: the handlers' view (read-only
        // while guarded) and the detector's writable alias
        const int fd = memfd_create("cdet_region", MFD_CLOEXEC);
        if (fd >= 0 && ftruncate(fd, (off_t)r.region_bytes) == 0) {
            m = mmap(nullptr, r.region_bytes, PROT_READ | PROT_WRITE, MAP_SHARED, fd, 0);
            void *al = m == MAP_FAILED ? MAP_FAILED
                                       : mmap(nullptr, r.region_bytes, PROT_READ | PROT_WRITE, MAP_SHARED, fd, 0);
            if (al == MAP_FAILED) {
                if (m != MAP_FAILED)
                    munmap(m, r.region_bytes);
                m = MAP_FAILED;
            } else {
                r.alias = static_cast<uint8_t *>(al);
            }
        }
        if (fd >= 0)
            close(fd);
    }
    if (m == MAP_FAILED)
        m = mmap(nullptr, r.region_bytes, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (m == MAP_FAILED)
        return AES_ENOMEM;
    r.region = static_cast<uint8_t *>(m);
    r.page_version.assign((size_t)r.npages, 0);
    r.page_writer.assign((size_t)r.npages, -1);
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
    if (r.alias)
        munmap(r.alias, r.region_bytes);
    res->final_count = total;
    res->lost_updates = (uint64_t)cfg->requests - total;
    res->conflicts = r.conflicts;
    res->restarts = r.restarts;
    res->elapsed_s = elapsed;
    res->emulated_stores = r.emulated;
    res->protect_calls = r.protect_calls;
    return r.error;
}

int cdet_store_selftest(int rounds, uint64_t *emulated, uint64_t *fallbacks)
{
    if (rounds < 1 || !emulated || !fallbacks)
        return AES_EINVAL;
    if (g_run)
        return AES_EINVAL;
    Run r;
    r.cfg = cdet_run_cfg_t{};
    r.cfg.mode = CDET_DETECT;
    r.page = sysconf(_SC_PAGESIZE);
    r.npages = 2;
    r.region_bytes = 2 * (size_t)r.page;
    r.detector = true;
    const int fd = memfd_create("cdet_selftest", MFD_CLOEXEC);
    if (fd < 0)
        return AES_ENOMEM;
    void *m = MAP_FAILED, *al = MAP_FAILED;
    if (ftruncate(fd, (off_t)r.region_bytes) == 0) {
        m = mmap(nullptr, r.region_bytes, PROT_READ | PROT_WRITE, MAP_SHARED, fd, 0);
        al = mmap(nullptr, r.region_bytes, PROT_READ | PROT_WRITE, MAP_SHARED, fd, 0);
    }
    close(fd);
    if (m == MAP_FAILED || al == MAP_FAILED) {
        if (m != MAP_FAILED)
            munmap(m, r.region_bytes);
        if (al != MAP_FAILED)
            munmap(al, r.region_bytes);
        return AES_ENOMEM;
    }
    r.region = static_cast<uint8_t *>(m);
    r.alias = static_cast<uint8_t *>(al);
    r.page_version.assign(2, 0);
    r.page_writer.assign(2, -1);
    r.fibers.resize(1);
    r.current = &r.fibers[0];  // no park: every fault is a plain guarded write
    std::vector<uint8_t> shadow(r.region_bytes, 0);
    struct sigaction sa {};
    sa.sa_sigaction = on_fault;
    sa.sa_flags = SA_SIGINFO;
    sigemptyset(&sa.sa_mask);
    if (sigaction(SIGSEGV, &sa, &g_prev_segv) != 0) {
        munmap(m, r.region_bytes);
        munmap(al, r.region_bytes);
        return AES_EINVAL;
    }
    g_run = &r;
    // Stores of every width at run-time offsets (base + scaled index, with
    // and without displacement), mirrored into a plain shadow copy; each
    // round starts with the region read-only again.
    volatile uint8_t *b8 = r.region;
    volatile uint16_t *b16 = reinterpret_cast<volatile uint16_t *>(r.region);
    volatile uint32_t *b32 = reinterpret_cast<volatile uint32_t *>(r.region);
    volatile uint64_t *b64 = reinterpret_cast<volatile uint64_t *>(r.region);
    uint64_t x = 0x9E3779B97F4A7C15ull;
    const size_t n64 = r.region_bytes / 8;
    for (int k = 0; k < rounds; ++k) {
        mprotect(r.region, r.region_bytes, PROT_READ);
        r.fibers[0].dirty_lo = 0;
        r.fibers[0].dirty_hi = -1;
        x ^= x << 13;
        x ^= x >> 7;
        x ^= x << 17;
        const size_t i = (size_t)(x % (n64 - 320));
        const uint64_t v = x * 0xD6E8FEB86659FD93ull;
        switch (k % 10) {
        case 6: {  // constants: stored from an immediate on x86-64
            b64[i] = 0x5A5A1234ull;
            const uint64_t t = 0x5A5A1234ull;
            std::memcpy(&shadow[8 * i], &t, 8);
            break;
        }
        case 7: {
            b16[4 * i + 1] = 0xBEEF;
            const uint16_t h = 0xBEEF;
            std::memcpy(&shadow[8 * i + 2], &h, 2);
            break;
        }
        case 8:
            b8[8 * i + 7] = 0x7F;
            shadow[8 * i + 7] = 0x7F;
            break;
        case 0:
            b64[i] = v;
            std::memcpy(&shadow[8 * i], &v, 8);
            break;
        case 1: {
            const uint32_t w = (uint32_t)(v >> 7);
            b32[2 * i + 1] = w;
            std::memcpy(&shadow[8 * i + 4], &w, 4);
            break;
        }
        case 2: {
            const uint16_t h = (uint16_t)(v >> 21);
            b16[4 * i + 3] = h;
            std::memcpy(&shadow[8 * i + 6], &h, 2);
            break;
        }
        case 3: {
            const uint8_t c = (uint8_t)(v >> 40);
            b8[8 * i + 5] = c;
            shadow[8 * i + 5] = c;
            break;
        }
        case 4:  // displacement past the index
            b64[i + 7] = v ^ (uint64_t)k;
            {
                const uint64_t t = v ^ (uint64_t)k;
                std::memcpy(&shadow[8 * (i + 7)], &t, 8);
            }
            break;
        case 5: {  // a displacement beyond 8 bits (2560 bytes past the index)
            const uint64_t t = ~v;
            b64[i + 319] = t;
            std::memcpy(&shadow[8 * (i + 319)], &t, 8);
            break;
        }
        default: {  // a stored value that is the index itself
            const uint64_t t = (uint64_t)i;
            b64[i] = t;
            std::memcpy(&shadow[8 * i], &t, 8);
            break;
        }
        }
    }
    sigaction(SIGSEGV, &g_prev_segv, nullptr);
    g_run = nullptr;
    mprotect(r.region, r.region_bytes, PROT_READ | PROT_WRITE);
    const bool same = std::memcmp(r.region, shadow.data(), r.region_bytes) == 0;
    *emulated = r.emulated;
    *fallbacks = r.protect_calls;
    munmap(m, r.region_bytes);
    munmap(al, r.region_bytes);
    return same ? AES_OK : AES_EDESC;
}

}  // extern "C"
