// served_protocol_sim.cpp -- host threads stand in for the served kernel's
// resident CTAs and run its request protocol (served_protocol.cuh, compiled
// for the host) against a producer that submits and reaps requests the way
// offload_submit / offload_poll do.  Each CTA is an agent thread running
// the kernel's agent loop and two worker threads taking tiles from the
// kernel's shared ring, as the kernel's worker warps do.  Checked: every tile of every request is processed exactly once
// and while its request still owns the slot, every request completes once
// with the right status, zero-length and rejected requests complete at
// dispatch, emulated offloads take one tile, and idle exits and relaunches
// behave.  Scenario 1 raises the stop flag with work in flight (every CTA
// must exit); scenario 2 queues an entry naming a slot the host never
// issues (the CTAs must stop with ERROR).  Logic only: host memory ordering
// is not the GPU's.
//
// usage: served_protocol_sim mode ctas slots requests tile_blocks idle_us seed [scenario [chaos [weak]]]
// (chaos n > 0: every protocol memory operation yields with probability 1/n;
//  weak 1: stores become visible late and out of order, as on the device)
#include "served_protocol.cuh"

#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <random>
#include <thread>
#include <vector>

using namespace srvp;

namespace {

constexpr int kMaxKeys = 4;

struct alignas(64) Word {
    unsigned long long v = 0;
};

struct Req {
    uint64_t len = 0;
    uint64_t iv_lo = 0;
    int key_slot = 0;
    bool valid = true;
    bool emulated = false;
    uint32_t ntiles = 0;                       // expected tile count
    std::unique_ptr<std::atomic<uint8_t>[]> marks;
    std::atomic<int> completions{0};
};

struct Tile {
    uint32_t d, t, seq;
};

// One stand-in CTA: the agent and kWorkers worker warps, joined by the
// kernel's own shared ring (served_protocol.cuh).
constexpr int kWorkers = 5;  // warps 1..5: partitions 1, 2, 3, 0, 1
struct Cta {
    Ring ring{};
    Cta() { ring_init(ring); }
};

struct Sim {
    int mode = 0, nctas = 4, slots = 64, nreq = 2000, tile_blocks = 0, scenario = 0;
    uint64_t idle_ns = 2000000;
    uint32_t seed = 1;

    Word cursor, adv, disp;
    std::vector<unsigned long long> ring;
    SrvRec *recs = nullptr;
    std::vector<uint4> keys;
    std::vector<int> key_nr;
    QEntry *queue = nullptr;  // one body per slot
    std::vector<uint64_t> order;
    uint32_t qsize = 1;
    std::vector<unsigned long long> done;
    unsigned int ctrl[16] = {};
    SrvParams P{};

    std::unique_ptr<Req[]> reqs;
    std::vector<unsigned long long> tracebuf;  // SRV_TRACE builds: stamps of every request
    std::atomic<int> errors{0};
    std::mutex err_mu;
    char first_error[256] = "";
    std::atomic<uint64_t> tiles_done{0};

    std::vector<std::thread> threads;
    std::vector<std::unique_ptr<Cta>> ctas;
    std::atomic<int> live{0};
    int launches = 0;

    void fail(const char *fmt, uint64_t a = 0, uint64_t b = 0, uint64_t c = 0)
    {
        std::lock_guard<std::mutex> lk(err_mu);
        if (errors.fetch_add(1) == 0)
            std::snprintf(first_error, sizeof(first_error), fmt, (unsigned long long)a, (unsigned long long)b,
                          (unsigned long long)c);
    }

    void setup()
    {
        ring.assign(kDispRing, 0);
        recs = static_cast<SrvRec *>(std::aligned_alloc(128, sizeof(SrvRec) * (size_t)slots));
        std::memset(recs, 0, sizeof(SrvRec) * (size_t)slots);
        keys.assign(15 * kMaxKeys, make_uint4(0, 0, 0, 0));
        key_nr.assign(kMaxKeys, 0);
        key_nr[0] = 10;
        key_nr[1] = 14;
        key_nr[2] = 12;  // key slot 3 stays unregistered: requests naming it are rejected
        while (qsize < (uint32_t)slots)
            qsize <<= 1;
        queue = static_cast<QEntry *>(std::aligned_alloc(64, sizeof(QEntry) * (size_t)slots));
        std::memset(queue, 0, sizeof(QEntry) * (size_t)slots);
        order.assign(qsize, 0);
        done.assign((size_t)slots, 0);
        disp.v = 1;                 // sequence numbers start at 1
        cursor.v = mode ? 1 : 0;    // per-request claims: low starts at the first sequence number
        P.cursor = &cursor.v;
        P.adv = &adv.v;
        P.disp = &disp.v;
        P.disp_ring = ring.data();
        P.recs = recs;
        P.keys = keys.data();
        P.queue = queue;
        P.order = order.data();
        P.done = done.data();
        P.stop = &ctrl[0];
        P.kstatus = &ctrl[1];
        P.te0 = nullptr;
        P.qmask = qsize - 1;
        P.max_keys = kMaxKeys;
        P.tile_blocks = (uint32_t)tile_blocks;
        P.nslots = (uint32_t)slots;
        P.nctas = (uint32_t)nctas;
        P.idle_ns = idle_ns;
        P.max_len = 1ull << 40;
#ifdef SRV_TRACE
        uint32_t tcap = 1;
        while (tcap < (uint32_t)nreq + 2)
            tcap <<= 1;
        tracebuf.assign((size_t)tcap * kTracePoints, 0);
        P.trace = tracebuf.data();
        P.trace_mask = tcap - 1;
#endif
    }

    // SRV_TRACE builds: every completed request's stamps come in protocol
    // order (dispatched, published, first claim, first pop, done; a request
    // without tiles: dispatched, published, done).
    void check_trace()
    {
#ifdef SRV_TRACE
        for (int i = 0; i < nreq && !errors.load(); ++i) {
            const unsigned long long *row = &tracebuf[(size_t)((i + 1) & P.trace_mask) * kTracePoints];
            const Req &r = reqs[(size_t)i];
            if (r.ntiles) {
                const uint32_t order[] = {kTrDispatch, kTrPublished, kTrFirstClaim, kTrFirstPop, kTrDone};
                for (int k = 0; k < 5; ++k)
                    if (!row[order[k]] || (k && row[order[k]] < row[order[k - 1]]))
                        fail("seq %llu: stamp %llu missing or out of order", (uint64_t)i + 1, order[k]);
            } else if (!row[kTrDispatch] || row[kTrPublished] < row[kTrDispatch] ||
                       row[kTrDone] < row[kTrPublished] || row[kTrFirstClaim]) {
                fail("seq %llu (no tiles): stamps out of order", (uint64_t)i + 1);
            }
        }
#endif
    }

    // The tile count dispatch gives a request (restated here to size the
    // per-tile marks and to check the record against).
    uint32_t tile_count(uint64_t len, uint64_t iv_lo) const
    {
        if (len == 0)
            return 0;
        const uint64_t nb = (len + 15) >> 4;
        const uint64_t groups = (((iv_lo & 255u) + nb - 1) >> 8) + 1;
        uint32_t tb = (uint32_t)tile_blocks;
        if (!tb) {
            tb = 64;
            while (tb < 1024 && (uint64_t)tb * 512 < nb)
                tb <<= 1;
        }
        const uint32_t tg = tb >= 256 ? tb / 256 : 1, tp = tb >= 256 ? 1 : 256 / tb;
        return (uint32_t)((groups + tg - 1) / tg * tp);
    }

    // The agent warp's lane 0: the kernel's own agent loop, then what the
    // kernel does with its exit code.
    template <bool PER_REQ>
    void agent_thread(Cta *c)
    {
        srvp::agent<PER_REQ>(P, c->ring);
        const uint32_t code = ld_vol(&c->ring.exit_code);
        if ((code & kExitError) && scenario != 2)
            fail("agent stopped with ERROR");
        if (code)
            __atomic_fetch_or(P.kstatus, code, __ATOMIC_RELAXED);
        drain_stores();  // a CTA's stores are visible once it has exited
        live.fetch_sub(1);
    }

    // A worker warp's lane 0: the kernel's ring_pop, the tile (checked here
    // instead of encrypted) and the kernel's completion step.
    void worker_thread(Cta *c, uint32_t warp)
    {
        for (;;) {
            Tile tl{};
            uint32_t nt = 0;
            if (!ring_pop(c->ring, warp, &tl.d, &tl.t, &tl.seq, &nt))
                break;
            if (tl.t == 0)
                trace(P, tl.seq, kTrFirstPop);
            // the kernel's worker reads the record's generation with the record
            const uint64_t gen = ld_cg(&recs[tl.d].gen);
            process(tl, nt);
            tile_finished(P, tl.d, nt, tl.seq, gen);
        }
        drain_stores();
        live.fetch_sub(1);
    }

    void process(const Tile &tl, uint32_t item_nt)
    {
        const uint64_t sn = ld_relaxed_gpu(&recs[tl.d].seq_ntiles);
        const uint32_t nt = (uint32_t)(sn & kTileMask);
        if ((uint32_t)(sn >> kTileBits) != tl.seq || tl.t >= nt) {
            fail("tile %llu of seq %llu: slot holds seq %llu", tl.t, tl.seq, sn >> kTileBits);
            return;
        }
        if (item_nt != nt) {
            fail("seq %llu: ring item says %llu tiles, record %llu", tl.seq, item_nt, nt);
            return;
        }
        const uint64_t idx = tl.seq - 1;
        if (idx >= (uint64_t)nreq) {
            fail("tile of unknown seq %llu", tl.seq);
            return;
        }
        Req &r = reqs[idx];
        if (nt != r.ntiles) {
            fail("seq %llu: record has %llu tiles, expected %llu", tl.seq, nt, r.ntiles);
            return;
        }
        if (r.marks[tl.t].exchange(1) != 0)
            fail("tile %llu of seq %llu processed twice", tl.t, tl.seq);
        tiles_done.fetch_add(1);
    }

    void launch()
    {
        for (auto &t : threads)
            t.join();
        threads.clear();
        ctas.clear();
        ctrl[1] = 0;
        ++launches;
        live.store(nctas * (1 + kWorkers));
        for (int i = 0; i < nctas; ++i) {
            ctas.emplace_back(new Cta());
            Cta *c = ctas.back().get();
            if (mode)
                threads.emplace_back([this, c] { agent_thread<true>(c); });
            else
                threads.emplace_back([this, c] { agent_thread<false>(c); });
            for (int w = 1; w <= kWorkers; ++w)
                threads.emplace_back([this, c, w] { worker_thread(c, (uint32_t)w); });
        }
    }

    // offload_submit's relaunch rule: start the CTAs again once all of them
    // have exited.
    void ensure_running()
    {
        if (live.load() == 0)
            launch();
    }

    int run()
    {
        setup();
        std::mt19937_64 g(seed);
        reqs.reset(new Req[(size_t)nreq]);
        for (int i = 0; i < nreq; ++i) {
            Req &r = reqs[(size_t)i];
            const int kind = (int)(g() % 20);
            if (kind == 0)
                r.len = 0;
            else if (kind < 12)
                r.len = 1 + g() % 8192;
            else if (kind < 18)
                r.len = 1 + g() % (256u << 10);
            else if (kind < 19)
                r.len = 1 + g() % (2u << 20);
            else
                r.len = 1 + g() % 5000;  // emulated: a duration in ns
            r.emulated = kind == 19;
            r.iv_lo = g();
            r.key_slot = (int)(g() % kMaxKeys);
            r.valid = r.emulated || key_nr[(size_t)r.key_slot] != 0;
            r.ntiles = r.emulated ? 1 : (r.valid ? tile_count(r.len, r.iv_lo) : 0);
            r.marks.reset(new std::atomic<uint8_t>[r.ntiles ? r.ntiles : 1]);
            for (uint32_t t = 0; t < r.ntiles; ++t)
                r.marks[t].store(0);
        }
        std::vector<uint32_t> free_slots;
        for (int i = slots - 1; i >= 0; --i)
            free_slots.push_back((uint32_t)i);
        std::vector<uint64_t> gen((size_t)slots, 0);
        std::vector<int64_t> owner((size_t)slots, -1);
        int inflight = 0, completed = 0;
        auto reap = [&]() {
            for (int d = 0; d < slots; ++d) {
                if (owner[(size_t)d] < 0)
                    continue;
                const uint64_t v = __atomic_load_n(&done[(size_t)d], __ATOMIC_ACQUIRE);
                if ((v >> 2) != gen[(size_t)d])
                    continue;
                Req &r = reqs[(size_t)owner[(size_t)d]];
                const uint32_t status = (uint32_t)(v & 3);
                if (status != (r.valid ? 1u : 2u))
                    fail("seq %llu completed with status %llu", (uint64_t)owner[(size_t)d] + 1, status);
                for (uint32_t t = 0; t < r.ntiles; ++t)
                    if (r.marks[t].load() != 1)
                        fail("seq %llu completed with tile %llu unprocessed", (uint64_t)owner[(size_t)d] + 1, t);
                r.completions.fetch_add(1);
                owner[(size_t)d] = -1;
                free_slots.push_back((uint32_t)d);
                --inflight;
                ++completed;
            }
        };
        launch();
        uint64_t seq = 1;
        auto t_start = std::chrono::steady_clock::now();
        auto timed_out = [&]() {
            return std::chrono::steady_clock::now() - t_start > std::chrono::seconds(60);
        };
        for (int i = 0; i < nreq && !errors.load(); ++i) {
            while (free_slots.empty() && !errors.load()) {
                reap();
                ensure_running();
                if (timed_out()) {
                    fail("no slot freed (in flight %llu)", (uint64_t)inflight);
                    break;
                }
                std::this_thread::yield();
            }
            if (errors.load())
                break;
            if (i % 400 == 399)  // a pause longer than the idle timeout: the CTAs exit
                std::this_thread::sleep_for(std::chrono::nanoseconds(3 * idle_ns));
            const uint32_t d = free_slots.back();
            free_slots.pop_back();
            const Req &r = reqs[(size_t)i];
            const uint64_t gn = ++gen[(size_t)d];
            owner[(size_t)d] = i;
            ++inflight;
            QEntry &qe = queue[d];  // offload_submit's layout: body in the slot, then the order word
            qe.in = r.len && !r.emulated ? 0x100000 : 0;
            qe.out = r.len && !r.emulated ? 0x200000 : 0;
            qe.len = r.len;
            qe.iv_hi = 0x0123456789abcdefull;
            qe.iv_lo = r.iv_lo;
            qe.gen = gn;
            qe.key_slot = (uint32_t)r.key_slot | (uint32_t)key_nr[(size_t)r.key_slot] << 24;  // slot | Nr
            qe.desc = (uint16_t)d;
            qe.flags = r.emulated ? (uint16_t)kFlagEmulated : 0;
            qe.tag = seq + 1;
            __atomic_store_n(&order[seq & (qsize - 1)], ((seq + 1) << 16) | d, __ATOMIC_RELEASE);
            ++seq;
            ensure_running();
            reap();
            if (scenario && i == nreq / 2) {
                // The invalid entry takes the next order word without a slot,
                // so first let every request complete (it must not reuse the
                // order word of one that is not dispatched yet).
                while (scenario == 2 && inflight > 0 && !errors.load()) {
                    reap();
                    ensure_running();
                    if (timed_out()) {
                        fail("%llu requests never completed", (uint64_t)inflight);
                        break;
                    }
                    std::this_thread::yield();
                }
                return finish_scenario(seq, inflight);
            }
        }
        while (inflight > 0 && !errors.load()) {
            reap();
            ensure_running();
            if (timed_out()) {
                fail("%llu requests never completed", (uint64_t)inflight);
                break;
            }
            std::this_thread::yield();
        }
        __atomic_store_n(&ctrl[0], 1u, __ATOMIC_RELAXED);  // stop
        for (auto &t : threads)
            t.join();
        uint64_t want_tiles = 0;
        for (int i = 0; i < nreq; ++i) {
            want_tiles += reqs[(size_t)i].ntiles;
            if (!errors.load() && reqs[(size_t)i].completions.load() != 1)
                fail("seq %llu completed %llu times", (uint64_t)i + 1, (uint64_t)reqs[(size_t)i].completions.load());
        }
        if (!errors.load() && tiles_done.load() != want_tiles)
            fail("%llu tiles processed, %llu expected", tiles_done.load(), want_tiles);
        check_trace();
        const HostStats &hs = host_stats();
        std::printf("%s mode=%d ctas=%d slots=%d requests=%d completed=%d tiles=%llu launches=%d "
                    "stale_retries=%llu recycled=%llu repairs=%llu %s\n",
                    errors.load() ? "FAIL" : "OK", mode, nctas, slots, nreq, completed,
                    (unsigned long long)tiles_done.load(), launches,
                    (unsigned long long)hs.stale_claim_retries.load(), (unsigned long long)hs.recycled_claims.load(),
                    (unsigned long long)hs.low_repairs.load(), first_error);
        std::free(recs);
        std::free(queue);
        return errors.load() ? 1 : 0;
    }

    // Wait (bounded) until every stand-in CTA has exited, then join them.
    bool all_exit(double seconds)
    {
        const auto t0 = std::chrono::steady_clock::now();
        while (live.load() > 0) {
            if (std::chrono::steady_clock::now() - t0 > std::chrono::duration<double>(seconds))
                return false;
            std::this_thread::sleep_for(std::chrono::microseconds(100));
        }
        for (auto &t : threads)
            t.join();
        threads.clear();
        return true;
    }

    // Scenario 1: stop with requests in flight.  Scenario 2: an entry the
    // host never writes (slot beyond nslots) stops the CTAs with ERROR.
    int finish_scenario(uint64_t seq, int inflight)
    {
        const char *what = "stop";
        if (scenario == 1) {
            __atomic_store_n(&ctrl[0], 1u, __ATOMIC_RELAXED);
            if (!all_exit(10.0))
                fail("CTAs still running 10 s after the stop flag (in flight %llu)", (uint64_t)inflight);
            else if (!(__atomic_load_n(&ctrl[1], __ATOMIC_RELAXED) & kExitStop))
                fail("no CTA reported STOP (status %llu)", __atomic_load_n(&ctrl[1], __ATOMIC_RELAXED));
        } else {
            what = "bad entry";
            __atomic_store_n(&order[seq & (qsize - 1)], ((seq + 1) << 16) | 0xffffu, __ATOMIC_RELEASE);
            // Like offload_poll's relaunch rule: a launch that ended idle (its
            // CTAs left just as requests arrived) is relaunched; one that ended
            // with ERROR is not.
            const auto t0 = std::chrono::steady_clock::now();
            for (;;) {
                if (!all_exit(10.0 + 2e-9 * (double)idle_ns)) {
                    fail("CTAs still running after an invalid queue entry");
                    break;
                }
                if (__atomic_load_n(&ctrl[1], __ATOMIC_RELAXED) & kExitError)
                    break;
                if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(30)) {
                    fail("no CTA reported ERROR (status %llu)", __atomic_load_n(&ctrl[1], __ATOMIC_RELAXED));
                    break;
                }
                launch();
            }
            __atomic_store_n(&ctrl[0], 1u, __ATOMIC_RELAXED);
        }
        std::printf("%s mode=%d scenario=%s ctas=%d tiles=%llu status=%u %s\n", errors.load() ? "FAIL" : "OK",
                    mode, what, nctas, (unsigned long long)tiles_done.load(), ctrl[1], first_error);
        std::free(recs);
        std::free(queue);
        return errors.load() ? 1 : 0;
    }
};

}  // namespace

int main(int argc, char **argv)
{
    if (argc < 8 || argc > 11) {
        std::fprintf(stderr, "usage: %s mode ctas slots requests tile_blocks idle_us seed [scenario [chaos [weak]]]\n",
                     argv[0]);
        return 2;
    }
    Sim s;
    s.mode = std::atoi(argv[1]);
    s.nctas = std::atoi(argv[2]);
    s.slots = std::atoi(argv[3]);
    s.nreq = std::atoi(argv[4]);
    s.tile_blocks = std::atoi(argv[5]);
    s.idle_ns = 1000ull * (uint64_t)std::atoll(argv[6]);
    s.seed = (uint32_t)std::atoi(argv[7]);
    s.scenario = argc >= 9 ? std::atoi(argv[8]) : 0;
    srvp::chaos_period() = argc >= 10 ? std::atoi(argv[9]) : 0;
    srvp::weak_stores() = argc >= 11 && std::atoi(argv[10]) != 0;
    return s.run();
}
