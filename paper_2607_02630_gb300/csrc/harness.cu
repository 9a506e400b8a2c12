// harness.cu -- open-loop drivers for the served and per-call paths.
//
// The paper measures latency under offered load with open-loop Poisson
// arrivals and reports median and tail latency (Sec. 6, "Latency under
// offered load"), and its servers hand offloads to a pool of executor
// threads (Sec. 3, Listing 1).  These drivers reproduce that measurement on
// the library's own entry points: `nthreads` submitter threads, thread k
// owning requests k, k + nthreads, ...; each request is submitted at its
// scheduled arrival time (never earlier; late if the thread is behind, which
// counts against the latency, so there is no coordinated omission), and its
// latency is the time from the scheduled arrival to the moment the thread
// observes completion.  The served driver also runs the paper's blocking
// server (a thread takes its next request only when the previous offload is
// done) and the controlled emulated offload of its load study.
#include "../../include/aesoffload.h"
#include "internal.h"
#include "runtime.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <deque>
#include <thread>
#include <vector>

namespace {

using clk = std::chrono::steady_clock;

double seconds_since(clk::time_point t0)
{
    return std::chrono::duration<double>(clk::now() - t0).count();
}

struct Shared {
    std::atomic<uint64_t> bytes{0}, retries{0};
    std::atomic<int> errors{0};
    std::atomic<double> last_done{0.0};
    std::atomic<bool> timed_out{false};
};

// A driver gives up when no request of its thread has completed for this
// long (a stuck or failed device), marking what is left as failed.
constexpr double kNoProgressSeconds = 30.0;

void note_done(Shared &sh, double t)
{
    double cur = sh.last_done.load();
    while (t > cur && !sh.last_done.compare_exchange_weak(cur, t)) {
    }
}

}  // namespace

using namespace aesrt;

extern "C" {

int offload_drive_ex(offload_server_t srv, const aes_drive_req_t *reqs, int n, int nthreads,
                     const aes_drive_opts_t *opts, double *latency_us, aes_drive_result_t *res)
{
    if (!srv || (n > 0 && (!reqs || !latency_us)) || n < 0 || nthreads < 1 || nthreads > 256 || !res)
        return AES_EINVAL;
    const bool blocking = opts && opts->blocking;
    const uint64_t emulated_ns = opts ? opts->emulated_ns : 0;
    int dev = 0;
    cudaGetDevice(&dev);
    Shared sh;
    const clk::time_point t0 = clk::now();
    auto submit = [&](int i, uint64_t *t) {
        const aes_drive_req_t &r = reqs[i];
        return emulated_ns ? offload_submit_emulated(srv, emulated_ns, t)
                           : offload_submit(srv, r.key_slot, r.iv, r.in, r.out, r.len, t);
    };
    auto finish = [&](int idx, int rc, double now) {
        if (rc == AES_OK) {
            latency_us[idx] = (now - reqs[idx].arrival_s) * 1e6;
            sh.bytes.fetch_add(emulated_ns ? 0 : reqs[idx].len);
            note_done(sh, now);
        } else {
            latency_us[idx] = -1.0;
            sh.errors.fetch_add(1);
        }
    };
    auto worker = [&](int k) {
        cudaSetDevice(dev);
        std::vector<std::pair<uint64_t, int>> pending;  // (ticket, request index)
        int next = k;
        double last_progress = seconds_since(t0);
        while (next < n || !pending.empty()) {
            if (seconds_since(t0) - last_progress > kNoProgressSeconds) {
                sh.timed_out.store(true);
                int failed = (int)pending.size();
                for (auto &pr : pending)
                    latency_us[pr.second] = -1.0;
                for (; next < n; next += nthreads, ++failed)
                    latency_us[next] = -1.0;
                sh.errors.fetch_add(failed);
                break;
            }
            // blocking: a request is taken only once the previous one is done
            if (next < n && (!blocking || pending.empty()) && seconds_since(t0) >= reqs[next].arrival_s) {
                uint64_t t = 0;
                const int rc = submit(next, &t);
                if (rc == AES_OK) {
                    pending.emplace_back(t, next);
                    next += nthreads;
                    last_progress = seconds_since(t0);
                } else if (rc == AES_EAGAIN) {
                    sh.retries.fetch_add(1);  // back-pressure: poll below, then retry
                } else {
                    finish(next, rc, 0.0);
                    next += nthreads;
                }
            }
            for (size_t i = 0; i < pending.size();) {
                const int rc = offload_poll(srv, pending[i].first);
                if (rc == AES_PENDING) {
                    ++i;
                    continue;
                }
                const double now = seconds_since(t0);
                last_progress = now;
                finish(pending[i].second, rc, now);
                pending[i] = pending.back();
                pending.pop_back();
            }
        }
    };
    std::vector<std::thread> th;
    for (int k = 0; k < nthreads; ++k)
        th.emplace_back(worker, k);
    for (auto &t : th)
        t.join();
    const double first = n ? reqs[0].arrival_s : 0.0;
    res->elapsed_s = sh.last_done.load() - first;
    res->bytes = sh.bytes.load();
    res->eagain_retries = sh.retries.load();
    res->errors = sh.errors.load();
    return sh.timed_out.load() ? AES_ETIMEOUT : AES_OK;
}

int offload_drive(offload_server_t srv, const aes_drive_req_t *reqs, int n, int nthreads,
                  double *latency_us, aes_drive_result_t *res)
{
    return offload_drive_ex(srv, reqs, n, nthreads, nullptr, latency_us, res);
}

int aes_ctr_drive(const aes_ctx_t *ctxs, int nctx, const aes_drive_req_t *reqs, int n, int nthreads,
                  double *latency_us, aes_drive_result_t *res)
{
    if (!ctxs || nctx < 1 || (n > 0 && (!reqs || !latency_us)) || n < 0 || nthreads < 1 || nthreads > 256 ||
        !res)
        return AES_EINVAL;
    for (int i = 0; i < n; ++i)
        if (reqs[i].key_slot < 0 || reqs[i].key_slot >= nctx)
            return AES_EINVAL;
    int dev = 0;
    cudaGetDevice(&dev);
    Shared sh;
    const clk::time_point t0 = clk::now();
    auto worker = [&](int k) {
        cudaSetDevice(dev);
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            int failed = 0;
            for (int i = k; i < n; i += nthreads, ++failed)
                latency_us[i] = -1.0;
            sh.errors.fetch_add(failed);
            return;
        }
        constexpr int kMaxPending = 256;
        std::vector<cudaEvent_t> free_ev;
        for (int i = 0; i < kMaxPending; ++i) {
            cudaEvent_t e;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess)
                free_ev.push_back(e);
        }
        // Events recorded on one stream complete in the order they were
        // recorded, so only the oldest pending one is queried: a thread
        // makes at most one cudaEventQuery per loop pass however many of
        // its requests are in flight (querying every pending event made
        // eight threads contend on the driver and capped the baseline far
        // below what the same launches sustain from one stream).
        std::deque<std::pair<cudaEvent_t, int>> pending;
        int next = k;
        double last_progress = seconds_since(t0);
        while (next < n || !pending.empty()) {
            if (seconds_since(t0) - last_progress > kNoProgressSeconds) {
                sh.timed_out.store(true);
                int failed = (int)pending.size();
                for (auto &pr : pending)
                    latency_us[pr.second] = -1.0;
                for (; next < n; next += nthreads, ++failed)
                    latency_us[next] = -1.0;
                sh.errors.fetch_add(failed);
                break;
            }
            if (next < n && !free_ev.empty() && seconds_since(t0) >= reqs[next].arrival_s) {
                const aes_drive_req_t &r = reqs[next];
                const int rc = aes_ctr(ctxs[r.key_slot], r.iv, r.in, r.out, r.len, s);
                cudaEvent_t e = free_ev.back();
                if (rc == AES_OK && cudaEventRecord(e, s) == cudaSuccess) {
                    free_ev.pop_back();
                    pending.emplace_back(e, next);
                    last_progress = seconds_since(t0);
                } else {
                    latency_us[next] = -1.0;
                    sh.errors.fetch_add(1);
                }
                next += nthreads;
            }
            while (!pending.empty()) {
                const cudaError_t q = cudaEventQuery(pending.front().first);
                if (q == cudaErrorNotReady)
                    break;
                const int idx = pending.front().second;
                const double now = seconds_since(t0);
                last_progress = now;
                if (q == cudaSuccess) {
                    latency_us[idx] = (now - reqs[idx].arrival_s) * 1e6;
                    sh.bytes.fetch_add(reqs[idx].len);
                    note_done(sh, now);
                } else {
                    latency_us[idx] = -1.0;
                    sh.errors.fetch_add(1);
                }
                free_ev.push_back(pending.front().first);
                pending.pop_front();
            }
        }
        cudaStreamSynchronize(s);
        for (auto &pr : pending)
            free_ev.push_back(pr.first);
        for (cudaEvent_t e : free_ev)
            cudaEventDestroy(e);
        cudaStreamDestroy(s);
    };
    std::vector<std::thread> th;
    for (int k = 0; k < nthreads; ++k)
        th.emplace_back(worker, k);
    for (auto &t : th)
        t.join();
    const double first = n ? reqs[0].arrival_s : 0.0;
    res->elapsed_s = sh.last_done.load() - first;
    res->bytes = sh.bytes.load();
    res->eagain_retries = 0;
    res->errors = sh.errors.load();
    return sh.timed_out.load() ? AES_ETIMEOUT : AES_OK;
}

}  // extern "C"
