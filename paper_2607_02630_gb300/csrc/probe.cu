// probe.cu -- aes_measure_peaks: the per-SM issue rates and the host-link
// bandwidths behind the roofline the benchmark reports.
//
// The AES-CTR path is bound on chip (T-table lookups in shared memory, or
// the logic ops of the bitsliced circuit), and end to end by NVLink-C2C, so
// the roofline's denominators are rates this device must be measured for:
//   - conflict-free 32-bit shared-memory loads per SM clock: each thread
//     walks 8 independent pointer chains through a 32 KiB table laid out like
//     the lane-replicated T-tables (entry e, lane l at word 32e + l), one
//     ld.shared per step with the address taken from the previous load, so
//     nothing but the loads issues;
//   - three-input logic (lop3.b32), byte permute (prmt.b32) and 32-bit add
//     lanes per SM clock: 8 independent dependency chains per thread;
//   - copy-engine bandwidth host->device, device->host and both at once
//     (pinned host memory, cudaMemcpyAsync), and the zero-copy bandwidth of a
//     kernel that reads pinned host memory and writes pinned host memory over
//     the link at the same time (the end-to-end path's access pattern).
// Rates per clock come from clock64() on each SM (per-SM cycles, %smid), so
// they do not depend on the clock the GPU runs at; bandwidths from CUDA
// events.  Every loop has a fixed trip count and every index stays inside its
// table or buffer.
#include "../../include/aesoffload.h"
#include "internal.h"
#include "runtime.h"

#include <algorithm>
#include <cstring>
#include <vector>

namespace {

constexpr int kProbeThreads = 1024;
constexpr int kCtasPerSm = 2;
constexpr int kChains = 8;
constexpr uint32_t kTableWords = 256 * 32;  // 32 KiB

struct CtaStamp {
    unsigned long long start, end;
    uint32_t smid, pad;
};

__device__ __forceinline__ uint32_t smid()
{
    uint32_t s;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
    return s;
}

__device__ __forceinline__ void stamp_begin(CtaStamp *st, unsigned long long &t0)
{
    __syncthreads();
    t0 = clock64();
    (void)st;
}

__device__ __forceinline__ void stamp_end(CtaStamp *st, unsigned long long t0)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        st[blockIdx.x].start = t0;
        st[blockIdx.x].end = clock64();
        st[blockIdx.x].smid = smid();
    }
}

// Shared-memory lookups: 8 chains per thread; word 32e + l holds the shared
// address of word 32 * next(e) + l, next(e) = (167 e + 13) mod 256, so lane l
// always reads bank l (conflict-free) and every step is one ld.shared.
__global__ void __launch_bounds__(kProbeThreads) probe_lds(int iters, CtaStamp *st, uint32_t *sink)
{
    __shared__ uint32_t tab[kTableWords];
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(tab);
    for (uint32_t w = threadIdx.x; w < kTableWords; w += blockDim.x) {
        const uint32_t e = w >> 5, l = w & 31u;
        tab[w] = base + 4u * (32u * ((167u * e + 13u) & 255u) + l);
    }
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j)
        a[j] = base + 4u * (32u * ((uint32_t)(threadIdx.x >> 5) * 8u + (uint32_t)j & 255u) + lane);
    unsigned long long t0;
    stamp_begin(st, t0);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j < kChains; ++j)
                asm volatile("ld.shared.u32 %0, [%0];" : "+r"(a[j]));
    }
    stamp_end(st, t0);
    uint32_t x = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j)
        x ^= a[j];
    if (x == 0x12345678u)  // never true in practice; keeps the chains live
        sink[0] = x;
}

// Arithmetic issue: 8 independent chains of one instruction kind per thread.
template <int OP>
__global__ void __launch_bounds__(kProbeThreads) probe_alu(int iters, uint32_t seed, CtaStamp *st, uint32_t *sink)
{
    uint32_t a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j)
        a[j] = seed * (threadIdx.x + 1u) + (uint32_t)j * 0x9E3779B9u;
    const uint32_t b = seed ^ 0x5bd1e995u, c = seed + 0x27d4eb2fu;
    unsigned long long t0;
    stamp_begin(st, t0);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j < kChains; ++j) {
                if (OP == 0)
                    asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[j]) : "r"(b), "r"(c));
                else if (OP == 1)
                    asm volatile("prmt.b32 %0, %0, %1, 0x5410;" : "+r"(a[j]) : "r"(b));
                else
                    asm volatile("add.u32 %0, %0, %1;" : "+r"(a[j]) : "r"(b));
            }
    }
    stamp_end(st, t0);
    uint32_t x = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j)
        x ^= a[j];
    if (x == 0x12345678u)
        sink[0] = x;
}

// Zero-copy: read `in` and write `out` (device aliases of pinned host
// memory) 16 bytes at a time, grid-stride.
__global__ void probe_zero_copy(const uint4 *__restrict__ in, uint4 *__restrict__ out, size_t n16)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x)
        out[i] = in[i];
}

// Median over SMs of (operations on the SM) / (cycles from its first CTA's
// start to its last CTA's end).
double per_sm_rate(const std::vector<CtaStamp> &st, double ops_per_cta, int nsm)
{
    std::vector<unsigned long long> lo(nsm, ~0ull), hi(nsm, 0);
    std::vector<int> ctas(nsm, 0);
    for (const CtaStamp &s : st) {
        if ((int)s.smid >= nsm)
            continue;
        lo[s.smid] = std::min(lo[s.smid], s.start);
        hi[s.smid] = std::max(hi[s.smid], s.end);
        ++ctas[s.smid];
    }
    std::vector<double> r;
    for (int k = 0; k < nsm; ++k)
        if (ctas[k] && hi[k] > lo[k])
            r.push_back(ops_per_cta * ctas[k] / (double)(hi[k] - lo[k]));
    if (r.empty())
        return 0.0;
    std::sort(r.begin(), r.end());
    return r[r.size() / 2];
}

struct Probe {
    cudaStream_t s = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    CtaStamp *d_st = nullptr;
    uint32_t *d_sink = nullptr;
    int nsm = 0, ctas = 0;
    ~Probe()
    {
        if (d_st)
            cudaFree(d_st);
        if (d_sink)
            cudaFree(d_sink);
        if (a)
            cudaEventDestroy(a);
        if (b)
            cudaEventDestroy(b);
        if (s)
            cudaStreamDestroy(s);
    }
    // launch the rate kernel `k` once (warm-up) and once timed; returns the
    // per-SM rate of `ops_per_thread_iter` operations a thread per iteration
    template <class L>
    cudaError_t rate(L launch, int iters, double ops_per_thread_iter, double *out, double *mhz)
    {
        cudaError_t e = launch(iters / 8);
        if (!e)
            e = cudaEventRecord(a, s);
        if (!e)
            e = launch(iters);
        if (!e)
            e = cudaEventRecord(b, s);
        if (!e)
            e = cudaStreamSynchronize(s);
        if (e)
            return e;
        std::vector<CtaStamp> st((size_t)ctas);
        if ((e = cudaMemcpy(st.data(), d_st, sizeof(CtaStamp) * st.size(), cudaMemcpyDeviceToHost)))
            return e;
        *out = per_sm_rate(st, ops_per_thread_iter * iters * kProbeThreads, nsm);
        if (mhz) {
            float ms = 0;
            cudaEventElapsedTime(&ms, a, b);
            unsigned long long cyc = 0;
            for (const CtaStamp &c : st)
                cyc = std::max(cyc, c.end - c.start);
            *mhz = ms > 0 ? (double)cyc / (ms * 1e3) : 0.0;
        }
        return cudaSuccess;
    }
};

float time_copy(cudaStream_t s1, cudaStream_t s2, cudaEvent_t a, cudaEvent_t b, cudaEvent_t c, void *dst1,
                const void *src1, cudaMemcpyKind k1, void *dst2, const void *src2, cudaMemcpyKind k2, size_t n)
{
    // s2 == nullptr: one copy on s1; else both at once (s2 waits for s1's start)
    std::vector<float> t;
    for (int r = 0; r < 4; ++r) {
        cudaEventRecord(a, s1);
        cudaMemcpyAsync(dst1, src1, n, k1, s1);
        if (s2) {
            cudaStreamWaitEvent(s2, a, 0);
            cudaMemcpyAsync(dst2, src2, n, k2, s2);
            cudaEventRecord(c, s2);
            cudaStreamWaitEvent(s1, c, 0);
        }
        cudaEventRecord(b, s1);
        if (cudaEventSynchronize(b) != cudaSuccess)
            return -1.f;
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (r)
            t.push_back(ms);
    }
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

}  // namespace

using namespace aesrt;

extern "C" int aes_measure_peaks(aes_peaks_t *out)
{
    if (!out)
        return AES_EINVAL;
    std::memset(out, 0, sizeof(*out));
    DeviceState *st = nullptr;
    int rc = device_state(&st);
    if (rc)
        return rc;
    Probe p;
    p.nsm = st->nsm;
    p.ctas = st->nsm * kCtasPerSm;
    cudaError_t e = cudaStreamCreateWithFlags(&p.s, cudaStreamNonBlocking);
    if (!e)
        e = cudaEventCreate(&p.a);
    if (!e)
        e = cudaEventCreate(&p.b);
    if (!e)
        e = cudaMalloc(&p.d_st, sizeof(CtaStamp) * (size_t)p.ctas);
    if (!e)
        e = cudaMalloc(&p.d_sink, 256);
    if (e)
        return e == cudaErrorMemoryAllocation ? AES_ENOMEM : cuda_fail(e, "aes_measure_peaks set-up");
    out->sms = st->nsm;
    const int iters = 4096;
    auto lds = [&](int it) {
        probe_lds<<<p.ctas, kProbeThreads, 0, p.s>>>(it, p.d_st, p.d_sink);
        return cudaGetLastError();
    };
    double mhz = 0;
    if ((e = p.rate(lds, iters, 4.0 * kChains, &out->lds32_per_clk_sm, &mhz)))
        return cuda_fail(e, "probe_lds");
    out->sm_mhz_during_probe = mhz;
    auto lop3 = [&](int it) {
        probe_alu<0><<<p.ctas, kProbeThreads, 0, p.s>>>(it, 0x1234567u, p.d_st, p.d_sink);
        return cudaGetLastError();
    };
    if ((e = p.rate(lop3, iters, 4.0 * kChains, &out->lop3_per_clk_sm, nullptr)))
        return cuda_fail(e, "probe_lop3");
    auto prmt = [&](int it) {
        probe_alu<1><<<p.ctas, kProbeThreads, 0, p.s>>>(it, 0x1234567u, p.d_st, p.d_sink);
        return cudaGetLastError();
    };
    if ((e = p.rate(prmt, iters, 4.0 * kChains, &out->prmt_per_clk_sm, nullptr)))
        return cuda_fail(e, "probe_prmt");
    auto iadd = [&](int it) {
        probe_alu<2><<<p.ctas, kProbeThreads, 0, p.s>>>(it, 0x1234567u, p.d_st, p.d_sink);
        return cudaGetLastError();
    };
    if ((e = p.rate(iadd, iters, 4.0 * kChains, &out->iadd_per_clk_sm, nullptr)))
        return cuda_fail(e, "probe_iadd");

    // host link: 256 MiB each way
    const size_t n = (size_t)256 << 20;
    void *h_in = nullptr, *h_out = nullptr, *d_a = nullptr, *d_b = nullptr;
    cudaStream_t s2 = nullptr;
    cudaEvent_t c = nullptr;
    e = cudaHostAlloc(&h_in, n, cudaHostAllocMapped | cudaHostAllocPortable);
    if (!e)
        e = cudaHostAlloc(&h_out, n, cudaHostAllocMapped | cudaHostAllocPortable);
    if (!e)
        e = cudaMalloc(&d_a, n);
    if (!e)
        e = cudaMalloc(&d_b, n);
    if (!e)
        e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
    if (!e)
        e = cudaEventCreate(&c);
    if (!e) {
        std::memset(h_in, 0x3c, n);
        std::memset(h_out, 0, n);
        const float h2d = time_copy(p.s, nullptr, p.a, p.b, c, d_a, h_in, cudaMemcpyHostToDevice, nullptr, nullptr,
                                    cudaMemcpyHostToDevice, n);
        const float d2h = time_copy(p.s, nullptr, p.a, p.b, c, h_out, d_b, cudaMemcpyDeviceToHost, nullptr, nullptr,
                                    cudaMemcpyDeviceToHost, n);
        const float both = time_copy(p.s, s2, p.a, p.b, c, d_a, h_in, cudaMemcpyHostToDevice, h_out, d_b,
                                     cudaMemcpyDeviceToHost, n);
        out->h2d_gbs = h2d > 0 ? n / (h2d * 1e-3) / 1e9 : 0.0;
        out->d2h_gbs = d2h > 0 ? n / (d2h * 1e-3) / 1e9 : 0.0;
        out->h2d_d2h_each_way_gbs = both > 0 ? n / (both * 1e-3) / 1e9 : 0.0;
        void *din = nullptr, *dout = nullptr;
        e = cudaHostGetDevicePointer(&din, h_in, 0);
        if (!e)
            e = cudaHostGetDevicePointer(&dout, h_out, 0);
        std::vector<float> t;
        for (int r = 0; r < 4 && !e; ++r) {
            cudaEventRecord(p.a, p.s);
            probe_zero_copy<<<st->nsm * 8, 256, 0, p.s>>>(static_cast<const uint4 *>(din), static_cast<uint4 *>(dout),
                                                         n / 16);
            cudaEventRecord(p.b, p.s);
            e = cudaEventSynchronize(p.b);
            float ms = 0;
            cudaEventElapsedTime(&ms, p.a, p.b);
            if (r)
                t.push_back(ms);
        }
        if (!e && !t.empty()) {
            std::sort(t.begin(), t.end());
            out->zero_copy_each_way_gbs = n / (t[t.size() / 2] * 1e-3) / 1e9;
        }
    }
    if (c)
        cudaEventDestroy(c);
    if (s2)
        cudaStreamDestroy(s2);
    cudaFree(d_a);
    cudaFree(d_b);
    cudaFreeHost(h_in);
    cudaFreeHost(h_out);
    if (e)
        return e == cudaErrorMemoryAllocation ? AES_ENOMEM : cuda_fail(e, "aes_measure_peaks link");
    return AES_OK;
}
