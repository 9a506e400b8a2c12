// tune.cu -- launch-shape table and the autotuner.
//
// For every (Nr, length bucket) the table holds the CTR kernel variant and
// shape to use when the caller asks for AES_VARIANT_AUTO.  Defaults come
// from occupancy arithmetic; aes_autotune() replaces them with the fastest
// candidate measured on this device with CUDA events.
#include "../../include/aesoffload.h"
#include "internal.h"
#include "runtime.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

namespace aesrt {

int len_bucket(size_t len)
{
    int b = 0;
    while (b + 1 < kLenBuckets && ((size_t)1 << (b + 1)) <= len)
        ++b;
    return b;
}

static int nr_index(int nr) { return nr == 10 ? 0 : (nr == 12 ? 1 : 2); }

int validate_ctr_shape(const CtrShape &s)
{
    if (s.variant == AES_VARIANT_BITSLICE)
        return s.threads == 128 && s.ctas >= 0 ? AES_OK : AES_EINVAL;
    if (s.variant != AES_VARIANT_TTABLE)
        return AES_EINVAL;
    if (s.threads < 32 || s.threads > 1024 || (s.threads & 31))
        return AES_EINVAL;
    if (s.nb != 1 && s.nb != 2 && s.nb != 4)
        return AES_EINVAL;
    return s.ctas >= 0 ? AES_OK : AES_EINVAL;
}

// Default: one T-table CTA per SM; as many threads as keep every SM busy.
static CtrShape default_shape(int nsm, int bucket)
{
    const uint64_t nblocks = ((uint64_t)1 << bucket) / 16 + 1;
    CtrShape s{AES_VARIANT_TTABLE, 256, 1, 0};
    if (nblocks >= (uint64_t)nsm * 1024 * 2 * 4)
        s = CtrShape{AES_VARIANT_TTABLE, 1024, 2, 0};
    else if (nblocks >= (uint64_t)nsm * 1024)
        s = CtrShape{AES_VARIANT_TTABLE, 1024, 1, 0};
    else if (nblocks >= (uint64_t)nsm * 512)
        s = CtrShape{AES_VARIANT_TTABLE, 512, 1, 0};
    return s;
}

void tune_defaults(DeviceState &st)
{
    for (int i = 0; i < 3; ++i)
        for (int b = 0; b < kLenBuckets; ++b)
            st.ctr_tuned[i][b] = default_shape(st.nsm, b);
    st.batch_tuned = BatchShape{AES_VARIANT_TTABLE, 512, 2048, 0, 2};
}

CtrShape tuned_ctr_shape(const DeviceState &st, size_t len, int nr)
{
    return st.ctr_tuned[nr_index(nr)][len_bucket(len)];
}

}  // namespace aesrt

using namespace aesrt;

namespace {

float time_ctr(aes_ctx_t ctx, const uint8_t *iv, void *buf_in, void *buf_out, size_t len,
               const aes_launch_t &cfg, cudaStream_t s, cudaEvent_t a, cudaEvent_t b, int reps)
{
    for (int w = 0; w < 2; ++w)
        if (aes_ctr_ex(ctx, iv, buf_in, buf_out, len, s, &cfg) != AES_OK)
            return -1.f;
    std::vector<float> t;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(a, s);
        aes_ctr_ex(ctx, iv, buf_in, buf_out, len, s, &cfg);
        cudaEventRecord(b, s);
        if (cudaEventSynchronize(b) != cudaSuccess)
            return -1.f;
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        t.push_back(ms);
    }
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

// The batch kernel's candidate shapes: T-table CTAs of 256, 512 (round keys
// in registers) and 1024 threads (keys in shared memory) x 1, 2 or 4 blocks
// per lane in flight x tiles of 4, 8 or 16 counter groups; and the bitsliced
// kernel (128-thread CTAs) x the same tiles.
std::vector<BatchShape> batch_candidates()
{
    std::vector<BatchShape> c;
    for (int tb : {1024, 2048, 4096}) {
        for (int th : {256, 512, 1024})
            for (int nb : {1, 2, 4})
                c.push_back(BatchShape{AES_VARIANT_TTABLE, th, tb, 0, nb});
        c.push_back(BatchShape{AES_VARIANT_BITSLICE, 128, tb, 0, 1});
    }
    return c;
}

// Time every candidate as a graph plan over `reqs` (median of `reps` launches
// after two warm-ups, CUDA events on `s`); the fastest in *pick.  Returns
// AES_OK, or the first error if no candidate ran.
int sweep_batch(DeviceState &st, const std::vector<aes_desc_t> &reqs, cudaStream_t s, cudaEvent_t a,
                cudaEvent_t b, int reps, BatchShape *pick, float *best_ms)
{
    float best = 1e30f;
    int err = AES_EINVAL;
    st.n_batch_results = 0;
    for (const BatchShape &c : batch_candidates()) {
        const int slot = st.n_batch_results < DeviceState::kMaxBatchCandidates ? st.n_batch_results++ : -1;
        if (slot >= 0) {
            st.batch_results[slot] = c;
            st.batch_results_ms[slot] = -1.f;
        }
        aes_batch_opts_t o{};
        o.variant = c.variant;
        o.threads = c.threads;
        o.tile_blocks = c.tile_blocks;
        o.blocks_per_thread = c.nb;
        aes_batch_plan_t plan = nullptr;
        if ((err = aes_batch_plan_create(&plan, reqs.data(), (int)reqs.size(), &o)) != AES_OK)
            continue;
        std::vector<float> t;
        for (int r = 0; r < reps + 2; ++r) {
            cudaEventRecord(a, s);
            const int lr = aes_batch_plan_launch(plan, s);
            cudaEventRecord(b, s);
            if (lr != AES_OK || cudaEventSynchronize(b) != cudaSuccess) {
                err = lr != AES_OK ? lr : AES_ECUDA;
                t.clear();
                break;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, a, b);
            if (r >= 2)
                t.push_back(ms);
        }
        aes_batch_plan_destroy(plan);
        if (t.empty())
            continue;
        std::sort(t.begin(), t.end());
        if (slot >= 0)
            st.batch_results_ms[slot] = t[t.size() / 2];
        if (t[t.size() / 2] < best) {
            best = t[t.size() / 2];
            *pick = c;
        }
    }
    if (best_ms)
        *best_ms = best;
    return best < 1e30f ? AES_OK : err;
}

// Batch shape on a synthetic mixed batch in [in, in + cap) -> [out, ...):
// lengths spread log-uniformly over 1 KiB .. 8 MiB by a fixed LCG, AES-128
// and AES-256 alternating, 256-byte aligned offsets.
int tune_batch(DeviceState &st, void *in, void *out, size_t cap, cudaStream_t s, cudaEvent_t a, cudaEvent_t b)
{
    const uint8_t key[32] = {7, 1, 3};
    aes_ctx_t ctx[2] = {nullptr, nullptr};
    int rc = aes_ctx_create(&ctx[0], key, 128);
    if (!rc)
        rc = aes_ctx_create(&ctx[1], key, 256);
    std::vector<aes_desc_t> reqs;
    uint64_t x = 0x2545F4914F6CDD1Dull;
    size_t off = 0;
    while (!rc && reqs.size() < 4096) {
        x = x * 6364136223846793005ull + 1442695040888963407ull;
        const double u = (double)(x >> 11) / 9007199254740992.0;  // [0, 1)
        const size_t len = (size_t)(1024.0 * std::pow(8192.0, u));
        if (off + len > cap)
            break;
        aes_desc_t d{};
        d.ctx = ctx[reqs.size() & 1];
        d.iv[15] = (uint8_t)(x >> 56);
        d.in = static_cast<const uint8_t *>(in) + off;
        d.out = static_cast<uint8_t *>(out) + off;
        d.len = len;
        reqs.push_back(d);
        off += (len + 255) / 256 * 256;
    }
    BatchShape pick = st.batch_tuned;
    if (!rc)
        rc = sweep_batch(st, reqs, s, a, b, 6, &pick, nullptr);
    aes_ctx_destroy(ctx[0]);
    aes_ctx_destroy(ctx[1]);
    if (!rc)
        st.batch_tuned = pick;
    return rc;
}

}  // namespace

extern "C" {

int aes_tuned_shape(size_t len, int bits, aes_launch_t *out)
{
    if (!out || (bits != 128 && bits != 192 && bits != 256))
        return AES_EINVAL;
    DeviceState *st = nullptr;
    int rc = device_state(&st);
    if (rc)
        return rc;
    const CtrShape s = tuned_ctr_shape(*st, len, bits / 32 + 6);
    out->variant = s.variant;
    out->threads = s.threads;
    out->blocks_per_thread = s.nb;
    uint32_t parts = 1;
    ctr_plan((len + 15) / 16, 0, s, st->nsm, &out->ctas, &parts);
    return AES_OK;
}

int aes_autotune(const char *path)
{
    DeviceState *st = nullptr;
    int rc = device_state(&st);
    if (rc)
        return rc;
    const int lo_b = 12, hi_b = 28;  // 4 KiB .. 256 MiB
    const size_t maxlen = (size_t)1 << hi_b;
    void *in = nullptr, *out = nullptr;
    cudaError_t e = cudaMalloc(&in, maxlen);
    if (!e)
        e = cudaMalloc(&out, maxlen);
    if (e) {
        cudaFree(in);
        return e == cudaErrorMemoryAllocation ? AES_ENOMEM : cuda_fail(e, "autotune alloc");
    }
    cudaMemset(in, 0x5a, maxlen);
    cudaStream_t s = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const uint8_t key[32] = {1, 2, 3};
    const uint8_t iv[16] = {9};
    const aes_launch_t cands[] = {
        {AES_VARIANT_TTABLE, 256, 1, 0},  {AES_VARIANT_TTABLE, 512, 1, 0},
        {AES_VARIANT_TTABLE, 1024, 1, 0}, {AES_VARIANT_TTABLE, 512, 2, 0},
        {AES_VARIANT_TTABLE, 1024, 2, 0}, {AES_VARIANT_TTABLE, 1024, 4, 0},
        {AES_VARIANT_BITSLICE, 128, 1, 0},
    };
    const int bits_list[3] = {128, 192, 256};
    for (int ki = 0; ki < 3 && rc == AES_OK; ++ki) {
        aes_ctx_t ctx = nullptr;
        if ((rc = aes_ctx_create(&ctx, key, bits_list[ki])))
            break;
        for (int bk = lo_b; bk <= hi_b; ++bk) {
            const size_t len = (size_t)1 << bk;
            const int reps = bk <= 20 ? 15 : (bk <= 24 ? 7 : 3);
            float best = 1e30f;
            CtrShape pick = st->ctr_tuned[ki][bk];
            for (const aes_launch_t &c : cands) {
                const float ms = time_ctr(ctx, iv, in, out, len, c, s, a, b, reps);
                if (ms > 0 && ms < best) {
                    best = ms;
                    pick = CtrShape{c.variant, c.threads, c.blocks_per_thread, 0};
                }
            }
            st->ctr_tuned[ki][bk] = pick;
        }
        for (int bk = 0; bk < lo_b; ++bk)
            st->ctr_tuned[ki][bk] = st->ctr_tuned[ki][lo_b];
        for (int bk = hi_b + 1; bk < kLenBuckets; ++bk)
            st->ctr_tuned[ki][bk] = st->ctr_tuned[ki][hi_b];
        aes_ctx_destroy(ctx);
    }
    if (rc == AES_OK)
        rc = tune_batch(*st, in, out, maxlen, s, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamDestroy(s);
    cudaFree(in);
    cudaFree(out);
    if (rc)
        return rc;
    if (path) {
        FILE *f = std::fopen(path, "w");
        if (!f)
            return AES_EINVAL;
        std::fprintf(f, "{\"device\": \"%s\", \"sms\": %d, \"ctr\": [\n", st->name, st->nsm);
        for (int ki = 0; ki < 3; ++ki)
            for (int bk = 0; bk < kLenBuckets; ++bk) {
                const CtrShape &c = st->ctr_tuned[ki][bk];
                std::fprintf(f, "  [%d, %d, %d, %d, %d]%s\n", ki, bk, c.variant, c.threads, c.nb,
                             (ki == 2 && bk == kLenBuckets - 1) ? "" : ",");
            }
        std::fprintf(f, "],\n\"batch\": [%d, %d, %d, %d]}\n", st->batch_tuned.variant,
                     st->batch_tuned.threads, st->batch_tuned.tile_blocks, st->batch_tuned.nb);
        std::fclose(f);
    }
    return AES_OK;
}

int aes_batch_autotune(const aes_desc_t *descs, int n, void *stream, aes_batch_opts_t *best)
{
    if (n < 1 || !descs)
        return AES_EINVAL;
    if (n > AES_BATCH_MAX)
        return AES_ETOOBIG;
    DeviceState *st = nullptr;
    int rc = device_state(&st);
    if (rc)
        return rc;
    const std::vector<aes_desc_t> reqs(descs, descs + n);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (!e)
        e = cudaEventCreate(&b);
    if (e) {
        if (a)
            cudaEventDestroy(a);
        return cuda_fail(e, "aes_batch_autotune events");
    }
    BatchShape pick = st->batch_tuned;
    rc = sweep_batch(*st, reqs, s, a, b, 5, &pick, nullptr);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc)
        return rc;
    st->batch_tuned = pick;
    if (best) {
        std::memset(best, 0, sizeof(*best));
        best->variant = pick.variant;
        best->threads = pick.threads;
        best->tile_blocks = pick.tile_blocks;
        best->ctas = pick.ctas;
        best->blocks_per_thread = pick.nb;
    }
    return AES_OK;
}

int aes_batch_tune_results(aes_batch_opts_t *shapes, float *ms, int cap)
{
    if (cap < 0 || (cap > 0 && (!shapes || !ms)))
        return AES_EINVAL;
    DeviceState *st = nullptr;
    int rc = device_state(&st);
    if (rc)
        return rc;
    const int n = st->n_batch_results < cap ? st->n_batch_results : cap;
    for (int i = 0; i < n; ++i) {
        std::memset(&shapes[i], 0, sizeof(shapes[i]));
        shapes[i].variant = st->batch_results[i].variant;
        shapes[i].threads = st->batch_results[i].threads;
        shapes[i].tile_blocks = st->batch_results[i].tile_blocks;
        shapes[i].blocks_per_thread = st->batch_results[i].nb;
        ms[i] = st->batch_results_ms[i];
    }
    return n;
}

int aes_batch_tuned_shape(aes_batch_opts_t *out)
{
    if (!out)
        return AES_EINVAL;
    DeviceState *st = nullptr;
    int rc = device_state(&st);
    if (rc)
        return rc;
    std::memset(out, 0, sizeof(*out));
    out->variant = st->batch_tuned.variant;
    out->threads = st->batch_tuned.threads;
    out->tile_blocks = st->batch_tuned.tile_blocks;
    out->ctas = st->batch_tuned.ctas;
    out->blocks_per_thread = st->batch_tuned.nb;
    return AES_OK;
}

int aes_autotune_load(const char *path)
{
    if (!path)
        return AES_EINVAL;
    DeviceState *st = nullptr;
    int rc = device_state(&st);
    if (rc)
        return rc;
    FILE *f = std::fopen(path, "r");
    if (!f)
        return AES_EINVAL;
    char line[512];
    int sms = -1;
    char name[256] = {0};
    int nread = 0;
    CtrShape table[3][kLenBuckets];
    std::memcpy(table, st->ctr_tuned, sizeof(table));
    BatchShape bs = st->batch_tuned;
    while (std::fgets(line, sizeof(line), f)) {
        int ki, bk, v, t, nb;
        if (std::sscanf(line, "{\"device\": \"%255[^\"]\", \"sms\": %d", name, &sms) == 2)
            continue;
        if (std::sscanf(line, " [%d, %d, %d, %d, %d]", &ki, &bk, &v, &t, &nb) == 5) {
            if (ki < 0 || ki > 2 || bk < 0 || bk >= kLenBuckets)
                continue;
            CtrShape c{v, t, nb, 0};
            if (validate_ctr_shape(c) == AES_OK) {
                table[ki][bk] = c;
                ++nread;
            }
            continue;
        }
        int tb = 0, bnb = 2;
        const int got = std::sscanf(line, "\"batch\": [%d, %d, %d, %d]", &v, &t, &tb, &bnb);
        if (got == 3 || got == 4) {  // three fields: written before blocks per lane were tuned (2)
            BatchShape c{v, t, tb, 0, got == 4 ? bnb : 2};
            if (validate_batch_shape(c) == AES_OK)
                bs = c;
        }
    }
    std::fclose(f);
    if (sms != st->nsm || std::strcmp(name, st->name) != 0)
        return AES_OK;  // measured elsewhere: keep the current table
    if (nread == 0)
        return AES_EINVAL;
    std::memcpy(st->ctr_tuned, table, sizeof(table));
    st->batch_tuned = bs;
    return AES_OK;
}

}  // extern "C"
