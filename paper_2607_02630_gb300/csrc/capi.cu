// capi.cu -- the C ABI: status codes, per-device state, key contexts and the
// single-buffer CTR entry points.  Batch and served entry points live in
// batch.cu and server.cu; shared host helpers are in runtime.h.
#include "../../include/aesoffload.h"
#include "internal.h"
#include "runtime.h"

#include <cstring>
#include <mutex>
#include <new>

namespace aesrt {

thread_local char g_last_error[256] = "";

int cuda_fail(cudaError_t e, const char *where)
{
    std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(e));
    return AES_ECUDA;
}

static DeviceState g_devices[kMaxDevices];
static std::mutex g_dev_mutex;

int device_state(DeviceState **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return AES_EINVAL;
    DeviceState &st = g_devices[dev];
    if (st.ready.load(std::memory_order_acquire)) {
        *out = &st;
        return AES_OK;
    }
    std::lock_guard<std::mutex> lock(g_dev_mutex);
    if (!st.ready.load(std::memory_order_relaxed)) {
        st.device = dev;
        if ((e = cudaDeviceGetAttribute(&st.nsm, cudaDevAttrMultiProcessorCount, dev)))
            return cuda_fail(e, "cudaDeviceGetAttribute");
        cudaDeviceProp prop;
        if ((e = cudaGetDeviceProperties(&prop, dev)))
            return cuda_fail(e, "cudaGetDeviceProperties");
        std::snprintf(st.name, sizeof(st.name), "%s", prop.name);
        if ((e = cudaStreamCreateWithFlags(&st.setup, cudaStreamNonBlocking)))
            return cuda_fail(e, "cudaStreamCreateWithFlags");
        if ((e = cudaMalloc(&st.te0, 256 * sizeof(uint32_t))))
            return cuda_fail(e, "cudaMalloc(te0)");
        if ((e = launch_te0_init(st.te0, st.setup)))
            return cuda_fail(e, "te0_init");
        if ((e = ctr_set_attributes()))
            return cuda_fail(e, "ctr_set_attributes");
        if ((e = batch_set_attributes()))
            return cuda_fail(e, "batch_set_attributes");
        if ((e = cudaStreamSynchronize(st.setup)))
            return cuda_fail(e, "te0_init sync");
        tune_defaults(st);
        st.ready.store(true, std::memory_order_release);
    }
    *out = &st;
    return AES_OK;
}

// The current device's state if an earlier call already set it up; never
// initialises (and so never allocates).
int device_state_ready(DeviceState **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices || !g_devices[dev].ready.load(std::memory_order_acquire))
        return AES_EINVAL;
    *out = &g_devices[dev];
    return AES_OK;
}

// A payload pointer must be device-addressable on `dev`: device or managed
// memory of that device, or pinned host memory (its device alias is used).
int resolve_ptr(const void *p, int dev, const void **dptr, bool *is_host)
{
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return AES_EPTR;
    }
    switch (a.type) {
    case cudaMemoryTypeDevice:
    case cudaMemoryTypeManaged:
        if (a.device != dev)
            return AES_EPTR;
        *dptr = a.devicePointer ? a.devicePointer : p;
        return AES_OK;
    case cudaMemoryTypeHost:
        if (!a.devicePointer)
            return AES_EPTR;
        *dptr = a.devicePointer;
        if (is_host)
            *is_host = true;
        return AES_OK;
    default:
        return AES_EPTR;
    }
}

int check_payload(const void *in, const void *out, size_t len, int dev, const void **din, void **dout,
                  bool *out_is_host)
{
    if (!in || !out)
        return AES_EINVAL;
    if (((uintptr_t)in | (uintptr_t)out) & 15u)
        return AES_EALIGN;
    if (in != out) {
        const uintptr_t a = (uintptr_t)in, b = (uintptr_t)out;
        if (a < b + len && b < a + len)
            return AES_EOVERLAP;
    }
    const void *di = nullptr, *dout_c = nullptr;
    bool in_host = false, o_host = false;
    int rc = resolve_ptr(in, dev, &di, &in_host);
    if (rc)
        return rc;
    if (out == in) {
        dout_c = di;
        o_host = in_host;
    } else if ((rc = resolve_ptr(out, dev, &dout_c, &o_host))) {
        return rc;
    }
    if (out_is_host)
        *out_is_host = o_host;
    *din = di;
    *dout = const_cast<void *>(dout_c);
    return AES_OK;
}

void iv_halves(const uint8_t *iv, uint64_t *hi, uint64_t *lo)
{
    uint64_t h = 0, l = 0;
    for (int i = 0; i < 8; ++i) {
        h = (h << 8) | iv[i];
        l = (l << 8) | iv[8 + i];
    }
    *hi = h;
    *lo = l;
}

}  // namespace aesrt

using namespace aesrt;

extern "C" {

const char *aes_strerror(int s)
{
    switch (s) {
    case AES_OK: return "AES_OK";
    case AES_PENDING: return "AES_PENDING";
    case AES_EINVAL: return "AES_EINVAL: invalid argument";
    case AES_EKEYBITS: return "AES_EKEYBITS: key size must be 128, 192 or 256 bits";
    case AES_EALIGN: return "AES_EALIGN: payload pointers must be 16-byte aligned";
    case AES_EOVERLAP: return "AES_EOVERLAP: in and out overlap without being equal";
    case AES_EAGAIN: return "AES_EAGAIN: no slot or budget free, retry later";
    case AES_ETIMEOUT: return "AES_ETIMEOUT: bounded wait expired";
    case AES_ECUDA: return "AES_ECUDA: CUDA runtime error (see aes_last_error)";
    case AES_ESTOPPED: return "AES_ESTOPPED: server stopped";
    case AES_ENOMEM: return "AES_ENOMEM: allocation failed";
    case AES_ETOOBIG: return "AES_ETOOBIG: size above the documented maximum";
    case AES_EPTR: return "AES_EPTR: pointer not addressable by this GPU";
    case AES_EDESC: return "AES_EDESC: request rejected by the device";
    default: return "unknown status";
    }
}

const char *aes_last_error(void) { return g_last_error; }

int aes_version(void) { return 0x000100; }

int aes_ctx_create(aes_ctx_t *out, const uint8_t *key, int bits)
{
    if (!out)
        return AES_EINVAL;
    *out = nullptr;
    if (!key)
        return AES_EINVAL;
    if (bits != 128 && bits != 192 && bits != 256)
        return AES_EKEYBITS;
    DeviceState *st = nullptr;
    int rc = device_state(&st);
    if (rc)
        return rc;
    aes_ctx_s *ctx = new (std::nothrow) aes_ctx_s();
    if (!ctx)
        return AES_ENOMEM;
    ctx->device = st->device;
    ctx->bits = bits;
    ctx->nr = bits / 32 + 6;
    // one allocation: the 60-word schedule, then (at byte 256) the staging
    // area for the expansion kernel's input, 32 key bytes + 4-byte key size.
    // No temporary buffer is freed here: cudaFree waits for the device to go
    // idle, which a resident served kernel may postpone.
    static_assert(kMaxRoundKeyWords * sizeof(uint32_t) <= 256, "schedule fits below the stage");
    cudaError_t e = cudaMalloc(&ctx->d_rk, 256 + 64);
    if (e) {
        delete ctx;
        return e == cudaErrorMemoryAllocation ? AES_ENOMEM : cuda_fail(e, "cudaMalloc(rk)");
    }
    uint8_t *stage = reinterpret_cast<uint8_t *>(ctx->d_rk) + 256;
    uint8_t hstage[64] = {0};
    std::memcpy(hstage, key, bits / 8);
    const int32_t b32 = bits;
    std::memcpy(hstage + 32, &b32, 4);
    if (!e) e = cudaMemcpyAsync(stage, hstage, 64, cudaMemcpyHostToDevice, st->setup);
    if (!e) e = launch_key_expand(stage, reinterpret_cast<const int32_t *>(stage + 32), st->te0,
                                  ctx->d_rk, 1, st->setup);
    if (!e) e = cudaMemcpyAsync(ctx->h_rk, ctx->d_rk, sizeof(ctx->h_rk), cudaMemcpyDeviceToHost,
                                st->setup);
    if (!e) e = cudaStreamSynchronize(st->setup);
    if (e) {
        cudaFree(ctx->d_rk);
        delete ctx;
        return cuda_fail(e, "key expansion");
    }
    *out = ctx;
    return AES_OK;
}

int aes_ctx_destroy(aes_ctx_t ctx)
{
    if (!ctx)
        return AES_OK;
    cudaFree(ctx->d_rk);
    delete ctx;
    return AES_OK;
}

int aes_ctx_bits(aes_ctx_t ctx) { return ctx ? ctx->bits : AES_EINVAL; }

int aes_ctx_round_keys(aes_ctx_t ctx, uint8_t *w, size_t cap)
{
    if (!ctx || !w)
        return AES_EINVAL;
    const size_t n = 16u * (size_t)(ctx->nr + 1);
    if (cap < n)
        return AES_ETOOBIG;
    DeviceState *st = nullptr;
    int rc = device_state(&st);
    if (rc)
        return rc;
    uint32_t tmp[kMaxRoundKeyWords];
    cudaError_t e = cudaMemcpyAsync(tmp, ctx->d_rk, n, cudaMemcpyDeviceToHost, st->setup);
    if (!e) e = cudaStreamSynchronize(st->setup);
    if (e)
        return cuda_fail(e, "aes_ctx_round_keys");
    std::memcpy(w, tmp, n);
    return (int)n;
}

int aes_ctr_ex(aes_ctx_t ctx, const uint8_t *iv, const void *in, void *out, size_t len,
               void *stream, const aes_launch_t *cfg)
{
    if (!ctx || !iv)
        return AES_EINVAL;
    if (len == 0)
        return AES_OK;
    DeviceState *st = nullptr;
    int rc = device_state(&st);
    if (rc)
        return rc;
    if (st->device != ctx->device)
        return AES_EINVAL;
    const void *din = nullptr;
    void *dout = nullptr;
    if ((rc = check_payload(in, out, len, ctx->device, &din, &dout)))
        return rc;
    CtrShape shape;
    if (cfg && cfg->variant != AES_VARIANT_AUTO) {
        shape.variant = cfg->variant;
        shape.threads = cfg->threads;
        shape.nb = cfg->blocks_per_thread;
        shape.ctas = cfg->ctas;
        if (rc = validate_ctr_shape(shape))
            return rc;
    } else {
        shape = tuned_ctr_shape(*st, len, ctx->nr);
        if (cfg && cfg->ctas > 0)
            shape.ctas = cfg->ctas;
    }
    CtrParams p;
    p.in = static_cast<const uint4 *>(din);
    p.out = static_cast<uint4 *>(dout);
    p.len = len;
    iv_halves(iv, &p.iv_hi, &p.iv_lo);
    p.te0 = st->te0;
    std::memcpy(p.rk, ctx->h_rk, sizeof(p.rk));
    cudaError_t e = launch_ctr(p, ctx->nr, shape, st->nsm, static_cast<cudaStream_t>(stream));
    if (e)
        return cuda_fail(e, "launch_ctr");
    return AES_OK;
}

int aes_ctr(aes_ctx_t ctx, const uint8_t *iv, const void *in, void *out, size_t len, void *stream)
{
    return aes_ctr_ex(ctx, iv, in, out, len, stream, nullptr);
}

int aes_ctr_sync(aes_ctx_t ctx, const uint8_t *iv, const void *in, void *out, size_t len, void *stream)
{
    int rc = aes_ctr_ex(ctx, iv, in, out, len, stream, nullptr);
    if (rc)
        return rc;
    // one completion event per host thread and device, reused across calls
    struct ThreadEvent {
        int device = -1;
        cudaEvent_t ev = nullptr;
        ~ThreadEvent()
        {
            if (ev)
                cudaEventDestroy(ev);
        }
    };
    thread_local ThreadEvent te;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e && (te.device != dev || !te.ev)) {
        if (te.ev)
            cudaEventDestroy(te.ev);
        te.ev = nullptr;
        e = cudaEventCreateWithFlags(&te.ev, cudaEventDisableTiming);
        te.device = e ? -1 : dev;
    }
    if (!e)
        e = cudaEventRecord(te.ev, static_cast<cudaStream_t>(stream));
    while (!e) {
        e = cudaEventQuery(te.ev);
        if (e == cudaErrorNotReady)
            e = cudaSuccess;
        else
            break;
    }
    if (e)
        return cuda_fail(e, "aes_ctr_sync");
    return AES_OK;
}

}  // extern "C"
