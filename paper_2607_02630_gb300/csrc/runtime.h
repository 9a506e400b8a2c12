// runtime.h -- host-side state shared by the C ABI translation units.
#pragma once
#include "../../include/aesoffload.h"
#include "internal.h"

#include <atomic>
#include <cstdio>

struct aes_ctx_s {
    int device;
    int bits;
    int nr;
    uint32_t *d_rk;                         // device schedule (60 words)
    uint32_t h_rk[aesrt::kMaxRoundKeyWords];  // host mirror for kernel parameters
};

namespace aesrt {

constexpr int kMaxDevices = 64;
constexpr int kLenBuckets = 41;  // bucket b holds lengths in [2^b, 2^(b+1))

struct DeviceState {
    std::atomic<bool> ready{false};
    int device = -1;
    int nsm = 0;
    char name[256] = {0};
    uint32_t *te0 = nullptr;        // 256-word T-table seed
    cudaStream_t setup = nullptr;   // internal non-blocking stream
    CtrShape ctr_tuned[3][kLenBuckets];  // [nr index: 10/12/14][length bucket]
    BatchShape batch_tuned;
    // the last batch-shape sweep: every candidate and its median launch time
    // (ms; negative if it did not run)
    static constexpr int kMaxBatchCandidates = 64;
    int n_batch_results = 0;
    BatchShape batch_results[kMaxBatchCandidates];
    float batch_results_ms[kMaxBatchCandidates];
};

extern thread_local char g_last_error[256];
int cuda_fail(cudaError_t e, const char *where);
int device_state(DeviceState **out);
int device_state_ready(DeviceState **out);
// A payload pointer the GPU can address on `dev`: device or managed memory of
// that device, or pinned host memory (*is_host set); its device alias in *dptr.
int resolve_ptr(const void *p, int dev, const void **dptr, bool *is_host = nullptr);
int check_payload(const void *in, const void *out, size_t len, int dev, const void **din, void **dout,
                  bool *out_is_host = nullptr);
void iv_halves(const uint8_t *iv, uint64_t *hi, uint64_t *lo);

// tune.cu
void tune_defaults(DeviceState &st);
int validate_ctr_shape(const CtrShape &s);
// batch.cu: AES_OK for a shape the batch kernels take (AUTO becomes T-table)
int validate_batch_shape(BatchShape &s);
CtrShape tuned_ctr_shape(const DeviceState &st, size_t len, int nr);
int len_bucket(size_t len);

}  // namespace aesrt
