// internal.h -- host-side interfaces between the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

namespace aesrt {

constexpr int kMaxRoundKeyWords = 60;  // 4 * (14 + 1)

// Parameters of one single-key CTR launch.  Passed by value (kernel
// parameter space), so the round keys are constant-bank operands.
struct CtrParams {
    const uint4 *in;
    uint4 *out;
    uint64_t len;           // payload bytes
    uint64_t iv_hi, iv_lo;  // initial counter block as big-endian halves
    const uint32_t *te0;    // 256-word T-table seed (device)
    uint32_t parts;         // T-table: work units per 256-block counter group (1, 2, 4, 8)
    uint32_t rk[kMaxRoundKeyWords];  // round keys, little-endian column words
};

struct CtrShape {
    int variant;  // 1 = T-table, 2 = bitsliced
    int threads;
    int nb;       // T-table blocks per thread per pass (1, 2, 4)
    int ctas;     // 0 = derive
};

// Device tables and key expansion (tables.cu).
cudaError_t launch_te0_init(uint32_t *te0, cudaStream_t stream);
cudaError_t launch_key_expand(const uint8_t *keys, const int32_t *bits, const uint32_t *te0,
                              uint32_t *w, int n, cudaStream_t stream);

// Single-buffer CTR (ctr.cu).
cudaError_t ctr_set_attributes();  // once per device
int ctr_max_ctas(const CtrShape &s, int nsm);
// Grid size and counter-group split of one launch of `nblocks` blocks whose
// initial counter has low byte v0.
void ctr_plan(uint64_t nblocks, uint32_t v0, const CtrShape &s, int nsm, int *ctas, uint32_t *parts);
cudaError_t launch_ctr(const CtrParams &p, int nr, const CtrShape &s, int nsm, cudaStream_t stream);

// Batched varlen CTR (batch.cu).
struct BatchReq {        // one request, device-side descriptor (64 bytes)
    const uint4 *in;
    uint4 *out;
    uint64_t len;
    uint64_t iv_hi, iv_lo;
    const uint4 *rk;     // device round keys (4*(Nr+1) words as uint4 per round)
    uint32_t nr;
    uint32_t pad;
    uint64_t tile_begin; // prefix sum of tiles before this request
};
static_assert(sizeof(BatchReq) == 64, "descriptor is one 64-byte line");

struct BatchShape {
    int variant;      // AES_VARIANT_TTABLE or AES_VARIANT_BITSLICE
    int threads;
    int tile_blocks;  // a multiple of 256: tiles are runs of whole counter groups
    int ctas;
    int nb;           // T-table: blocks each lane keeps in flight (1, 2 or 4)
};

// Tiles of one batch request of `len` bytes whose initial counter has low
// byte `iv_low_byte`: runs of tile_blocks / 256 whole 256-block counter
// groups (group g holds the blocks whose counter low byte wrapped g times).
inline uint64_t tiles_of(uint64_t len, uint32_t iv_low_byte, int tile_blocks)
{
    const uint64_t nb = (len + 15) / 16;
    if (!nb)
        return 0;
    const uint64_t groups = ((iv_low_byte + nb - 1) >> 8) + 1;
    const uint64_t per = (uint64_t)tile_blocks / 256u;
    return (groups + per - 1) / per;
}

cudaError_t batch_set_attributes();
// The persistent T-table batch kernel over requests reqs[0..n) whose tiles
// start at reqs[i].tile_begin; the owner of a claimed tile is found by a
// binary search over those starts in shared memory (no tile map, so the
// caller needs no scratch beyond reqs and the claim counter).  n <= 1024.
cudaError_t launch_batch_search(const BatchReq *reqs, int n, uint64_t total_tiles, unsigned long long *counter,
                                const uint32_t *te0, const BatchShape &s, int nsm, cudaStream_t stream);
constexpr int kSearchMaxReqs = 1024;

}  // namespace aesrt
