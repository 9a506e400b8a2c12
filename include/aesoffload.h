/*
 * aesoffload.h -- C ABI of the GB300 AES-CTR offload library (libaesoffload.so).
 *
 * The offload is the one the paper routes through each server's own
 * concurrency (Sec. 3: submit the work to an executor, suspend the request,
 * resume it on completion; Sec. 6 setup: "GPU AES" on its own CUDA stream,
 * completion detected by polling).  The paper fixes neither mode nor key
 * size; this library computes AES-128/192/256 (FIPS-197) in counter mode
 * (NIST SP 800-38A Sec. 6.5) with the caller supplying the whole 16-byte
 * initial counter block T_1, incremented as one 128-bit big-endian integer
 * (SP 800-38A App. B.1, m = 128; wraps modulo 2^128).  Encryption and
 * decryption are the same operation.
 *
 * Conventions shared by every call:
 *   - Status codes: AES_OK (0), AES_PENDING (1, served mode only) or a
 *     negative AES_E* code.  No call aborts or throws; CUDA errors become
 *     AES_ECUDA and the CUDA error string is kept for aes_last_error().
 *   - Payload pointers (in/out) are device pointers (cudaMalloc, or the
 *     device alias of pinned host memory allocated with cudaHostAlloc /
 *     registered with cudaHostRegister).  Both must be 16-byte aligned
 *     (AES_EALIGN otherwise).  in == out (in place) is allowed; any other
 *     overlap returns AES_EOVERLAP.  Bytes of out past len are never written.
 *     The caller owns payload buffers and keeps them alive until the work is
 *     complete (stream order, or AES_OK from offload_poll).
 *   - Streams are passed as void* holding a cudaStream_t (NULL = the legacy
 *     default stream).  Work is asynchronous on that stream.
 *   - Key material and descriptor arrays are host memory, copied during the
 *     call; the caller may reuse them as soon as the call returns.
 *   - Every call acts on the CUDA device that is current on the calling
 *     thread; an aes_ctx_t / plan / server stays bound to the device it was
 *     created on.
 */
#ifndef AESOFFLOAD_H
#define AESOFFLOAD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define AES_OK 0
#define AES_PENDING 1       /* served request not finished yet */
#define AES_EINVAL (-1)     /* null / malformed argument */
#define AES_EKEYBITS (-2)   /* key size not 128, 192 or 256 bits */
#define AES_EALIGN (-3)     /* in/out not 16-byte aligned */
#define AES_EOVERLAP (-4)   /* in and out overlap without being equal */
#define AES_EAGAIN (-5)     /* served mode: no slot or HBM budget free now */
#define AES_ETIMEOUT (-6)   /* a bounded wait ran out */
#define AES_ECUDA (-7)      /* a CUDA runtime call failed */
#define AES_ESTOPPED (-8)   /* served mode: the server is stopping/stopped */
#define AES_ENOMEM (-9)     /* allocation failed */
#define AES_ETOOBIG (-10)   /* a size exceeds a documented maximum */
#define AES_EPTR (-11)      /* a payload pointer is not device-accessible */
#define AES_EDESC (-12)     /* served mode: the device rejected the request */

/* Human-readable name of a status code (static string, never NULL). */
const char *aes_strerror(int status);

/* The last CUDA error text seen by this thread (static/thread-local storage,
 * never NULL; "" when none). */
const char *aes_last_error(void);

/* Library version as 0xMMmmpp. */
int aes_version(void);

/* ------------------------------------------------------------ key contexts */

/* Opaque key context: owns the device-resident key schedule of one key. */
typedef struct aes_ctx_s *aes_ctx_t;

/* Create a context for `key` (host pointer, bits/8 bytes), bits in
 * {128, 192, 256}.  KeyExpansion (FIPS-197 Sec. 5.2) runs in a CUDA kernel
 * on the current device and the 4*(Nr+1)-word schedule stays in device
 * memory.  Synchronous (allocates and waits for the expansion).  Not for use
 * inside stream capture.  Errors: AES_EINVAL (null out/key), AES_EKEYBITS,
 * AES_ENOMEM, AES_ECUDA.  On error *out is set to NULL. */
int aes_ctx_create(aes_ctx_t *out, const uint8_t *key, int bits);

/* Release a context (NULL is a no-op).  The caller must ensure no work that
 * uses it is still queued or running.  Returns AES_OK.  Frees device memory
 * with cudaFree, which waits for the device's work in flight, a resident
 * served kernel included (until its idle exit); create contexts up front
 * and destroy them at shutdown when a server is running.  (aes_ctx_create
 * frees nothing.) */
int aes_ctx_destroy(aes_ctx_t ctx);

/* Key size in bits, or AES_EINVAL for a NULL ctx. */
int aes_ctx_bits(aes_ctx_t ctx);

/* Copy the device-expanded key schedule to host memory `w` (capacity `cap`
 * bytes): 16*(Nr+1) bytes, word i of FIPS-197 Sec. 5.2 at w[4i..4i+3].
 * Returns the number of bytes written, or AES_EINVAL / AES_ETOOBIG (cap too
 * small) / AES_ECUDA.  Synchronous. */
int aes_ctx_round_keys(aes_ctx_t ctx, uint8_t *w, size_t cap);

/* ------------------------------------------------------- single-buffer CTR */

/* Kernel variants for the block cipher (SubBytes/ShiftRows/MixColumns). */
#define AES_VARIANT_AUTO 0      /* the tuned choice for (size, Nr) */
#define AES_VARIANT_TTABLE 1    /* 32-way bank-replicated T-tables in shared memory */
#define AES_VARIANT_BITSLICE 2  /* 32 blocks per thread, boolean circuit (LOP3) */

/* Launch shape override (all-zero fields mean "use the tuned value"). */
typedef struct {
    int variant;        /* AES_VARIANT_* */
    int threads;        /* CTA size: multiple of 32, 32..1024 */
    int blocks_per_thread; /* T-table: 16-byte blocks each thread keeps in flight (1, 2 or 4) */
    int ctas;           /* grid size; 0 = enough for the data, capped at SMs x occupancy */
} aes_launch_t;

/* out[0..len) = in[0..len) xor AES-CTR keystream from T_1 = iv (host
 * pointer, 16 bytes), SP 800-38A Sec. 6.5: block j (0-based) is xored with
 * CIPH_K(T_1 + j mod 2^128); a final partial block uses the leading bytes of
 * its keystream block.  One kernel launch on `stream` (none when len == 0).
 * Errors: AES_EINVAL (null ctx/iv, null in/out with len > 0), AES_EALIGN,
 * AES_EOVERLAP, AES_EPTR (a pointer the GPU cannot address), AES_ECUDA. */
int aes_ctr(aes_ctx_t ctx, const uint8_t *iv, const void *in, void *out, size_t len,
            void *stream);

/* The blocking offload call a server makes on its own thread (the call
 * Sec. 3's reroute moves off the event loop): aes_ctr on `stream`, then poll
 * an event recorded behind it with cudaEventQuery until the work is done,
 * the completion mechanism of the paper's GPU offload (Sec. 6 setup).  Same
 * arguments and errors as aes_ctr, plus AES_ECUDA if the wait fails.  Uses
 * one event per calling thread, created on first use. */
int aes_ctr_sync(aes_ctx_t ctx, const uint8_t *iv, const void *in, void *out, size_t len, void *stream);

/* aes_ctr with an explicit launch shape (autotuner, tests, sweeps); `cfg`
 * NULL behaves like aes_ctr.  Extra error: AES_EINVAL for a shape outside the
 * documented ranges. */
int aes_ctr_ex(aes_ctx_t ctx, const uint8_t *iv, const void *in, void *out, size_t len,
               void *stream, const aes_launch_t *cfg);

/* ----------------------------------------------------------- batched varlen */

/* One request of a batch: its own key context, initial counter and length. */
typedef struct {
    aes_ctx_t ctx;
    uint8_t iv[16];
    const void *in;
    void *out;
    size_t len;
} aes_desc_t;

/* Options of the persistent batch kernel (all-zero = tuned defaults). */
typedef struct {
    int variant;        /* AES_VARIANT_* (AUTO: the tuned variant, T-table
                           until aes_batch_autotune picks otherwise) */
    int threads;        /* CTA size, multiple of 32, 32..1024 (default 512): up
                           to 512 the warps keep round keys in registers,
                           above it in shared memory; the bitsliced kernel
                           takes 128 only */
    int tile_blocks;    /* 16-byte blocks per work tile: a multiple of 256 (whole counter groups) */
    int ctas;           /* persistent CTAs; 0 = one per SM (x occupancy) */
    uint32_t tile_order_seed; /* nonzero: tiles are claimed in a seeded
                                 pseudo-random permutation (testing aid; the
                                 result must not change) */
    int blocks_per_thread; /* T-table: 16-byte blocks each lane keeps in flight
                              (1, 2 or 4); ignored by the bitsliced kernel,
                              which always holds 32 per lane */
} aes_batch_opts_t;

/* Encrypt n independent requests in ONE persistent-kernel launch on
 * `stream`: the requests are cut into tiles of 16-byte blocks and the CTAs
 * claim tiles through a device atomic (work stealing).  Any mix of key sizes
 * and lengths; each request follows aes_ctr's contract.  The descriptor
 * table is uploaded from host memory inside the call (descs may be reused on
 * return).  n == 0 is a no-op.  Errors: AES_EINVAL (n < 0, null descs, a
 * NULL ctx), AES_EALIGN / AES_EOVERLAP / AES_EPTR for the first bad request,
 * AES_ETOOBIG (n > AES_BATCH_MAX), AES_ENOMEM, AES_ECUDA. */
#define AES_BATCH_MAX (1 << 20)
int aes_ctr_batch(const aes_desc_t *descs, int n, void *stream);
int aes_ctr_batch_ex(const aes_desc_t *descs, int n, void *stream, const aes_batch_opts_t *opts);

/* aes_ctr_batch for callers that cannot allocate device memory -- e.g. a
 * process whose HBM is entirely reserved by another framework's pool, a
 * latency-critical path that must not pay for cudaMalloc/cudaFree (which can
 * synchronise the device), or a runtime that forbids allocation after
 * start-up.  The paper has no counterpart: this is a deployment variant of
 * the batched launch.  Same contract and result as aes_ctr_batch, but the
 * call allocates nothing: its scratch (descriptor table + claim counter)
 * lives in one static device array of AES_NOALLOC_MAX_REQUESTS descriptors
 * (about 64 KiB) that every GPU loading the library keeps until exit.  The
 * key contexts must already exist on the current device (AES_EINVAL if no
 * context was ever created on it).  The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress) and keeps it.  Every
 * call copies its descriptors into the array with cudaMemcpyAsync from
 * pageable host memory, so no call -- the first or a later one -- may be
 * made while `stream` is being captured into a CUDA graph (the capture
 * would refuse the copy); callers that need a graph use the batch plans
 * (aes_batch_plan_create), which allocate once, up front.  Every call reuses
 * the same array and leaves its contents behind: calls whose work may
 * overlap on the GPU (other streams, other threads) race on it and must be
 * serialised by the caller.  The kernel is the T-table batch kernel in the
 * device's tuned T-table shape (tiles of whole counter groups, claimed by
 * each warp), finding each tile's request by a binary search in shared
 * memory instead of a tile map.  Errors: those of aes_ctr_batch, and
 * AES_ETOOBIG when n exceeds AES_NOALLOC_MAX_REQUESTS. */
#define AES_NOALLOC_MAX_REQUESTS 1024
int aes_ctr_batch_noalloc(const aes_desc_t *descs, int n, void *stream);

/* A prepared batch: the descriptor table lives on the device and the launch
 * (counter reset + persistent kernel) is captured once into a CUDA graph, so
 * repeated encryption of the same request layout costs one graph launch.
 * Payload contents may change between launches; pointers, lengths, keys and
 * IVs are fixed at creation. */
typedef struct aes_batch_plan_s *aes_batch_plan_t;
int aes_batch_plan_create(aes_batch_plan_t *out, const aes_desc_t *descs, int n,
                          const aes_batch_opts_t *opts);
int aes_batch_plan_launch(aes_batch_plan_t plan, void *stream);
/* Payload bytes covered by one launch of the plan. */
int64_t aes_batch_plan_bytes(aes_batch_plan_t plan);
int aes_batch_plan_destroy(aes_batch_plan_t plan);

/* --------------------------------------------------------------- autotuner */

/* Time the candidate launch shapes of aes_ctr (per size bucket and key
 * size) and of the batch kernel on the current device, on scratch buffers
 * the call allocates and frees, and keep the fastest for AES_VARIANT_AUTO.
 * Synchronous; takes roughly a second.  `path` (may be NULL) names a JSON
 * file the table is written to. */
int aes_autotune(const char *path);

/* Load a table written by aes_autotune (ignored if it was measured on a
 * device with another name or SM count).  AES_EINVAL if unreadable. */
int aes_autotune_load(const char *path);

/* Tune the batch kernel on the caller's own requests (the batching pattern's
 * autotuner): every candidate shape -- variant (T-table or bitsliced), CTA
 * size, blocks per lane in flight and tile size -- is built as a plan over
 * descs[0..n) and timed with CUDA events on `stream` (median of 5 launches
 * after 2 warm-ups); the fastest becomes the device's shape for
 * AES_VARIANT_AUTO batches and plans, and is returned in *best (may be
 * NULL).  Every candidate encrypts the requests several times, so their
 * outputs are overwritten (with the correct ciphertext: each launch computes
 * out = in xor keystream).  Requests must not be in place (in == out) if the
 * input has to survive.  Synchronous; allocates; not for use inside stream
 * capture.  Errors: those of aes_batch_plan_create, AES_ECUDA. */
int aes_batch_autotune(const aes_desc_t *descs, int n, void *stream, aes_batch_opts_t *best);

/* The batch shape AES_VARIANT_AUTO uses on the current device (the default,
 * or the last aes_batch_autotune / aes_autotune / aes_autotune_load). */
int aes_batch_tuned_shape(aes_batch_opts_t *out);

/* The candidates of the last batch-shape sweep on the current device
 * (aes_batch_autotune or aes_autotune) with their median launch times in ms
 * (negative: the candidate did not run): up to `cap` entries into shapes[]
 * and ms[].  Returns the number written (0 before any sweep), or
 * AES_EINVAL. */
int aes_batch_tune_results(aes_batch_opts_t *shapes, float *ms, int cap);

/* Describe the shape AES_VARIANT_AUTO picks for (len, bits). */
int aes_tuned_shape(size_t len, int bits, aes_launch_t *out);

/* ------------------------------------------------------------ measurement */

/* Device rates behind the benchmark's roofline (this call computes no AES;
 * the paper has no counterpart: it reports no device-side rates).  Per-SM
 * rates come from clock64() on each SM (median over SMs of operations per
 * SM clock, 2 CTAs of 1024 threads per SM, 8 independent chains a thread);
 * link bandwidths from CUDA events over 256 MiB transfers (median of 3).
 *   lds32_per_clk_sm        conflict-free 32-bit shared-memory loads (lane l
 *                           reads bank l; the T-table lookup pattern)
 *   lop3_per_clk_sm         three-input logic ops (lop3.b32)
 *   prmt_per_clk_sm         byte permutes (prmt.b32)
 *   iadd_per_clk_sm         32-bit adds
 *   sm_mhz_during_probe     SM cycles / event time of the load probe
 *   h2d_gbs, d2h_gbs        copy engine, pinned host memory, one direction
 *   h2d_d2h_each_way_gbs    both directions at once, per direction
 *   zero_copy_each_way_gbs  a kernel reading pinned host memory and writing
 *                           pinned host memory at once (NVLink-C2C), per
 *                           direction: the end-to-end path's link bound
 * Synchronous; allocates and frees its buffers (512 MiB pinned host memory,
 * 512 MiB device memory).  Errors: AES_EINVAL (NULL out), AES_ENOMEM,
 * AES_ECUDA. */
typedef struct {
    int sms;
    double lds32_per_clk_sm;
    double lop3_per_clk_sm;
    double prmt_per_clk_sm;
    double iadd_per_clk_sm;
    double sm_mhz_during_probe;
    double h2d_gbs;
    double d2h_gbs;
    double h2d_d2h_each_way_gbs;
    double zero_copy_each_way_gbs;
} aes_peaks_t;
int aes_measure_peaks(aes_peaks_t *out);

/* ---------------------------------------------------------------- served mode */

/* A resident persistent kernel polls a descriptor queue in pinned, mapped
 * host memory, so a request costs no kernel launch: offload_submit writes a
 * descriptor and returns a ticket at once (submit + suspend), the kernel
 * encrypts the request's tiles alongside every other request in flight
 * (continuous batching), and the CTA finishing the last tile raises the
 * request's completion flag, which offload_poll reads (resume). */
typedef struct offload_server_s *offload_server_t;

typedef struct {
    int slots;              /* requests in flight at most (<= 65536); 0 = 1024 */
    int max_keys;           /* resident key schedules; 0 = 64 */
    uint64_t hbm_budget;    /* bytes of payload in flight at most (in + out,
                               in-place counted once); 0 = unlimited */
    int ctas;               /* resident CTAs; 0 = SM count - 4 */
    int threads;            /* CTA size, multiple of 32, 64..512; 0 = 512 (warp 0 dispatches) */
    int tile_blocks;        /* 16-byte blocks per tile: 64, 128 or a multiple of 256;
                               0 = per request (~512 tiles of 64..1024 blocks:
                               the latency setting).  Fewer, larger tiles serve
                               more requests per second (measured on GB300,
                               served mix: 269 k req/s by default, 370 k with
                               1024), at the cost of one-in-flight latency. */
    uint32_t idle_timeout_us; /* resident kernel exits after this long with no
                                 work (relaunched on the next submit); 0 = 200000 */
    int claim_mode;         /* how agents claim tiles: 0 = one global cursor
                               moved from request to request (default);
                               1 = per-request claim words that agents walk in
                               sequence order, several requests cut at once
                               (same results; measured slower on GB300) */
    int trace_requests;     /* trace builds (libaesoffload_trace.so): keep timer
                               stamps of the protocol's steps for the last
                               trace_requests requests (a power of two up to
                               2^20; 0 = off); read with offload_server_trace.
                               Other builds refuse a nonzero value (AES_EINVAL). */
} offload_cfg_t;

typedef struct {
    uint64_t submitted, completed, rejected_eagain, device_errors, relaunches;
    uint64_t bytes_completed;
    uint32_t kernel_status;    /* exit reasons (1 stop, 2 idle, 4 error) raised by
                                  the CTAs of the current launch, or of the
                                  last one once it has ended; 0 while every
                                  CTA of a running launch is resident */
    int running;               /* resident kernel currently launched */
} offload_stats_t;

/* Start a server on the current device: allocates the key store, the mapped
 * descriptor queue and device state, and launches the resident kernel on a
 * stream of its own.  Errors: AES_EINVAL, AES_ENOMEM, AES_ECUDA. */
int offload_server_create(offload_server_t *out, const offload_cfg_t *cfg);

/* Expand `key` (host pointer, bits/8 bytes; bits in {128, 192, 256}) into
 * resident key slot *slot_out (device kernel, FIPS-197 Sec. 5.2).
 * Thread-safe.  AES_ETOOBIG when all max_keys slots are used.
 * May be called while the resident kernel runs: the expansion kernel runs on
 * the SMs the resident kernel leaves free (ctas < SM count, the default), and
 * the resident kernel reads round keys through L2, so a request submitted
 * after this returns sees the new schedule.  With ctas = SM count the call
 * returns after the resident kernel's next idle exit. */
int offload_key_register(offload_server_t srv, const uint8_t *key, int bits, int *slot_out);

/* Submit one request; never blocks on the GPU.  On AES_OK *ticket identifies
 * it for offload_poll.  Thread-safe (any number of submitter threads).
 * Ordering: the resident kernel runs on the server's own stream and may read
 * `in` and write `out` as soon as the call returns, so any GPU work that
 * produces `in` or still touches `out` (a fill, a copy, a kernel on another
 * stream) must be complete before the call -- e.g. synchronise that stream
 * first.  `out` must not be touched again until offload_poll returns AES_OK.
 * Errors: AES_EAGAIN (no slot or budget free: back-pressure), AES_EINVAL
 * (bad key slot, null iv/in/out with len > 0), AES_EALIGN, AES_EOVERLAP,
 * AES_ETOOBIG (len > 16 GiB), AES_ESTOPPED, AES_ECUDA. */
int offload_submit(offload_server_t srv, int key_slot, const uint8_t *iv, const void *in,
                   void *out, size_t len, uint64_t *ticket);

/* Emulated offload for controlled-load studies (the paper sweeps offered
 * load over a fixed 20 us emulated offload, Sec. 6 "Latency under offered
 * load"): the request takes the whole served path -- queue entry, dispatch,
 * claim, completion flag -- but its single tile holds one worker warp for
 * duration_ns instead of encrypting; it moves no data and needs no key.
 * Poll it like any ticket.  Errors: AES_EINVAL (duration_ns > 10 ms, null
 * ticket), AES_EAGAIN (no slot free), AES_ESTOPPED, AES_ECUDA. */
int offload_submit_emulated(offload_server_t srv, uint64_t duration_ns, uint64_t *ticket);

/* AES_OK once the request is complete and its output visible to the host
 * and to later GPU work (the ticket is then released; polling it again gives
 * AES_EINVAL), AES_PENDING while in flight, AES_EDESC if the device rejected
 * the descriptor, AES_EINVAL for an unknown ticket.  Thread-safe. */
int offload_poll(offload_server_t srv, uint64_t ticket);

/* Completion wait over many tickets, for a server's completion thread
 * (the resume step of Sec. 3 for a batch of suspended requests): poll every
 * ticket until at least one is no longer pending or `timeout_us` passes.
 * status[i] receives offload_poll's result for tickets[i] (AES_PENDING for
 * those still in flight; a finished ticket is released exactly as by
 * offload_poll).  Returns the number of tickets no longer pending, 0 on
 * timeout, AES_EINVAL for bad arguments.  n == 0 returns 0 at once. */
int offload_poll_many(offload_server_t srv, const uint64_t *tickets, int n, int *status, uint64_t timeout_us);

/* Poll until done or `timeout_us` passes (AES_ETIMEOUT, ticket stays live). */
int offload_wait(offload_server_t srv, uint64_t ticket, uint64_t timeout_us);

int offload_server_stats(offload_server_t srv, offload_stats_t *out);

/* Trace builds: copy the stamp buffer (trace_requests rows of
 * AES_TRACE_POINTS %globaltimer values in ns; row s & (trace_requests - 1)
 * belongs to request sequence number s, counted from 1 in submit order; 0 =
 * not reached) into `out`, at most `max_words` values.  The points, in order:
 * dispatched (its order word claimed), published (record complete, ring
 * entry about to be stored), first tile claimed, first tile taken by a
 * worker, record loaded, round keys loaded, first tile done, completion
 * raised.  Returns the number
 * of values copied; AES_EINVAL without tracing. */
#define AES_TRACE_POINTS 8
int offload_server_trace(offload_server_t srv, uint64_t *out, size_t max_words);

/* Raise the stop flag, wait (bounded, 5 s) for the resident kernel to exit,
 * and free everything.  Requests still in flight are abandoned.  Returns
 * AES_ETIMEOUT if the kernel did not exit in time (resources are then leaked
 * rather than freed under a running kernel).  The frees (cudaFree,
 * cudaFreeHost) wait for the device's work in flight, so with other servers
 * resident this returns after their next idle exit. */
int offload_server_destroy(offload_server_t srv);

/* ------------------------------------------------------------ load drivers */

/* Open-loop load drivers for the served and per-call paths.  The paper
 * measures latency under offered load with open-loop Poisson arrivals and
 * reports median and tail latency (Sec. 6, "Latency under offered load"),
 * and its servers hand each offload to a pool of executor threads (Sec. 3,
 * Listing 1).  These drivers reproduce that measurement natively:
 * `nthreads` submitter threads, thread k owning requests k, k+nthreads, ...,
 * each submitted at its scheduled arrival_s (seconds from the call) or as
 * soon after as the thread can, and latency_us[i] = time from the scheduled
 * arrival to the moment the thread observes completion (-1 on error).
 * reqs must be sorted by arrival_s.  Host-side only; synchronous.  A thread
 * that sees no completion for 30 s marks its remaining requests failed and
 * the call returns AES_ETIMEOUT (a stuck or failed device). */
typedef struct {
    int key_slot;       /* offload_drive: server key slot; aes_ctr_drive: index into ctxs */
    uint8_t iv[16];
    const void *in;
    void *out;
    size_t len;
    double arrival_s;
} aes_drive_req_t;

typedef struct {
    double elapsed_s;         /* first scheduled arrival to last completion */
    uint64_t bytes;           /* payload bytes completed */
    uint64_t eagain_retries;  /* submissions retried after AES_EAGAIN */
    int errors;               /* requests that failed */
} aes_drive_result_t;

/* Served path: offload_submit, then offload_poll until AES_OK; AES_EAGAIN
 * (back-pressure) is retried.  Errors: AES_EINVAL for bad arguments. */
int offload_drive(offload_server_t srv, const aes_drive_req_t *reqs, int n, int nthreads,
                  double *latency_us, aes_drive_result_t *res);

/* Driver options.  blocking != 0: each thread serves its requests one at a
 * time, waiting for each offload before taking the next (the blocking server
 * of Sec. 6; latency still counts from the scheduled arrival); 0: threads
 * submit at arrival and poll all their pending requests (the overlapping,
 * rerouted server).  emulated_ns > 0: every request is an emulated offload
 * of that duration (offload_submit_emulated; only arrival_s is read). */
typedef struct {
    int blocking;
    uint64_t emulated_ns;
} aes_drive_opts_t;

/* offload_drive with options (NULL = offload_drive). */
int offload_drive_ex(offload_server_t srv, const aes_drive_req_t *reqs, int n, int nthreads,
                     const aes_drive_opts_t *opts, double *latency_us, aes_drive_result_t *res);

/* Per-call path with the same schedule: each thread owns a CUDA stream,
 * launches aes_ctr, records an event and polls it with cudaEventQuery (the
 * paper's completion mechanism, Sec. 6 setup); at most 256 requests in
 * flight per thread.  Events on one stream complete in order, so a thread
 * queries only its oldest pending event on each pass. */
int aes_ctr_drive(const aes_ctx_t *ctxs, int nctx, const aes_drive_req_t *reqs, int n, int nthreads,
                  double *latency_us, aes_drive_result_t *res);

/* ------------------------------------------------ shared-state conflicts */

/* The page-protection conflict detector (Sec. 5, "A transparent conflict
 * detector") measured on a synthetic server: `handlers` cooperative handlers
 * on the calling thread serve `requests` requests; each reads one of
 * `counters` shared counters (`counters_per_page` to a page, 1..64), parks
 * at an offload, and writes the counter back incremented -- the unlocked
 * read-modify-write that rerouting exposes.  The detector write-protects the
 * counters' pages, snapshots a version clock when a handler parks, and flags
 * a write fault on a page modified during the park; CDET_ENFORCE restarts a
 * conflicting handler and re-runs it serialized.  The offload: a host timer
 * of offload_ns when srv is NULL; else the served path -- an emulated
 * offload of offload_ns when bytes == 0, or AES-CTR of `bytes` with key
 * `key_slot` from buf_in + h*stride to buf_out + h*stride for handler h
 * (stride = bytes rounded up to 256).  Installs a SIGSEGV handler for the
 * duration (the previous one is restored; faults outside the detector's
 * pages go to it); one run at a time per process.  Synchronous.  Errors:
 * AES_EINVAL, AES_ENOMEM, or the offload's error. */
#define CDET_UNPROTECTED 0 /* overlap, nothing guards the counters */
#define CDET_LOCK 1        /* one coarse lock held across the offload */
#define CDET_DETECT 2      /* overlap, conflicts counted, not prevented */
#define CDET_ENFORCE 3     /* overlap, conflicting handlers re-run serialized */

/* Shared-state patterns of the synthetic server (the paper's taxonomy,
 * Sec. 5): only the first is hazardous under overlap. */
#define CDET_PATTERN_SHARED 0     /* unlocked read-modify-write of a shared counter across the offload */
#define CDET_PATTERN_READONLY 1   /* the shared counter is only read */
#define CDET_PATTERN_PER_CONN 2   /* each handler (connection) updates a counter of its own;
                                     needs counters >= handlers */
#define CDET_PATTERN_LOCKED 3     /* the application holds a lock across its read-modify-write */

/* cdet_run_cfg_t.store_mode */
#define CDET_STORES_EMULATE 0     /* the fault handler performs guarded stores (default) */
#define CDET_STORES_UNPROTECT 1   /* guarded writes unprotect the page */

typedef struct {
    int handlers;
    int requests;
    int counters;
    int counters_per_page;
    int mode;
    uint64_t offload_ns;
    offload_server_t srv;
    int key_slot;
    const void *buf_in;
    void *buf_out;
    size_t bytes;
    int pattern;            /* CDET_PATTERN_*; 0 = the shared unlocked counter */
    int store_mode;         /* detector, how a guarded write proceeds:
                               CDET_STORES_EMULATE (0, the default): the pages
                               stay read-only and the fault handler performs
                               each faulting store itself (through a second,
                               writable mapping), so a guarded write changes no
                               protection (0.8 us a write on the Grace host);
                               stores it cannot decode (only plain
                               general-register stores are: x86-64 MOV, AArch64
                               STR/STUR/STTR) unprotect the page instead.
                               CDET_STORES_UNPROTECT: unprotect the page at the
                               write and protect it again when the writer parks
                               or finishes (two protection changes, 48 us a write
                               in a process with a CUDA context on the Grace
                               host, where the GPU shares the page tables).
                               Other values: AES_EINVAL. */
} cdet_run_cfg_t;

typedef struct {
    uint64_t final_count;   /* sum of the counters (requests if no update was lost);
                               CDET_PATTERN_READONLY: requests whose read completed */
    uint64_t lost_updates;  /* requests - final_count */
    uint64_t conflicts;     /* write faults on a page modified during the writer's park */
    uint64_t restarts;      /* handlers re-run serialized (CDET_ENFORCE) */
    double elapsed_s;
    uint64_t emulated_stores; /* guarded writes performed by the fault handler */
    uint64_t protect_calls;   /* protection changes during the run (setup and teardown excluded) */
} cdet_run_result_t;

int cdet_run(const cdet_run_cfg_t *cfg, cdet_run_result_t *res);

/* Self-test of the detector's store emulation on this CPU: `rounds` guarded
 * stores of 8, 16, 32 and 64 bits at run-time offsets of a read-only
 * region, each performed by the fault handler where it can decode the
 * instruction (else by unprotecting the page), checked against a plain
 * shadow copy.  *emulated / *fallbacks: stores performed each way.
 * AES_OK if the region matches the shadow, AES_EDESC if not; AES_EINVAL
 * (bad arguments, or a cdet_run in progress), AES_ENOMEM. */
int cdet_store_selftest(int rounds, uint64_t *emulated, uint64_t *fallbacks);

#ifdef __cplusplus
}
#endif
#endif /* AESOFFLOAD_H */
