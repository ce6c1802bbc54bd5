/*
 * ntc.h -- C ABI of the GB300 (sm_103a) library for AO accelerated stochastic
 * nonnegative tensor completion (Siaminou, Papagiannakos, Kolomvakis, Liavas,
 * "Accelerated Stochastic Gradient for Nonnegative Tensor Completion and
 * Parallel Implementation", arXiv 2109.09534).
 *
 * Model and problem (Sec. II): an order-N tensor X is observed on the index
 * set Omega; the library fits nonnegative factors U^(i) in R_+^{I_i x R}
 * of the CPD model [[U^(1), ..., U^(N)]] (eq. 1) by minimising
 *     1/2 ||M .* (X - [[U]])||_F^2 + lambda/2 sum_i ||U^(i)||_F^2   (eq. 3)
 * with Algorithm 2 (alternating optimisation over the modes), each mode
 * solved by Algorithm 1 (the per-row stochastic accelerated gradient).
 *
 * Conventions for every call:
 *   - Return value: NTC_OK or an error status; ntc_last_error() gives a
 *     message.  A call that fails leaves the handle's data unchanged.
 *   - Ownership: the library copies every input array; the caller keeps
 *     ownership of what it passes and allocates every output buffer.  The
 *     handle owns all device memory it allocates and frees it in
 *     ntc_destroy().
 *   - Memory spaces: pointers are HOST pointers unless the name ends in _dev,
 *     in which case they are DEVICE pointers on the handle's current device.
 *   - Layouts: indices are zero based, int32, row-major [n][order]; factors
 *     are float32 row-major [dims[mode]][rank].
 *   - Threads: one handle must not be used from several threads at once.
 *     Work is enqueued on the handle's stream (ntc_set_stream); calls that
 *     return host data synchronise that stream.
 *   - Observations: Omega is a multiset: duplicate index tuples are separate
 *     observations.  Held-out test entries go only to ntc_rmse/ntc_predict.
 *   - Sizes: 2 <= order <= 8, 1 <= rank <= 64, 0 <= nnz < 2^31,
 *     1 <= dims[i] < 2^31.
 */
#ifndef NTC_H
#define NTC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ntc_handle ntc_handle;

typedef enum {
    NTC_OK = 0,
    NTC_ERR_ARG = 1,    /* invalid argument (sizes, lambda, c, mode order, key) */
    NTC_ERR_INDEX = 2,  /* an observed or queried index is out of range        */
    NTC_ERR_OOM = 3,    /* device or host allocation failed                    */
    NTC_ERR_STATE = 4,  /* call not valid in the handle's current state        */
    NTC_ERR_CUDA = 5    /* a CUDA runtime call or kernel launch failed          */
} ntc_status;

/* Create a problem (the inputs R and lambda of Alg. 2, Sec. III): order N,
 * mode sizes dims[order] (host), rank R, ridge weight lambda >= 0.  Factors
 * are allocated on the current CUDA device and zeroed; they receive their
 * initial values at ntc_set_observed unless set with ntc_set_factor.
 * Errors: NTC_ERR_ARG (order, dims, rank, lambda out of range), NTC_ERR_OOM,
 * NTC_ERR_CUDA.  *out is NULL on failure. */
ntc_status ntc_create(int order, const int64_t* dims, int rank, double lambda, ntc_handle** out);

/* Set a tuning or method parameter:
 *   "max_inner"      MAX_INNER of Alg. 1 (default 1, >= 1)
 *   "power_iters"    power-method iterations for L_p (Alg. 1 line 10; default 10)
 *   "storage_bf16"   0: factors gathered as float32; 1: gathered from a bfloat16
 *                    copy (round-to-nearest-even of the float32 master)
 *   "init_seed"      seed of the initial factors drawn at ntc_set_observed (default 3)
 *   "keep_perm"      1: keep the bucket permutation for ntc_get_bucket (default 0)
 *   "sampler"        0: independent minibatch per AO iteration (the reading of
 *                    Alg. 1 line 5, default); 1: epoch permutation -- in each
 *                    epoch of T = ceil(1/c) AO iterations a row is read in one
 *                    keyed pseudo-random permutation (8-round Feistel network,
 *                    counters {0xF2000000|mode, epoch, row, 0/1}) and minibatch
 *                    slot s takes positions pi((s k_p + j) mod n_p), j < k_p
 *   "power_warm"     1: each row's power method for L_p starts from the vector
 *                    that row's previous update of the same mode ended with
 *                    (ones/sqrt(R) the first time and after ntc_set_observed);
 *                    with "power_iters" lowered this is a cheaper L_p (Sec. II-B
 *                    leaves cheaper L_p estimation open).  Default 0
 *   "cache_staging"  1: keep ntc_set_observed's staging copy of the observations
 *                    and its sort buffers (about nnz*(4N+20) bytes) for the next
 *                    call instead of allocating and freeing them each time
 *                    (default 1)
 *   "bracket_z"      width, in standard deviations, of the sampler's key bracket
 *                    (default 6; a row's k-th key falls outside it, so that the
 *                    row takes the exact fallback selector, with probability
 *                    about 2e-9 per update; 0 forces the fallback)
 *   "heavy_rows"     rows with more than this many observations are split over
 *                    several thread blocks (default 4096, range 64..4096)
 *   "chunk"          observations per thread block of a split row (default 65536)
 *   "pipeline"       1 (default): split-row sampling runs on its own stream with
 *                    two scratch sets, so the next mode update's sampling runs
 *                    beside this one's Gram (it needs no factors); 0: in stream
 *                    order.  Set before ntc_set_observed (NTC_ERR_STATE after)
 *   "gram_tc"        1 (default): at padded rank 32 and orders 2-4 the split rows'
 *                    Gram G = sum k k^T runs on the tensor cores (TF32 operands
 *                    split into big + small parts for FP32 accuracy); 0: FP32
 *                    FMA.  Other shapes always use FP32 FMA
 *   "overlap"        2 (default): rows that fit one block run on a second stream
 *                    beside the split rows' Gram of the same mode update (after
 *                    their sampling); 1: beside the split rows' sampler; 0:
 *                    stream order.  With 1 or 2 the per-kernel profile times of
 *                    the light rows and the finish include concurrent work
 * Must be called before ntc_set_observed for "keep_perm".  Errors: NTC_ERR_ARG. */
ntc_status ntc_set_param(ntc_handle* h, const char* key, double value);
/* (also "profile": 1 brackets every mode-update kernel with CUDA events, see
 * ntc_get_profile; and the test hook "test_gram_stall": N > 0 makes block 0
 * of every tensor-core Gram launch wait up to N SM cycles on a phase that no
 * MMA was committed to, before it issues any, so that its bounded wait gives
 * up with nothing in flight -- default 0, off) */

/* Enqueue all further work on this cudaStream_t (e.g. a PyTorch stream);
 * NULL selects the legacy default stream.  Errors: none besides NTC_ERR_ARG. */
ntc_status ntc_set_stream(ntc_handle* h, void* cuda_stream);

/* Set the observed entries X(Omega) (Alg. 2 inputs X and Omega, Sec. II,
 * eq. M_def): idx[nnz][order] int32 and vals[nnz] float32 on the HOST.  Copies
 * them to the device, validates every index (NTC_ERR_INDEX if one is out of
 * range), buckets the entries of every mode by row with a stable device
 * counting sort, and, for modes whose factor was not set by ntc_set_factor,
 * draws the initial factors i.i.d. U[0, 2a], a = (mean(vals)/R)^(1/N).
 * Replaces any earlier observations.  Resets the AO iteration counter to 0. */
ntc_status ntc_set_observed(ntc_handle* h, int64_t nnz, const int32_t* idx, const float* vals);
/* Same, with idx_dev and vals_dev in device memory. */
ntc_status ntc_set_observed_dev(ntc_handle* h, int64_t nnz, const int32_t* idx_dev, const float* vals_dev);

/* One epoch of Algorithm 2: ceil(1/c) AO iterations (an epoch touches every
 * observation once on average, Sec. IV); in each, every mode in mode_order
 * (a permutation of 0..order-1; NULL means 0..order-1) is updated by
 * Algorithm 1 with minibatch fraction c (Sec. II-B: row p draws
 * floor(c n_p) of its n_p observations uniformly without replacement): the
 * k_p positions of the row with the smallest (key, position), where the key
 * of bucket position q is word q mod 4 of Philox4x32-10 with counter
 * {mode, AO iteration, inner iteration, q / 4} and key `seed`.  Modes updated
 * earlier in the AO iteration are used by later ones (Gauss-Seidel, Sec. III).
 * Enqueued on the stream; returns without synchronising.  0 < c <= 1.
 * Errors: NTC_ERR_STATE before ntc_set_observed, NTC_ERR_ARG. */
ntc_status ntc_epoch(ntc_handle* h, const int* mode_order, double c, uint64_t seed);

/* One call of Algorithm 1 (S_NMC) on `mode` at the current AO iteration
 * counter, which is left unchanged.  Errors as ntc_epoch. */
ntc_status ntc_snmc(ntc_handle* h, int mode, double c, uint64_t seed);

/* CPD model (eq. 1) at n host indices idx[n][order]; out[n] float32 (host).
 * Errors: NTC_ERR_INDEX, NTC_ERR_ARG. */
ntc_status ntc_predict(ntc_handle* h, int64_t n, const int32_t* idx, float* out);
/* Same with device buffers; enqueued, not synchronised.  The indices are
 * checked on the device: a query with an index out of range gives NaN. */
ntc_status ntc_predict_dev(ntc_handle* h, int64_t n, const int32_t* idx_dev, float* out_dev);

/* Root mean squared error of the model against vals[n] at idx[n][order]
 * (host), reduced in double precision in a fixed order.  *out on the host. */
ntc_status ntc_rmse(ntc_handle* h, int64_t n, const int32_t* idx, const float* vals, double* out);

/* Cost of eq. 3 over the observed set, reduced in double precision. */
ntc_status ntc_cost(ntc_handle* h, double* out);

/* Copy factor `mode` to/from host float32 [dims[mode]][rank].  Set rejects
 * negative or NaN values (NTC_ERR_ARG).  Get synchronises the stream. */
ntc_status ntc_get_factor(ntc_handle* h, int mode, float* out);
ntc_status ntc_set_factor(ntc_handle* h, int mode, const float* in);

/* AO iteration counter k (Alg. 2), which with the factors and the seed fixes
 * every later sample: a checkpoint is (factors, k). */
ntc_status ntc_get_state(ntc_handle* h, uint64_t* ao_iter);
ntc_status ntc_set_state(ntc_handle* h, uint64_t ao_iter);

/* Wait for all work enqueued by this handle.  NTC_ERR_CUDA if a kernel failed
 * or a tensor-core Gram wait gave up (see ntc_stats). */
ntc_status ntc_sync(ntc_handle* h);

/* Counters of the last ntc_epoch/ntc_snmc: visits = sum over row updates of
 * floor(c n_p) (the sampled observations), the part of them in rows split over
 * several blocks, rows updated, rows skipped (floor(c n_p) = 0), rows that used
 * the exact fallback selector, the algorithmic bytes moved (index, value and
 * factor-row reads per visit, factor-row reads/writes per row update), the
 * number of kernel launches enqueued, and the number of tensor-core Gram blocks
 * whose bounded wait (about one second) for their MMAs gave up (0 unless the
 * device misbehaved).  Such a block stops, frees its tensor memory and writes
 * no partial sums, so the rows it served are not valid: the next call that
 * synchronises the stream (ntc_sync, ntc_get_factor, ntc_predict, ntc_rmse,
 * ntc_cost) returns NTC_ERR_CUDA with a message, once per new timeout. */
typedef struct {
    int64_t visits;
    int64_t visits_heavy;
    int64_t rows_updated;
    int64_t rows_skipped;
    int64_t fallback_rows;
    int64_t alg_bytes;
    int64_t kernel_launches;
    int64_t wait_timeouts;
} ntc_stats;
ntc_status ntc_get_stats(ntc_handle* h, ntc_stats* out);

/* Per-kernel timing on the handle's stream.  With "profile" set to 1
 * (ntc_set_param), every kernel launch of the mode update is bracketed by CUDA
 * events.  ntc_get_profile synchronises the stream and returns, for kernel
 * class `kind` (NTC_K_*), the summed event time in ms, the number of launches
 * and the algorithmic bytes those launches moved by the model of the sampled
 * visits (index, value and factor-row reads per visit; factor-row traffic per
 * row update), then clears that class.  Errors: NTC_ERR_ARG for a bad kind. */
enum {
    NTC_K_LIGHT = 0,          /* fused sample + Gram/data sums, one block per row      */
    NTC_K_HEAVY_SAMPLE = 1,   /* keys and certain/candidate split per chunk            */
    NTC_K_HEAVY_RESOLVE = 2,  /* exact k-subset per split row                          */
    NTC_K_HEAVY_GRAM = 3,     /* Gram/data partials per chunk                           */
    NTC_K_FINISH = 4,         /* split-row partial sums, then every row's update       */
    NTC_K_COUNT = 5
};
ntc_status ntc_get_profile(ntc_handle* h, int kind, double* ms, int64_t* launches, int64_t* alg_bytes);

/* Utility: FP32 fused multiply-add throughput of the current device in
 * TFLOP/s, measured with a register-resident FMA kernel on `cuda_stream`
 * (2 flops per FMA).  The roofline of the ALU-bound Gram work uses it. */
ntc_status ntc_measure_fp32_peak(void* cuda_stream, double* tflops);

/* Test hooks.  ntc_get_bucket: the mode's bucket (Sec. II-B rows of X_(i)):
 * row_ptr[dims[mode]+1] and, if keep_perm was set, perm[nnz] (bucket position
 * -> observation index); either pointer may be NULL.  ntc_sample_mask: runs
 * only the sampler of Alg. 1 line 5 for `mode` at (c, seed, ao_iter, inner) and
 * writes mask[nnz] (host), 1 where the bucket position is sampled. */
ntc_status ntc_get_bucket(ntc_handle* h, int mode, int64_t* row_ptr, int64_t* perm);
ntc_status ntc_sample_mask(ntc_handle* h, int mode, double c, uint64_t seed, uint64_t ao_iter,
                           int inner, uint8_t* mask);

/* RMSE without allocating: the paper has no counterpart; this exists for
 * callers that cannot allocate device memory while they run -- a serving
 * process whose HBM is handed out up front to resident jobs, or a framework
 * whose caching allocator owns the device memory and must not see the
 * device-wide synchronisation that cudaMalloc/cudaFree can bring.  Same result
 * as ntc_rmse, but idx_dev[n][order] (int32) and vals_dev[n] (float32) are
 * DEVICE pointers on the handle's device, which must be current.  The indices
 * are checked on the device: if any is out of range the call returns
 * NTC_ERR_INDEX (no factor row is read for that query).  *out (host) receives
 * the RMSE; the call synchronises the handle's stream.  It calls no
 * cudaMalloc/cudaFree: its scratch is a fixed 32 KB array in the library's
 * device memory, one double per block of 2048 queries, so n may be at most
 * 4096 * 2048 = 8,388,608 (larger n returns NTC_ERR_ARG).  The first call on a
 * device looks up that array's address (a failed lookup is tried again on the
 * next call), so make that first call before any stream capture.  All calls
 * share the array: calls that overlap on the GPU (other streams, other
 * threads, other handles on the same device) race and must be serialised by
 * the caller.
 * Errors: NTC_ERR_ARG, NTC_ERR_INDEX, NTC_ERR_STATE (handle's device not
 * current), NTC_ERR_CUDA. */
ntc_status ntc_rmse_noalloc(ntc_handle* h, int64_t n, const int32_t* idx_dev, const float* vals_dev, double* out);

/* Message for the last failed call on h ("" if none); valid until the next call. */
const char* ntc_last_error(const ntc_handle* h);

/* Free the handle and all its device memory.  NULL is allowed. */
void ntc_destroy(ntc_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* NTC_H */
