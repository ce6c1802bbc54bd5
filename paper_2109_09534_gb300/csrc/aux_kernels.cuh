// aux_kernels.cuh -- device kernels around the NMC update: per-mode bucketing
// of the observed entries by row (a stable LSD radix counting sort), index
// validation, initial factors, and the model evaluations (eq. 1) behind
// predict, RMSE and the cost of eq. 3.
#pragma once

#include "ntc_internal.cuh"

namespace ntc {

constexpr int kSortIPT = 16;                       // keys per thread per tile
constexpr int kSortTile = kThreads * kSortIPT;     // 4096 keys per tile

// Storage row of each original row, per mode (factor rows are stored in
// descending order of their observation counts).
struct RowMaps {
    const int32_t* inv[kMaxOrder];   // original row -> storage row, per mode
};

// Any index outside [0, dims[i]) sets *bad.
__global__ void k_validate(const int32_t* idx, int64_t n, int order, const int64_t* dims_dev,
                           unsigned* bad) {
    int64_t dims[kMaxOrder];
    for (int i = 0; i < order; ++i) dims[i] = dims_dev[i];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        for (int i = 0; i < order; ++i) {
            const int32_t v = idx[e * order + i];
            if (v < 0 || v >= dims[i]) atomicOr(bad, 1u);
        }
    }
}

__global__ void k_extract_keys(const int32_t* idx, int64_t n, int order, int mode, uint32_t* keys,
                               uint32_t* payload) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        keys[e] = (uint32_t)idx[e * order + mode];
        payload[e] = (uint32_t)e;
    }
}

// Per-tile digit histograms, digit-major: hist[d * ntiles + tile].
__global__ void __launch_bounds__(kThreads) k_radix_hist(const uint32_t* keys, int64_t n, int shift,
                                                         uint32_t* hist, int ntiles) {
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
    for (int r = 0; r < kSortIPT; ++r) {
        const int64_t i = base + (int64_t)r * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: warp w of a tile owns keys [w*512, w*512+512) in order, in
// 16 rounds of 32; equal digits within a round are ranked by lane, rounds and
// warps in order, so the output keeps the input order of equal keys.  The tile
// is first placed in shared memory in (digit, input order) order and then
// written out front to back, so that the global writes of one digit's run are
// contiguous.
__global__ void __launch_bounds__(kThreads) k_radix_scatter(const uint32_t* kin, const uint32_t* vin,
                                                            uint32_t* kout, uint32_t* vout, int64_t n,
                                                            int shift, const uint32_t* offs, int ntiles) {
    __shared__ unsigned wh[kThreads / 32][256];
    __shared__ uint32_t sk[kSortTile], sv[kSortTile];
    __shared__ int gbase[256];   // global position of a digit's run minus its tile-local start
    __shared__ int scan_tmp[kThreads / 32 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
    const int64_t base = tile0 + (int64_t)warp * (32 * kSortIPT);
    uint32_t key[kSortIPT], val[kSortIPT];
#pragma unroll
    for (int r = 0; r < kSortIPT; ++r) {
        const int64_t i = base + r * 32 + lane;
        key[r] = i < n ? kin[i] : 0u;
        val[r] = i < n ? vin[i] : 0u;
    }
    for (int d = lane; d < 256; d += 32) wh[warp][d] = 0;
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kSortIPT; ++r) {
        const bool valid = base + r * 32 + lane < n;
        const unsigned d = valid ? ((key[r] >> shift) & 255u) : 256u + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (valid && (peers & lt) == 0) wh[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        // thread d: the digit's tile-local start, then per-warp starts
        const int d = threadIdx.x;
        int cnt = 0;
        for (int w = 0; w < kThreads / 32; ++w) cnt += (int)wh[w][d];
        int tot;
        const int start = block_exclusive_scan(cnt, scan_tmp, &tot);
        gbase[d] = (int)offs[(int64_t)d * ntiles + blockIdx.x] - start;
        unsigned run = (unsigned)start;
        for (int w = 0; w < kThreads / 32; ++w) {
            const unsigned t = wh[w][d];
            wh[w][d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortIPT; ++r) {
        const bool valid = base + r * 32 + lane < n;
        const unsigned d = valid ? ((key[r] >> shift) & 255u) : 256u + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned pos = 0;
        if (valid) pos = wh[warp][d] + __popc(peers & lt);
        __syncwarp();
        if (valid && (peers & lt) == 0) wh[warp][d] += __popc(peers);
        __syncwarp();
        if (valid) {
            sk[pos] = key[r];
            sv[pos] = val[r];
        }
    }
    __syncthreads();
    const int tn = (int)min((int64_t)kSortTile, n - tile0);
    for (int i = threadIdx.x; i < tn; i += kThreads) {
        const uint32_t k = sk[i];
        const int64_t g = (int64_t)gbase[(k >> shift) & 255u] + i;
        kout[g] = k;
        vout[g] = sv[i];
    }
}

// Keys of `mode` and the 16-byte bucket entries of orders 2-4 in input order,
// built from the COO in one coalesced pass: the other modes' indices mapped to
// storage rows (slot w holds mode w, or w + 1 past `mode`), then the value.
__global__ void k_build_keys_entries(const int32_t* idx, const float* vals, int64_t n, int order, int mode,
                                     RowMaps maps, uint32_t* keys, uint4* out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t* row = idx + e * order;
        uint32_t w[3];
#pragma unroll
        for (int sl = 0; sl < 3; ++sl) {
            const int src = sl + (sl >= mode ? 1 : 0);
            w[sl] = src < order ? (uint32_t)maps.inv[src][row[src]] : 0u;
        }
        keys[e] = (uint32_t)row[mode];
        out[e] = make_uint4(w[0], w[1], w[2], __float_as_uint(vals[e]));
    }
}

// The same stable scatter with 16-byte bucket entries as payloads, so that
// the last pass writes the bucket directly.  Dynamic shared memory:
// kEntScatterSmem bytes.
constexpr size_t kEntScatterSmem = (size_t)(kThreads / 32) * 256 * 4 + (size_t)kSortTile * 4 +
                                   (size_t)kSortTile * 16 + 256 * 4 + (kThreads / 32 + 1) * 4;
__global__ void __launch_bounds__(kThreads, 2) k_radix_scatter_ent(const uint32_t* kin, const uint4* pin,
                                                                   uint32_t* kout, uint4* pout, int64_t n, int shift,
                                                                   const uint32_t* offs, int ntiles) {
    extern __shared__ __align__(16) unsigned char es[];
    unsigned(*wh)[256] = reinterpret_cast<unsigned(*)[256]>(es);
    uint32_t* sk = reinterpret_cast<uint32_t*>(es + (kThreads / 32) * 256 * 4);
    uint4* sp = reinterpret_cast<uint4*>(sk + kSortTile);
    int* gbase = reinterpret_cast<int*>(sp + kSortTile);
    int* scan_tmp = gbase + 256;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
    const int64_t base = tile0 + (int64_t)warp * (32 * kSortIPT);
    uint32_t key[kSortIPT];
#pragma unroll
    for (int r = 0; r < kSortIPT; ++r) {
        const int64_t i = base + r * 32 + lane;
        key[r] = i < n ? kin[i] : 0u;
    }
    for (int d = lane; d < 256; d += 32) wh[warp][d] = 0;
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kSortIPT; ++r) {
        const bool valid = base + r * 32 + lane < n;
        const unsigned d = valid ? ((key[r] >> shift) & 255u) : 256u + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (valid && (peers & lt) == 0) wh[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        const int d = threadIdx.x;
        int cnt = 0;
        for (int w = 0; w < kThreads / 32; ++w) cnt += (int)wh[w][d];
        int tot;
        const int start = block_exclusive_scan(cnt, scan_tmp, &tot);
        gbase[d] = (int)offs[(int64_t)d * ntiles + blockIdx.x] - start;
        unsigned run = (unsigned)start;
        for (int w = 0; w < kThreads / 32; ++w) {
            const unsigned t = wh[w][d];
            wh[w][d] = run;
            run += t;
        }
    }
    __syncthreads();
    // ranks first (keys staged), then each payload loaded once and staged at
    // its key's slot, so that no thread holds all of its payloads at once
    unsigned pos[kSortIPT];
#pragma unroll
    for (int r = 0; r < kSortIPT; ++r) {
        const bool valid = base + r * 32 + lane < n;
        const unsigned d = valid ? ((key[r] >> shift) & 255u) : 256u + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        pos[r] = 0;
        if (valid) pos[r] = wh[warp][d] + __popc(peers & lt);
        __syncwarp();
        if (valid && (peers & lt) == 0) wh[warp][d] += __popc(peers);
        __syncwarp();
        if (valid) sk[pos[r]] = key[r];
    }
#pragma unroll
    for (int r = 0; r < kSortIPT; ++r) {
        const int64_t i = base + r * 32 + lane;
        if (i < n) sp[pos[r]] = pin[i];
    }
    __syncthreads();
    const int tn = (int)min((int64_t)kSortTile, n - tile0);
    for (int i = threadIdx.x; i < tn; i += kThreads) {
        const uint32_t k = sk[i];
        const int64_t g = (int64_t)gbase[(k >> shift) & 255u] + i;
        kout[g] = k;
        pout[g] = sp[i];
    }
}

// Exclusive scan of n uint32 values (n < 2^31), three phases: block sums,
// a one-block scan of the block sums, block-local scans with carry-in.
constexpr int kScanBlock = 2048;

__global__ void __launch_bounds__(kThreads) k_scan_sums(const uint32_t* in, int64_t n, uint32_t* sums) {
    __shared__ int tmp[kThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    unsigned s = 0;
    for (int i = threadIdx.x; i < kScanBlock; i += kThreads)
        if (base + i < n) s += in[base + i];
    int tot;
    block_exclusive_scan((int)s, tmp, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = (uint32_t)tot;
}

__global__ void __launch_bounds__(kThreads) k_scan_top(uint32_t* sums, int nb) {
    __shared__ int tmp[kThreads / 32 + 1];
    unsigned carry = 0;
    for (int base = 0; base < nb; base += kThreads) {
        const int i = base + threadIdx.x;
        const unsigned v = i < nb ? sums[i] : 0u;
        int tot;
        const int ex = block_exclusive_scan((int)v, tmp, &tot);
        if (i < nb) sums[i] = carry + (unsigned)ex;
        carry += (unsigned)tot;
    }
}

__global__ void __launch_bounds__(kThreads) k_scan_apply(const uint32_t* in, int64_t n, const uint32_t* sums,
                                                         uint32_t* out) {
    __shared__ int tmp[kThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    constexpr int PER = kScanBlock / kThreads;   // 8 consecutive values per thread
    unsigned v[PER];
    unsigned s = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int64_t i = base + (int64_t)threadIdx.x * PER + j;
        v[j] = i < n ? in[i] : 0u;
        s += v[j];
    }
    int tot;
    unsigned run = sums[blockIdx.x] + (unsigned)block_exclusive_scan((int)s, tmp, &tot);
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int64_t i = base + (int64_t)threadIdx.x * PER + j;
        if (i < n) out[i] = run;
        run += v[j];
    }
}

// row_ptr from sorted row keys: row_ptr[r] = first position whose key >= r.
__global__ void k_row_ptr(const uint32_t* keys, int64_t n, int64_t dim, int64_t* row_ptr) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q <= n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lo = q == 0 ? 0 : (int64_t)keys[q - 1] + 1;
        const int64_t hi = q == n ? dim : (int64_t)keys[q];
        for (int64_t r = lo; r <= hi; ++r) row_ptr[r] = q;
    }
}

// Observations per row of `mode` (exact integer histogram).  Skewed indices
// put a large share of all increments on a few rows, so increments are first
// combined: in a block-private shared-memory histogram when the mode has at
// most kCountSmemRows rows (flushed once per block), else among the lanes of a
// warp that hold the same row.
constexpr int kCountSmemRows = 12288;
__global__ void __launch_bounds__(256) k_count_rows(const int32_t* idx, int64_t n, int order, int mode, int64_t rows,
                                                    uint32_t* counts) {
    __shared__ uint32_t sh[kCountSmemRows];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (rows <= kCountSmemRows) {
        for (int i = threadIdx.x; i < rows; i += blockDim.x) sh[i] = 0u;
        __syncthreads();
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += stride)
            atomicAdd(&sh[idx[e * order + mode]], 1u);
        __syncthreads();
        for (int i = threadIdx.x; i < rows; i += blockDim.x)
            if (sh[i]) atomicAdd(&counts[i], sh[i]);
        return;
    }
    for (int64_t e0 = blockIdx.x * (int64_t)blockDim.x; e0 < n; e0 += stride) {
        const int64_t e = e0 + threadIdx.x;
        const bool in = e < n;
        const int r = in ? idx[e * order + mode] : -1;
        const unsigned same = __match_any_sync(0xffffffffu, r);
        if (in && (threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&counts[r], (unsigned)__popc(same));
    }
}


// Bucket entries of `mode` (the other modes' indices mapped to their storage
// rows, then the value) in input order, with coalesced reads of the COO;
// k_gather_entries then puts them in bucket order with one random 16- or
// 32-byte read per entry.
template <int EW>
__global__ void k_build_entries(const int32_t* idx, const float* vals, int64_t n, int order, int mode, RowMaps maps,
                                Entry<EW>* out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        Entry<EW> en;
        // slot w holds mode w, or w + 1 past `mode` (slot positions fixed at compile time)
#pragma unroll
        for (int w = 0; w < EW - 1; ++w) {
            const int src = w + (w >= mode ? 1 : 0);
            en.w[w] = src < order ? maps.inv[src][idx[e * order + src]] : 0;
        }
        en.w[EW - 1] = __float_as_int(vals[e]);
        out[e] = en;
    }
}

template <int EW>
__global__ void k_gather_entries(const Entry<EW>* in, const uint32_t* perm, int64_t n, Entry<EW>* out) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        out[q] = in[perm[q]];
}

// Fixed-order double-precision sums: per-block partials, then one block.
__device__ __forceinline__ double block_sum_d(double v, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) t += sh[w];
    __syncthreads();
    return t;   // valid in thread 0
}

__global__ void __launch_bounds__(kThreads) k_sum_f32(const float* x, int64_t n, double* partial) {
    __shared__ double sh[kThreads / 32];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
        s += (double)x[i];
    const double t = block_sum_d(s, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kThreads) k_sum_partials(const double* partial, int nb, double* out) {
    __shared__ double sh[kThreads / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += kThreads) s += partial[i];
    const double t = block_sum_d(s, sh);
    if (threadIdx.x == 0) *out = t;
}

// Initial factors: i.i.d. U[0, 2a] from Philox(counter {0xFFFF, mode, row,
// col}, key init_seed) with `row` the original row index, u = (word0 + 1/2)
// 2^-32, drawn in double, stored rounded to float at the row's storage slot;
// padding columns are zero.
// Cold start of the warm-started power method: ones/sqrt(R) in the R columns.
__global__ void k_fill_warm(float* V, int64_t rows, int R, int rp) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < rows * rp; q += (int64_t)gridDim.x * blockDim.x)
        V[q] = (int)(q % rp) < R ? 1.0f / sqrtf((float)R) : 0.f;
}

__global__ void k_init_factor(float* U, uint16_t* Ub, int64_t rows, int R, int rp, int mode,
                              const double* sum_vals, int64_t nnz, int order, uint32_t k0, uint32_t k1,
                              const int32_t* perm_rows) {
    const double mean = nnz > 0 ? *sum_vals / (double)nnz : 0.0;
    const double a = mean > 0.0 ? pow(mean / (double)R, 1.0 / (double)order) : 0.0;
    const int64_t total = rows * rp;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = t / rp;
        const int r = (int)(t - p * rp);
        float v = 0.f;
        if (r < R) {
            const uint32_t orig = (uint32_t)perm_rows[p];
            const uint4 w = philox4(0xFFFFu, (uint32_t)mode, orig, (uint32_t)r, k0, k1);
            const double u = ((double)w.x + 0.5) * (1.0 / 4294967296.0);
            v = (float)(2.0 * a * u);
        }
        U[t] = v;
        if (Ub) Ub[t] = f32_to_bf16_rne(v);
    }
}

__global__ void k_to_bf16(const float* U, uint16_t* Ub, int64_t n) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        Ub[t] = f32_to_bf16_rne(U[t]);
}

struct FactorSet {
    const float* U[kMaxOrder];
    const int32_t* inv[kMaxOrder];   // original row -> storage row
    int64_t dims[kMaxOrder];
    int order, R, rp;
};

// Every index of the tuple in [0, dims[i]): the kernels that take indices
// from device memory the host has not validated test this before any read.
__device__ __forceinline__ bool index_ok(const FactorSet& f, const int32_t* ix) {
    bool ok = true;
    for (int i = 0; i < f.order; ++i) ok = ok && ix[i] >= 0 && (int64_t)ix[i] < f.dims[i];
    return ok;
}

// Model value (eq. 1) at one index, float32 products and sum.
__device__ __forceinline__ float model_at(const FactorSet& f, const int32_t* ix) {
    const float* row[kMaxOrder];
    for (int i = 0; i < f.order; ++i) row[i] = f.U[i] + (size_t)f.inv[i][ix[i]] * f.rp;
    float acc = 0.f;
    for (int r = 0; r < f.R; ++r) {
        float p = row[0][r];
        for (int i = 1; i < f.order; ++i) p *= row[i][r];
        acc += p;
    }
    return acc;
}

// Model values at n index tuples; a tuple with an index out of range gives NaN
// and reads no factor.
__global__ void k_predict(FactorSet f, const int32_t* idx, int64_t n, float* out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t* ix = idx + e * f.order;
        out[e] = index_ok(f, ix) ? model_at(f, ix) : __int_as_float(0x7fc00000);
    }
}

// Queries of several jobs in one launch: query e reads job table[slot[e]] at
// the index idx[e * kMaxOrder ...] (entries past that job's order unused).
__global__ void k_predict_multi(const FactorSet* table, const int32_t* slot, const int32_t* idx, int64_t n,
                                float* out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const FactorSet& f = table[slot[e]];
        const int32_t* ix = idx + e * kMaxOrder;
        out[e] = index_ok(f, ix) ? model_at(f, ix) : __int_as_float(0x7fc00000);
    }
}

// Per-block double sums of (x - model)^2.  A tuple with an index out of range
// is left out of the sum and, if `bad` is not null, sets *bad to 1.
__global__ void __launch_bounds__(kThreads) k_sq_resid(FactorSet f, const int32_t* idx, const float* vals,
                                                       int64_t n, double* partial,
                                                       unsigned long long* bad = nullptr) {
    __shared__ double sh[kThreads / 32];
    double s = 0.0;
    bool any_bad = false;
    for (int64_t e = blockIdx.x * (int64_t)kThreads + threadIdx.x; e < n; e += (int64_t)gridDim.x * kThreads) {
        const int32_t* ix = idx + e * f.order;
        if (!index_ok(f, ix)) {
            any_bad = true;
            continue;
        }
        const double d = (double)vals[e] - (double)model_at(f, ix);
        s += d * d;
    }
    if (any_bad && bad) atomicOr(bad, 1ull);
    const double t = block_sum_d(s, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kThreads) k_sq_sum(const float* x, int64_t n, double* partial) {
    __shared__ double sh[kThreads / 32];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
        s += (double)x[i] * (double)x[i];
    const double t = block_sum_d(s, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

}  // namespace ntc
