// ntc_host.h -- host-side types shared by the C ABI implementation
// (ntc_api.cu) and the per-rank launch units (nmc_rp*.cu): device buffers,
// the per-(mode, c) work plan, the handle, and the kernel launcher.
#pragma once

#include <cstring>
#include <string>
#include <mutex>
#include <vector>

#include <cuda.h>

#include "../../include/ntc.h"
#include "ntc_internal.cuh"

namespace ntc {

struct DevMem {
    void* p = nullptr;
    size_t bytes = 0;
    DevMem() = default;
    DevMem(const DevMem&) = delete;
    DevMem& operator=(const DevMem&) = delete;
    ~DevMem() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    // grow-only; contents are not preserved
    cudaError_t ensure(size_t b) {
        if (b <= bytes && p) return cudaSuccess;
        release();
        if (b == 0) b = 16;
        cudaError_t e = cudaMalloc(&p, b);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        bytes = b;
        return cudaSuccess;
    }
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

struct ModePlan {
    bool valid = false;
    double c = 0.0;
    int heavy_threshold = 0, chunk = 0;
    double bracket_z = 0.0;
    int64_t visits = 0, visits_heavy = 0, rows_updated = 0, rows_skipped = 0;
    int n_light = 0, n_heavy = 0, n_chunks = 0, n_tiny = 0;
    int n_tiny_big = 0;   // leading one-warp rows with more than 32 visits (rows are longest first)
    bool tiny = false;   // rows of <= 509 observations went to the one-warp-per-row kernel
    int64_t cand_total = 0, extra_total = 0;
    int n_groups = 0;
    DevMem light_rows, light_k, chunks, chunk_caps, heavy, bracket, heavy_cand, groups, heavy_groups;
    DevMem tiny_rows, tiny_k;
    DevMem vis_off;   // per chunk: start of its visit list in the epoch-permutation variant
};

inline int pad_rank(int R) { return R <= 8 ? 8 : R <= 16 ? 16 : R <= 32 ? 32 : 64; }

// TMA descriptors of the other modes' factor matrices for the row gathers of
// one mode update (gram_tma.cuh reads them as a kernel parameter).
struct GatherMaps {
    CUtensorMap m[3];
};

}  // namespace ntc

struct ntc_handle {
    int order = 0;
    int64_t dims[ntc::kMaxOrder] = {};
    int rank = 0, rp = 0;
    double lambda = 0.0;
    // parameters
    int max_inner = 1, power_iters = 10, storage_bf16 = 0, keep_perm = 0;
    uint64_t init_seed = 3;
    // split-row chunks of 65536 positions and a bracket of 6 standard
    // deviations (a row misses it, and takes the exact fallback, with
    // probability about 2e-9 per update): on the Zipf(1.1) 10^4-cube at R = 32
    // the epoch took 20.7 ms with 16384 / 7, 19.4 with 65536 / 7, 19.1 with
    // 65536 / 6, 22.2 with 262144
    double bracket_z = 6.0;
    int heavy_threshold = 4096, chunk = 65536;
    cudaStream_t stream = nullptr;
    // light rows run on a side stream beside the split-row kernels of the same
    // mode update (they write disjoint rows); fork/join through two events
    int overlap = 2;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int device = 0;
    // state
    uint64_t ao_iter = 0;
    int64_t nnz = -1;
    bool factor_set[ntc::kMaxOrder] = {};
    std::string err;
    ntc_stats stats = {};
    // device data
    ntc::DevMem U[ntc::kMaxOrder], Ub[ntc::kMaxOrder], Y;
    ntc::DevMem row_ptr[ntc::kMaxOrder], bucket[ntc::kMaxOrder], perm[ntc::kMaxOrder];
    // Factor rows are stored in descending order of their mode's observation
    // counts (storage row = inv[original row], original row = rows[storage row]),
    // so that the most frequent rows of a mode are its first storage rows.
    // Identity until observations are set.  Bucket positions keep original order.
    ntc::DevMem inv_dev[ntc::kMaxOrder], rows_dev[ntc::kMaxOrder];
    std::vector<int32_t> inv_h[ntc::kMaxOrder], rows_h[ntc::kMaxOrder];
    ntc::DevMem coo_idx, coo_val, dims_dev;
    std::vector<int64_t> row_ptr_h[ntc::kMaxOrder];
    ntc::ModePlan plan[ntc::kMaxOrder];
    // scratch
    // split-row sampling scratch, two sets: update u uses set u % 2, so the
    // sampling of the next mode update can run while this one's Gram reads
    // its lists ("pipeline")
    ntc::DevMem vis[2], vis_cnt[2], cand[2], cand_cnt[2], extra[2], extra_cnt[2], flags[2];
    ntc::DevMem partial, partial2, row_sum, stat, red, mask;
    int pipeline = 1;
    int gram_tc = 1;         // split-row Gram on the tensor cores where a kernel exists (R_pad 32, orders 2-4)
    int tiny_rows = 1;       // rows of <= 509 observations one warp each (orders 2-4)
    // tensor-core Gram blocks that gave up a bounded wait, as last reported
    // to the caller; test hook that makes block 0 of each such launch give up
    unsigned long long faults_seen = 0;
    long long test_stall_cycles = 0;
    // TMA descriptors of the row gathers, per updated mode, encoded on first use
    // (factor buffers never move after ntc_create / storage_bf16)
    ntc::GatherMaps gmaps[ntc::kMaxOrder];
    int gmaps_state[ntc::kMaxOrder] = {};   // 0 none, 1 float32 masters, 2 bfloat16 copies
    uint64_t upd = 0;                       // mode updates launched so far
    cudaStream_t samp = nullptr;            // split-row sampling stream
    cudaEvent_t ev_sampled[2] = {}, ev_free[2] = {};
    // ntc_set_observed staging (the next COO) and radix-sort buffers, kept
    // between calls unless "cache_staging" is 0
    int cache_staging = 1;
    // warm-started power method: last vector per row, per mode (storage order)
    int power_warm = 0;
    int sampler = 0;   // 0: independent samples; 1: epoch permutation
    bool warm_ready[ntc::kMaxOrder] = {};
    ntc::DevMem vwarm[ntc::kMaxOrder];
    ntc::DevMem stage_idx, stage_val, sort_k0, sort_k1, sort_v0, sort_v1, sort_hist, sort_sums, bad_flag, row_cnt,
        entry_tmp;
    // per-kernel event timing ("profile")
    int profile = 0;
    struct Pending {
        int kind;
        int64_t bytes;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    double prof_ms[NTC_K_COUNT] = {};
    int64_t prof_launches[NTC_K_COUNT] = {}, prof_bytes[NTC_K_COUNT] = {};
    ~ntc_handle() {
        for (auto& q : pending) {
            cudaEventDestroy(q.a);
            cudaEventDestroy(q.b);
        }
        if (side) cudaStreamDestroy(side);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        for (int b = 0; b < 2; ++b) {
            if (ev_sampled[b]) cudaEventDestroy(ev_sampled[b]);
            if (ev_free[b]) cudaEventDestroy(ev_free[b]);
        }
        if (samp) cudaStreamDestroy(samp);
    }
};


namespace ntc {

// ---- one-time smem attributes per kernel instantiation --------------------
template <class K>
inline cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// ---- mode update launches ---------------------------------------------------
// Enqueues one kernel; with profiling on, brackets it with a pair of events.
struct Launcher {
    ntc_handle* h;
    cudaStream_t s;
    int64_t* launches;
    int64_t bpv, bpr;   // algorithmic bytes per visit and per row update
    template <class F>
    cudaError_t run(int kind, int64_t bytes, F&& f) { return run_on(s, kind, bytes, f); }
    template <class F>
    cudaError_t run_on(cudaStream_t s, int kind, int64_t bytes, F&& f) {
        cudaEvent_t a = nullptr, b = nullptr;
        if (h->profile) {
            cudaError_t e = cudaEventCreate(&a);
            if (e == cudaSuccess) e = cudaEventCreate(&b);
            if (e == cudaSuccess) e = cudaEventRecord(a, s);
            if (e != cudaSuccess) return e;
        }
        f();
        ++*launches;
        if (h->profile) {
            cudaError_t e = cudaEventRecord(b, s);
            if (e != cudaSuccess) return e;
            h->pending.push_back({kind, bytes, a, b});
        }
        return cudaSuccess;
    }
};

template <int RP>
cudaError_t launch_mode_rp(int ew, bool bf, const ModeArgs& a, const ModePlan& p, Launcher& L, bool mask_only);
extern template cudaError_t launch_mode_rp<8>(int, bool, const ModeArgs&, const ModePlan&, Launcher&, bool);
extern template cudaError_t launch_mode_rp<16>(int, bool, const ModeArgs&, const ModePlan&, Launcher&, bool);
extern template cudaError_t launch_mode_rp<32>(int, bool, const ModeArgs&, const ModePlan&, Launcher&, bool);
extern template cudaError_t launch_mode_rp<64>(int, bool, const ModeArgs&, const ModePlan&, Launcher&, bool);

// ---- entry points for the serving runtime (serve.cu), in ntc_api.cu ---------
// Held-out squared residual sum of the handle's current factors, reduced on
// the handle's stream into scratch (>= kRmseScratch doubles, device) and copied
// to *host_sum (pinned host memory) -- nothing waits.
constexpr int kRmseScratch = 1025;
cudaError_t rmse_enqueue(ntc_handle* h, const int32_t* idx, const float* vals, int64_t n, double* scratch,
                         double* host_sum);
// CP model values for n queries over several handles in one kernel launch on
// stream s: query e uses handles[slot[e]] and idx[e * kMaxOrder ...].  The
// factors are read from snaps[j] when it is not null (all modes of handle j,
// mode m at offset sum_{i<m} dims[i] * rp floats, as snapshot_factors writes
// them), else from the handle's masters.  table is device memory for nh factor
// tables (>= nh * factor_table_bytes()).
size_t factor_table_bytes();
cudaError_t predict_multi(ntc_handle* const* handles, const float* const* snaps, int nh, const int32_t* slot,
                          const int32_t* idx, int64_t n, float* out, void* table, cudaStream_t s);
// Copies every mode's FP32 masters into dst (layout above) on the handle's stream.
cudaError_t snapshot_factors(ntc_handle* h, float* dst);
int64_t snapshot_floats(const ntc_handle* h);
// Device bytes the handle holds now.
int64_t handle_device_bytes(const ntc_handle* h);
// Builds every mode's plan for minibatch fraction c and sizes the epoch
// scratch, so that the first ntc_epoch at c allocates nothing.
ntc_status prepare_epoch(ntc_handle* h, double c);
// The row-gather descriptors of mode `mode` for the handle's current storage
// (encoded once and cached in the handle).
cudaError_t gather_maps(ntc_handle* h, int mode, const GatherMaps** out);
// Enqueues on the handle's stream a copy of the number of tensor-core Gram
// blocks that have given up a bounded wait since the handle was created into
// *host (pinned host memory); 0 if the handle has not run an update.
cudaError_t fault_count_enqueue(ntc_handle* h, unsigned long long* host);

}  // namespace ntc
