// ntc_internal.cuh -- shared device helpers and kernel argument layouts of the
// GB300 tensor-completion library.  Nothing here is visible through the C ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ntc {

constexpr int kMaxOrder = 8;
constexpr int kThreads = 256;        // threads per block of every row/chunk kernel
constexpr int kLightMax = 4096;      // largest row whose keys fit in shared memory
constexpr int kReduceGroup = 16;     // split-row partials summed per block of the group reduction
// Largest row handled by one warp from sample to update (tiny_rows.cuh): its
// positions, widened to whole Philox blocks, are at most 32 lanes x 16 keys.
constexpr int kTinyMax = 509;
// One-warp rows at padded rank 64 with at most this many visits keep their
// gathered rows K instead of forming G, and take a launch of their own with a
// smaller shared-memory footprint (tiny_rows.cuh).
constexpr int kTinyKForm = 32;

// Bucket entry of one observation, seen from the mode being updated: the other
// modes' indices in increasing mode order, then the value in the last word.
// EW = 4 words (16 B, one 128-bit load) for order <= 4, else 8 words (32 B).
template <int EW>
struct alignas(EW * 4) Entry {
    int32_t w[EW];
};

// ---- Philox4x32-10 (Salmon et al., SC'11): two 32x32 multiplies per round,
// high halves xored with the other words and the round key; Weyl key bumps.
__device__ __forceinline__ uint4 philox4(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                         uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

// Sampling stream of one (mode, AO iteration, inner iteration): the key of
// bucket position q is word q mod 4 of Philox(counter {mode, k, l, q / 4},
// key seed), so one block gives the keys of four consecutive positions.
struct SampleStream {
    uint32_t mode, iter, inner, k0, k1;
};

// Keys of one sampling stream with the uniform part precomputed.  Within a
// launch only the counter's last word (the block index g = q / 4) varies, so
// in rounds 1-3 of Philox4x32-10 one product per round depends on g and the
// other is the same for every block.  key4(g) returns the four words of block
// g (the keys of positions 4g .. 4g+3), key(q) the key of one position.
struct KeyGen {
    uint32_t A, B, D, E, F, k0, k1;
    __device__ explicit KeyGen(const SampleStream& s) : k0(s.k0), k1(s.k1) {
        constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
        // round 1 on (mode, iter, inner, .): words 0, 1, 3 are uniform
        const unsigned long long p0 = (unsigned long long)M0 * s.mode, p1 = (unsigned long long)M1 * s.inner;
        const uint32_t c0_1 = (uint32_t)(p1 >> 32) ^ s.iter ^ k0, c1_1 = (uint32_t)p1, c3_1 = (uint32_t)p0;
        A = (uint32_t)(p0 >> 32) ^ k1;            // word 2 after round 1 is A ^ g
        // round 2: the product of word 0 is uniform
        B = c1_1 ^ (k0 + W0);
        const unsigned long long u0 = (unsigned long long)M0 * c0_1;
        const uint32_t c2_2 = (uint32_t)(u0 >> 32) ^ c3_1 ^ (k1 + W1), c3_2 = (uint32_t)u0;
        // round 3: the product of word 2 is uniform
        const unsigned long long u1 = (unsigned long long)M1 * c2_2;
        D = (uint32_t)(u1 >> 32) ^ (k0 + 2u * W0);
        F = (uint32_t)u1;
        E = c3_2 ^ (k1 + 2u * W1);
    }
    __device__ __forceinline__ uint4 key4(uint32_t g) const {
        constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
        const unsigned long long p1 = (unsigned long long)M1 * (A ^ g);
        const uint32_t c1_2 = (uint32_t)p1;
        const unsigned long long p0 = (unsigned long long)M0 * ((uint32_t)(p1 >> 32) ^ B);
        uint32_t c0 = c1_2 ^ D, c1 = F, c2 = (uint32_t)(p0 >> 32) ^ E, c3 = (uint32_t)p0;
        uint32_t r0 = k0 + 3u * W0, r1 = k1 + 3u * W1;
#pragma unroll
        for (int r = 3; r < 10; ++r) {
            const unsigned long long m0 = (unsigned long long)M0 * c0;
            const unsigned long long m1 = (unsigned long long)M1 * c2;
            c0 = (uint32_t)(m1 >> 32) ^ c1 ^ r0;
            c1 = (uint32_t)m1;
            c2 = (uint32_t)(m0 >> 32) ^ c3 ^ r1;
            c3 = (uint32_t)m0;
            r0 += W0;
            r1 += W1;
        }
        return make_uint4(c0, c1, c2, c3);
    }
    __device__ __forceinline__ uint32_t key(uint32_t q) const {
        const uint4 w = key4(q >> 2);
        const uint32_t j = q & 3u;
        return j == 0u ? w.x : j == 1u ? w.y : j == 2u ? w.z : w.w;
    }
};

// Epoch-permutation sampling variant: row `row`'s pseudo-random permutation
// of [0, n) in epoch `epoch` -- an 8-round balanced Feistel network on at
// least 8 bits (the smallest even number covering n), walked until the value
// falls below n.  Round keys: the words of two Philox4x32-10 blocks with
// counters {0xF2000000 | mode, epoch, row, 0 or 1} under the sampling seed;
// round function: MurmurHash3's 32-bit finaliser (Appleby) of the right half
// xor the round key.  The walk from i < n meets a value below n within one
// cycle of the network's permutation, so it ends.
__device__ __forceinline__ uint32_t fmix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x85ebca6bu;
    x ^= x >> 13;
    x *= 0xc2b2ae35u;
    x ^= x >> 16;
    return x;
}

struct PermGen {
    uint32_t K[8];
    uint32_t n, mask;
    int half;
    __device__ PermGen(uint32_t k0, uint32_t k1, uint32_t mode, uint32_t epoch, uint32_t row, uint32_t n_) : n(n_) {
        const uint4 a = philox4(0xF2000000u | mode, epoch, row, 0u, k0, k1);
        const uint4 b = philox4(0xF2000000u | mode, epoch, row, 1u, k0, k1);
        K[0] = a.x; K[1] = a.y; K[2] = a.z; K[3] = a.w;
        K[4] = b.x; K[5] = b.y; K[6] = b.z; K[7] = b.w;
        int bits = 0;
        while (bits < 32 && (1ull << bits) < (unsigned long long)n) ++bits;
        half = (bits + 1) / 2;
        if (half < 4) half = 4;
        mask = (1u << half) - 1u;
    }
    // one pass of the network (a permutation of [0, 2^(2 half)))
    __device__ __forceinline__ uint32_t pass(uint32_t x) const {
        uint32_t L = x >> half, R = x & mask;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const uint32_t t = L ^ (fmix32(R ^ K[r]) & mask);
            L = R;
            R = t;
        }
        return (L << half) | R;
    }
    __device__ __forceinline__ uint32_t map(uint32_t i) const {
        if (n <= 1) return 0u;
        uint32_t x = i;
        do x = pass(x);
        while (x >= n);
        return x;
    }
    // pi(s0 + j mod n) for j = j0, j0 + stride, ... < j1, each written by
    // emit(j, pi): a lane walks its own value one pass per step and moves to
    // its next j as soon as the value falls below n, so lanes of a warp do not
    // wait for each other's walks.  Every thread of the warp must call it.
    template <class Emit>
    __device__ __forceinline__ void map_range(uint32_t s0, uint32_t j0, uint32_t j1, uint32_t stride,
                                              const Emit& emit) const {
        uint32_t j = j0;
        bool have = j < j1;
        auto start = [&](uint32_t jj) {
            const uint32_t t = s0 + jj;
            return t >= n ? t - n : t;
        };
        uint32_t x = have ? start(j) : 0u;
        if (n <= 1) {
            for (; j < j1; j += stride) emit(j, 0u);
            return;
        }
        while (__any_sync(0xffffffffu, have)) {
            if (have) {
                x = pass(x);
                if (x < n) {
                    emit(j, x);
                    j += stride;
                    have = j < j1;
                    if (have) x = start(j);
                }
            }
        }
    }
};

// ---- bfloat16 storage helpers (round to nearest even on store).
__device__ __forceinline__ float4 bf16x4_to_f32(uint2 v) {
    float4 r;
    r.x = __uint_as_float(v.x << 16);
    r.y = __uint_as_float(v.x & 0xFFFF0000u);
    r.z = __uint_as_float(v.y << 16);
    r.w = __uint_as_float(v.y & 0xFFFF0000u);
    return r;
}

__device__ __forceinline__ uint16_t f32_to_bf16_rne(float f) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(f));
}

// ---- block-wide exclusive scan of one int per thread (NTH threads, a
// multiple of 32 up to 1024).  `tmp` holds NTH/32 + 1 ints.  Returns the exclusive prefix; *total gets
// the block sum.  Contains __syncthreads.
template <int NTH = kThreads>
__device__ __forceinline__ int block_exclusive_scan(int v, int* tmp, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < NTH / 32 ? tmp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NTH / 32) tmp[lane] = w;   // inclusive warp prefix
        if (lane == NTH / 32 - 1) tmp[NTH / 32] = w;
    }
    __syncthreads();
    const int before = warp > 0 ? tmp[warp - 1] : 0;
    *total = tmp[NTH / 32];
    const int r = before + x - v;
    __syncthreads();
    return r;
}

// ---- the arguments of one mode update (Alg. 1 on mode `mode`).
struct ModeArgs {
    // other modes' factors as gathered (float32 or bfloat16), in increasing
    // mode order with `mode` left out; row stride rp elements
    const void* other[kMaxOrder - 1];
    int n_other;
    int nhot;                 // storage rows 0..nhot-1 of every other mode are its most frequent rows
    int rank;        // R
    int rp;          // padded row length (8, 16, 32, 64)
    float lambda;
    double lambda_d;
    int power_iters;
    // updated mode
    float* U;                 // float32 master A_l, [I][rp] in storage-row order
    const int32_t* inv_self;  // original row -> storage row of the updated mode
    uint16_t* Ub;             // bfloat16 copy (or null)
    float* Y;                 // extrapolation buffer Y_l (null when MAX_INNER = 1)
    int read_y;               // 1: gradient point Y_l read from Y, 0: from U (l = 0)
    int write_y;              // 1: store Y_{l+1}
    const int64_t* row_ptr;   // bucket row pointers of `mode`
    const void* bucket;       // Entry<EW>[nnz]
    SampleStream ss;
    // light rows
    const int32_t* light_rows;
    const int32_t* light_k;
    // rows of at most 509 observations, one warp each (sample to update)
    const int32_t* tiny_rows;
    const int32_t* tiny_k;
    int n_tiny;
    int tiny_begin, tiny_end;   // the range of tiny_rows one launch takes
    // heavy rows
    const int4* chunks;       // {heavy index, pos_begin, pos_end, cand_off}
    const int4* chunk_caps;   // {cand_cap, 0, 0, 0}
    const int4* heavy;        // {row, k, chunk_begin, chunk_end}
    const longlong2* heavy_bracket;  // {lo, hi}: key < lo certain, lo <= key < hi candidate
    const int4* heavy_cand;   // {cand_begin, cand_total_cap, extra_off, extra_cap}
    int n_chunks;
    int n_heavy;
    uint32_t* vis;            // visit lists of chunks, indexed by bucket position
    uint32_t* vis_cnt;        // [n_chunks]
    unsigned long long* cand; // (key << 32 | position) candidates
    uint32_t* cand_cnt;       // [n_chunks]
    uint32_t* extra;          // chosen candidates per heavy row
    uint32_t* extra_cnt;      // [n_heavy]
    uint32_t* flags;          // [n_heavy]: 1 = candidate overflow
    float* partial;           // [(n_chunks + n_heavy)][pw]
    const int4* groups;       // reduction groups {heavy row, first item, end item, 0}
    const int2* heavy_groups; // per heavy row {first group, end group}
    int n_groups;
    float* partial2;          // [n_groups][pw]
    float* row_sum;           // [n_light + n_heavy][pw] reduced Gram/data sums: light rows, then split rows
    float* vwarm;             // [rows][rp] (storage order): each row's last power-method vector, or null
    // epoch-permutation sampling variant: slot perm_slot of epoch perm_epoch;
    // split rows' visits are stored from the row's start, chunk c's at vis_off[c]
    int perm;
    int sset;                 // sampling scratch set of this update (0 or 1)
    uint32_t perm_epoch;
    int64_t perm_slot;
    const int32_t* vis_off;
    int n_light;
    unsigned long long* stat_fallback;  // counter of rows that used the exact selector
    unsigned long long* stat_wait;      // tensor-core blocks whose wait timed out: [0] this call, [1] since creation
    long long test_stall_cycles;        // test hook: > 0 makes block 0 of a tensor-core Gram time out
    uint8_t* mask_out;        // sampler-only mode: mask over bucket positions
};

}  // namespace ntc
