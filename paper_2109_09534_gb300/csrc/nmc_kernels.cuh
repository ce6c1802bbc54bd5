// nmc_kernels.cuh -- device side of Algorithm 1 (accelerated stochastic
// gradient for NMC, Sec. II-B) for one mode: per-row sampling, Khatri-Rao row
// gathers, the row Gram/data reductions, the power method for L_p and the
// projected momentum step.  Instantiated from nmc.cu.
#pragma once

#include <type_traits>

#include "ntc_internal.cuh"

namespace ntc {

// ---------------------------------------------------------------------------
// Block radix select.  Items are unique 64-bit composites (key << 32 | bucket
// position), or ~0 for an unused slot.  Returns T such that exactly k items
// satisfy composite <= T (1 <= k <= number of items): the k-th smallest composite, or, when a whole radix bucket
// completes the count early, the largest composite that bucket can hold.
// This is how "the k_p positions with the smallest (key, position)" of the
// sampling rule (Sec. II-B, Alg. 1 line 5) are found without a sort.
// `hist` holds 256 + 8 unsigned ints of shared memory.
template <int NTH = kThreads, class Get>
__device__ unsigned long long block_select_kth(const Get& get, int n, int k, unsigned* hist) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long prefix = 0ull;
    int remaining = k;
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 56 - 8 * pass;
        for (int i = tid; i < 256; i += NTH) hist[i] = 0u;
        __syncthreads();
        for (int j = tid; j < n; j += NTH) {
            const unsigned long long c = get(j);
            // ~0 marks an unused slot; it is larger than every item, so
            // leaving it out cannot change the k-th smallest (k <= items)
            if (c == ~0ull) continue;
            const bool match = pass == 0 || ((c ^ prefix) >> (shift + 8)) == 0ull;
            if (match) atomicAdd(&hist[(c >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (warp == 0) {
            // lane owns bins 8*lane .. 8*lane+7
            unsigned loc[8];
            unsigned s = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                loc[i] = hist[8 * lane + i];
                s += loc[i];
            }
            unsigned inc = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            const unsigned excl = inc - s;
            const bool mine = excl < (unsigned)remaining && (unsigned)remaining <= inc;
            if (mine) {
                unsigned cum = excl;
                for (int i = 0; i < 8; ++i) {
                    if (cum + loc[i] >= (unsigned)remaining) {
                        hist[256] = 8 * lane + i;   // digit
                        hist[257] = cum;            // items below the digit
                        hist[258] = loc[i];         // items with the digit
                        break;
                    }
                    cum += loc[i];
                }
            }
        }
        __syncthreads();
        const unsigned d = hist[256], below = hist[257], cnt = hist[258];
        __syncthreads();
        remaining -= (int)below;
        prefix |= (unsigned long long)d << shift;
        if ((int)cnt == remaining) {
            return shift == 0 ? prefix : (prefix | ((1ull << shift) - 1ull));
        }
    }
    return prefix;
}

// ---------------------------------------------------------------------------
// Single-histogram select for the same problem when a monotone digit of the
// composite spreads the items over kSelBins bins (uniform Philox keys do):
// one histogram pass finds the bin that holds the m-th smallest item; if that
// bin is not taken whole, its few members are ranked exactly.  Loads are
// issued eight per thread before their histogram updates so that items read
// from global memory are not a chain of dependent latencies.  Falls back to
// block_select_kth when the boundary bin holds more than kSelCap items.
//   digit(c) -> bin in [0, kSelBins), non-decreasing in c
//   binmax(b) -> a composite >= every item of bins <= b and < every item of bins > b
// Shared memory: hist kSelPad + 16 unsigned, mem kSelCap composites.
constexpr int kSelBins = 4096;
constexpr int kSelPad = kSelBins + kSelBins / 32;   // one pad word per 32 bins
constexpr int kSelCap = 512;
// bin b lives at b + b / 32, so that the bins a thread owns, read one by one,
// start in a different bank for every lane
__device__ __forceinline__ int sel_slot(unsigned b) { return (int)(b + (b >> 5)); }

template <int NTH = kThreads, class Get, class Digit, class BinMax>
__device__ unsigned long long block_select_digit(const Get& get, int n, int m, const Digit& digit,
                                                 const BinMax& binmax, unsigned* hist,
                                                 unsigned long long* mem, int* scan_tmp) {
    constexpr int PER = kSelBins / NTH;
    static_assert(PER * NTH == kSelBins && kSelPad % 4 == 0, "bins per thread");
    const int tid = threadIdx.x;
    for (int i = tid; i < kSelPad / 4; i += NTH) reinterpret_cast<uint4*>(hist)[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) hist[kSelPad + 3] = 0u;
    __syncthreads();
    for (int base = 0; base < n; base += NTH * 8) {
        unsigned long long c[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int j = base + u * NTH + tid;
            c[u] = j < n ? get(j) : ~0ull;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (c[u] != ~0ull) atomicAdd(&hist[sel_slot(digit(c[u]))], 1u);
    }
    __syncthreads();
    unsigned loc[PER];
    int own = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        loc[i] = hist[sel_slot((unsigned)(tid * PER + i))];
        own += (int)loc[i];
    }
    int total;
    const int excl = block_exclusive_scan<NTH>(own, scan_tmp, &total);
    if (excl < m && m <= excl + own) {
        int cum = excl;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            if (cum < m && m <= cum + (int)loc[i]) {
                hist[kSelPad] = (unsigned)(tid * PER + i);   // bin
                hist[kSelPad + 1] = (unsigned)cum;           // items below the bin
                hist[kSelPad + 2] = loc[i];                  // items in the bin
            }
            cum += (int)loc[i];
        }
    }
    __syncthreads();
    const unsigned b = hist[kSelPad];
    const int below = (int)hist[kSelPad + 1], cnt = (int)hist[kSelPad + 2];
    const int need = m - below;   // 1 <= need <= cnt
    if (need == cnt) return binmax(b);
    if (cnt > kSelCap) {
        __syncthreads();
        return block_select_kth<NTH>(get, n, m, hist);
    }
    for (int base = 0; base < n; base += NTH * 8) {
        unsigned long long c[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int j = base + u * NTH + tid;
            c[u] = j < n ? get(j) : ~0ull;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (c[u] != ~0ull && digit(c[u]) == b) mem[atomicAdd(&hist[kSelPad + 3], 1u)] = c[u];
    }
    __syncthreads();
    unsigned long long* res = reinterpret_cast<unsigned long long*>(hist + kSelPad + 4);   // 8-byte aligned
    for (int t = tid; t < cnt; t += NTH) {
        const unsigned long long ct = mem[t];
        int r = 0;
        for (int u = 0; u < cnt; ++u) r += mem[u] < ct ? 1 : 0;
        if (r == need - 1) *res = ct;
    }
    __syncthreads();
    const unsigned long long T = *res;
    __syncthreads();
    return T;
}

// ---------------------------------------------------------------------------
// 16-byte asynchronous global -> shared copies (cp.async, L1 bypassed).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
// Same, cached in L1 as well: factor rows are re-read often (skewed indices
// make a few rows very hot), and L1 absorbs those repeats.
__device__ __forceinline__ void cp_async16_ca(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------
// Gram / data reduction over the sampled observations of one row (or one
// chunk of a row):
//   G = sum_e k_e k_e^T  (upper triangle),  b = sum_e x_e k_e
// k_e is the Khatri-Rao row of observation e (Hadamard product of the other
// modes' factor rows, Sec. II unfolding with K of Sec. III), so that
// H_{l,p} = G + lambda I (Alg. 1 line 9) and W_l(p,:) = -b (line 6).
//
// Per staged tile of VT visits: bucket entries (other-mode indices and the
// value) and then the other modes' factor rows are copied to shared memory
// with cp.async; a product pass forms each k_e once (and accumulates b), and
// the FMA pass adds k_e k_e^T into 8x8 register tiles (a, b), a <= b, owned by
// NP threads, NG groups of which take interleaved visits.  Iteration t runs
// the FMA pass of tile t and the product pass of tile t+1 while the factor
// rows of tiles t+2, t+3 and the entries of tiles t+4, t+5 are in flight and
// the bucket positions of tile t+6 are loaded into registers.
template <int RP, int EW, bool BF16, int NT = kThreads, int NHOT = 0, int NOR = 0, int RREG = 32, bool PK = false>
struct Gram {
    static constexpr int T = RP / 8;
    static constexpr int NP = T * (T + 1) / 2;
    static constexpr int NG = NT / NP;
    static constexpr int NACT = NG * NP;
    static constexpr int ES = BF16 ? 2 : 4;           // bytes per stored factor element
    static constexpr int ROWB = RP * ES;              // bytes per factor row
    static constexpr int RST = ROWB + 16;             // staged row stride (bank spread)
    static constexpr int CPR = ROWB / 16;             // 16-byte copies per row
    static constexpr int QPV = RP / 4;                // float4 per k row
    static constexpr int KST = RP + 4;                // k-tile row stride (floats)
    static constexpr int NOMAX = EW == 4 ? 3 : 7;     // other modes
    static constexpr int ENTB = EW * 4;               // bytes per bucket entry
    static constexpr int SR = 3;                      // factor-row stages
    static constexpr int SE = 5;                      // entry stages
    static constexpr int NOTYP = EW == 4 ? 2 : 4;     // other modes the tile size is tuned for
    static constexpr int BPV_TYP = SR * NOTYP * RST + SE * ENTB + 2 * KST * 4;
    static constexpr int BPV_MAX = SR * NOMAX * RST + SE * ENTB + 2 * KST * 4;
    static constexpr int VT_BUDGET = (NT >= 256 ? 100000 : 50000) / BPV_TYP;
    static constexpr int VT_MAX = 200000 / BPV_MAX;
    static constexpr int VT0 = VT_BUDGET < VT_MAX ? VT_BUDGET : VT_MAX;
    static constexpr int VT1 = VT0 >= NG ? (VT0 / NG) * NG : VT0;
    static constexpr int VTS = VT1 > NT ? NT : (VT1 < 1 ? 1 : VT1);
    // With NOR > 0 other modes known at compile time, factor rows go straight
    // to registers (RS product slots of four elements per row per thread, about
    // RREG registers) one tile ahead instead of through shared memory.
    static constexpr int RS0 = NOR > 0 ? RREG / (NOR * (BF16 ? 2 : 4)) : 1;
    static constexpr int RSMAX = PK ? 8 : 4;
    static constexpr int RS = RS0 < 1 ? 1 : (RS0 > RSMAX ? RSMAX : RS0);
    static constexpr int VTR = RS * NT / QPV < NT ? RS * NT / QPV : NT;   // visits the row slots hold
    // visits per tile; the packed form takes a whole number of groups so that
    // no warp runs an extra FMA pass before the tile's barrier
    static constexpr int VT = NOR > 0 ? (PK && VTR >= NG ? VTR / NG * NG : VTR) : VTS;
    static constexpr int VPG = (VT + NG - 1) / NG;    // visits per group per tile
    static constexpr int PW = NP * 64 + RP;           // reduced floats: the tiles, then b
    // slot stride of the reduction buffer: odd, so that the column reads of
    // consecutive slots fall in distinct banks
    static constexpr int RSTR = NACT | 1;
    static constexpr int RED_BYTES = (RSTR * 64 + NT * 4) * 4;
    static_assert(NT % QPV == 0, "a thread's product-pass quad must be fixed");

    __host__ __device__ static constexpr size_t pipe_bytes(int no) {
        return (NOR > 0 ? 0 : (size_t)SR * no * VT * RST) + (size_t)SE * VT * ENTB + (size_t)2 * VT * KST * 4;
    }
    // the most frequent NHOT rows of each other mode, resident for the block
    __host__ __device__ static constexpr size_t hot_bytes(int no) { return (size_t)no * NHOT * RST; }
    __host__ __device__ static constexpr size_t region_bytes(int no) {
        return pipe_bytes(no) > (size_t)RED_BYTES ? pipe_bytes(no) : (size_t)RED_BYTES;
    }
    __host__ __device__ static constexpr size_t total_bytes(int no) { return region_bytes(no) + hot_bytes(no); }

    // 8x8 tile; with PK as column pairs for packed FP32 FMA (two round-to-
    // nearest FMAs per instruction, so the sums equal the scalar form)
    std::conditional_t<PK, float2[8][4], float[8][8]> acc;
    float4 bq;       // b partial of this thread's product-pass quad
    int g, pa, pb;
    bool active;

    __device__ __forceinline__ void init() {
        const int tid = threadIdx.x;
        active = tid < NACT;
        g = tid / NP;
        int p = tid % NP;
        pa = 0;
        pb = 0;
        for (int a = 0; a < T; ++a) {
            if (p < T - a) {
                pa = a;
                pb = a + p;
                break;
            }
            p -= T - a;
        }
        bq = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if constexpr (PK) {
                    if (j < 4) acc[i][j] = make_float2(0.f, 0.f);
                } else {
                    acc[i][j] = 0.f;
                }
            }
    }

    __device__ __forceinline__ static float4 load4(const unsigned char* row, int q) {
        if (BF16) return bf16x4_to_f32(*reinterpret_cast<const uint2*>(row + q * 8));
        return *reinterpret_cast<const float4*>(row + q * 16);
    }

    // k rows of tile visits [0, nv) into the k-tile; b += x k.  Rows of the
    // hot set are read from the resident copy.
    __device__ __forceinline__ void product(const unsigned char* rows, const Entry<EW>* ents, float* kt, int nv,
                                            int no, const unsigned char* hot, int nhot) {
        const int q = threadIdx.x % QPV;
        for (int s = threadIdx.x; s < nv * QPV; s += NT) {
            const int v = s / QPV;
            auto row_of = [&](int o) -> const unsigned char* {
                const int idx = ents[v].w[o];
                return (NHOT > 0 && idx < nhot) ? hot + ((size_t)o * NHOT + idx) * RST
                                                : rows + ((size_t)o * VT + v) * RST;
            };
            float4 p = load4(row_of(0), q);
            for (int o = 1; o < no; ++o) {
                const float4 u = load4(row_of(o), q);
                p.x *= u.x;
                p.y *= u.y;
                p.z *= u.z;
                p.w *= u.w;
            }
            *reinterpret_cast<float4*>(kt + v * KST + 4 * q) = p;
            const float x = __int_as_float(ents[v].w[EW - 1]);
            bq.x = fmaf(x, p.x, bq.x);
            bq.y = fmaf(x, p.y, bq.y);
            bq.z = fmaf(x, p.z, bq.z);
            bq.w = fmaf(x, p.w, bq.w);
        }
    }

    using RowT = typename std::conditional<BF16, uint2, float4>::type;   // 4 factor elements
    __device__ __forceinline__ static float4 to_f4(const float4& v) { return v; }
    __device__ __forceinline__ static float4 to_f4(const uint2& v) { return bf16x4_to_f32(v); }

    // Register path: this thread's RS product slots of a tile -- the four
    // factor elements of each other mode's row -- loaded through L1.
    __device__ __forceinline__ void load_rows_reg(const ModeArgs& a, const Entry<EW>* ents, int nv,
                                                  RowT (&rb)[RS][NOR > 0 ? NOR : 1]) {
#pragma unroll
        for (int j = 0; j < RS; ++j) {
            const int s = threadIdx.x + j * NT;
            if (s < nv * QPV) {
                const int v = s / QPV, q = s % QPV;
#pragma unroll
                for (int o = 0; o < NOR; ++o) {
                    const unsigned char* src = static_cast<const unsigned char*>(a.other[o]) +
                                               (size_t)ents[v].w[o] * ROWB + q * (int)sizeof(RowT);
                    rb[j][o] = __ldg(reinterpret_cast<const RowT*>(src));
                }
            }
        }
    }

    __device__ __forceinline__ void product_reg(const Entry<EW>* ents, float* kt, int nv,
                                                const RowT (&rb)[RS][NOR > 0 ? NOR : 1]) {
#pragma unroll
        for (int j = 0; j < RS; ++j) {
            const int s = threadIdx.x + j * NT;
            if (s < nv * QPV) {
                const int v = s / QPV, q = s % QPV;
                float4 p = to_f4(rb[j][0]);
#pragma unroll
                for (int o = 1; o < NOR; ++o) {
                    const float4 u = to_f4(rb[j][o]);
                    p.x *= u.x;
                    p.y *= u.y;
                    p.z *= u.z;
                    p.w *= u.w;
                }
                *reinterpret_cast<float4*>(kt + v * KST + 4 * q) = p;
                const float x = __int_as_float(ents[v].w[EW - 1]);
                bq.x = fmaf(x, p.x, bq.x);
                bq.y = fmaf(x, p.y, bq.y);
                bq.z = fmaf(x, p.z, bq.z);
                bq.w = fmaf(x, p.w, bq.w);
            }
        }
    }

    __device__ __forceinline__ void accumulate(const float* kt, int nv) {
        if (!active) return;
#pragma unroll
        for (int j = 0; j < VPG; ++j) {
            const int v = g + j * NG;
            if (v >= nv) break;
            const float* kv = kt + v * KST;
            const float4 a0 = *reinterpret_cast<const float4*>(kv + 8 * pa);
            const float4 a1 = *reinterpret_cast<const float4*>(kv + 8 * pa + 4);
            const float4 b0 = *reinterpret_cast<const float4*>(kv + 8 * pb);
            const float4 b1 = *reinterpret_cast<const float4*>(kv + 8 * pb + 4);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            if constexpr (PK) {
                const float2 bv[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w), make_float2(b1.x, b1.y),
                                      make_float2(b1.z, b1.w)};
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float2 ai = make_float2(av[i], av[i]);
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) acc[i][jj] = __ffma2_rn(ai, bv[jj], acc[i][jj]);
                }
            } else {
                const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) acc[i][jj] = fmaf(av[i], bv[jj], acc[i][jj]);
            }
        }
    }

    // All nvis visits; getpos(i) is the bucket position of visit i.  `pipe`
    // holds region_bytes(no) bytes of shared memory.
    template <class GetPos>
    __device__ __forceinline__ void run(const ModeArgs& a, const GetPos& getpos, int nvis, unsigned char* pipe) {
        if constexpr (NOR > 0) {
            run_reg(a, getpos, nvis, pipe);
            return;
        }
        const int no = a.n_other;
        const int tid = threadIdx.x;
        unsigned char* hot = pipe + region_bytes(no);                                   // [no][NHOT][RST]
        const int nhot = NHOT > 0 ? min(NHOT, a.nhot) : 0;
        if constexpr (NHOT > 0) {
            for (int i = tid; i < no * nhot * CPR; i += NT) {
                const int c = i % CPR, ro = i / CPR, r = ro % nhot, o = ro / nhot;
                cp_async16_ca(hot + ((size_t)o * NHOT + r) * RST + 16 * c,
                              static_cast<const unsigned char*>(a.other[o]) + (size_t)r * ROWB + 16 * c);
            }
        }
        const size_t stage_rows = (size_t)no * VT * RST;
        unsigned char* rows = pipe;                                                       // [SR][no][VT][RST]
        Entry<EW>* ents = reinterpret_cast<Entry<EW>*>(pipe + SR * stage_rows);          // [SE][VT]
        float* ktile = reinterpret_cast<float*>(pipe + SR * stage_rows + (size_t)SE * VT * ENTB);  // [2][VT][KST]
        const Entry<EW>* bucket = reinterpret_cast<const Entry<EW>*>(a.bucket);
        const int ntiles = (nvis + VT - 1) / VT;
        auto tile_n = [&](int t) { return min(VT, nvis - t * VT); };
        auto pos_of = [&](int t) -> uint32_t {
            return (t < ntiles && tid < tile_n(t)) ? getpos(t * VT + tid) : 0u;
        };
        auto issue_entries = [&](int t, uint32_t pos) {
            if (t < ntiles && tid < tile_n(t)) {
                const unsigned char* src = reinterpret_cast<const unsigned char*>(bucket + pos);
                unsigned char* dst = reinterpret_cast<unsigned char*>(ents + (t % SE) * VT + tid);
#pragma unroll
                for (int c = 0; c < ENTB / 16; ++c) cp_async16(dst + 16 * c, src + 16 * c);
            }
        };
        auto issue_rows = [&](int t) {
            if (t >= ntiles) return;
            const int nv = tile_n(t);
            const Entry<EW>* e = ents + (t % SE) * VT;
            unsigned char* r = rows + (size_t)(t % SR) * stage_rows;
            // copy i = (o * VT + v) * CPR + c; VT and CPR are compile-time constants
            const int total = no * VT * CPR;
            for (int i = tid; i < total; i += NT) {
                const int c = i % CPR;
                const int vo = i / CPR;
                const int v = vo % VT;
                const int o = vo / VT;
                if (v >= nv) continue;
                const int idx = e[v].w[o];
                if (NHOT > 0 && idx < nhot) continue;   // resident
                const unsigned char* src = static_cast<const unsigned char*>(a.other[o]) + (size_t)idx * ROWB + 16 * c;
                cp_async16_ca(r + (size_t)vo * RST + 16 * c, src);
            }
        };
        auto do_product = [&](int t) {
            if (t < ntiles)
                product(rows + (size_t)(t % SR) * stage_rows, ents + (t % SE) * VT, ktile + (t & 1) * VT * KST,
                        tile_n(t), no, hot, nhot);
        };
        // prologue: k-tile 0 formed; rows 1, 2 and entries 3, 4 in flight;
        // the position of tile 5 in a register
        issue_entries(0, pos_of(0));
        issue_entries(1, pos_of(1));
        issue_entries(2, pos_of(2));
        cp_async_commit();
        uint32_t p3 = pos_of(3), p4 = pos_of(4);
        cp_async_wait<0>();
        __syncthreads();
        issue_rows(0);
        issue_rows(1);
        issue_entries(3, p3);
        cp_async_commit();
        issue_rows(2);
        issue_entries(4, p4);
        cp_async_commit();
        uint32_t pos_next = pos_of(5);
        cp_async_wait<1>();
        __syncthreads();
        do_product(0);
        for (int t = 0; t < ntiles; ++t) {
            cp_async_wait<1>();      // rows of t+1, entries of t+3
            __syncthreads();
            do_product(t + 1);
            issue_rows(t + 3);
            issue_entries(t + 5, pos_next);
            pos_next = pos_of(t + 6);
            cp_async_commit();
            accumulate(ktile + (t & 1) * VT * KST, tile_n(t));
            __syncthreads();
        }
        cp_async_wait<0>();
        __syncthreads();
    }

    // Register-path pipeline: iteration t forms the k-tile of t+1 from the rows
    // in registers, loads the rows of t+2 into them, copies the entries of t+4
    // and accumulates tile t.
    template <class GetPos>
    __device__ __forceinline__ void run_reg(const ModeArgs& a, const GetPos& getpos, int nvis, unsigned char* pipe) {
        const int tid = threadIdx.x;
        Entry<EW>* ents = reinterpret_cast<Entry<EW>*>(pipe);                          // [SE][VT]
        float* ktile = reinterpret_cast<float*>(pipe + (size_t)SE * VT * ENTB);        // [2][VT][KST]
        const Entry<EW>* bucket = reinterpret_cast<const Entry<EW>*>(a.bucket);
        const int ntiles = (nvis + VT - 1) / VT;
        auto tile_n = [&](int t) { return min(VT, nvis - t * VT); };
        auto pos_of = [&](int t) -> uint32_t {
            return (t < ntiles && tid < tile_n(t)) ? getpos(t * VT + tid) : 0u;
        };
        auto issue_entries = [&](int t, uint32_t pos) {
            if (t < ntiles && tid < tile_n(t)) {
                const unsigned char* src = reinterpret_cast<const unsigned char*>(bucket + pos);
                unsigned char* dst = reinterpret_cast<unsigned char*>(ents + (t % SE) * VT + tid);
#pragma unroll
                for (int c = 0; c < ENTB / 16; ++c) cp_async16(dst + 16 * c, src + 16 * c);
            }
        };
        RowT rb[RS][NOR > 0 ? NOR : 1];
        issue_entries(0, pos_of(0));
        issue_entries(1, pos_of(1));
        issue_entries(2, pos_of(2));
        cp_async_commit();
        const uint32_t p3 = pos_of(3);
        cp_async_wait<0>();
        __syncthreads();
        if (ntiles > 0) {
            load_rows_reg(a, ents, tile_n(0), rb);
            product_reg(ents, ktile, tile_n(0), rb);
        }
        if (ntiles > 1) load_rows_reg(a, ents + VT, tile_n(1), rb);
        issue_entries(3, p3);
        cp_async_commit();
        uint32_t pos_next = pos_of(4);
        for (int t = 0; t < ntiles; ++t) {
            cp_async_wait<1>();      // entries of t+2
            __syncthreads();
            if (t + 1 < ntiles) product_reg(ents + ((t + 1) % SE) * VT, ktile + ((t + 1) & 1) * VT * KST,
                                            tile_n(t + 1), rb);
            if (t + 2 < ntiles) load_rows_reg(a, ents + ((t + 2) % SE) * VT, tile_n(t + 2), rb);
            issue_entries(t + 4, pos_next);
            pos_next = pos_of(t + 5);
            cp_async_commit();
            accumulate(ktile + (t & 1) * VT * KST, tile_n(t));
            __syncthreads();
        }
        cp_async_wait<0>();
        __syncthreads();
    }

    // Fixed-order reduction over the NG groups (tiles) and over the threads of
    // each product quad (b) into sum[PW] (shared); `red` may alias `pipe`.
    // The buffer is slot-major (red[slot * RSTR + thread]) so that a warp's
    // stores fall in consecutive banks.
    __device__ __forceinline__ void reduce(float* red, float* sum) {
        if (active) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float v;
                    if constexpr (PK) v = (j & 1) ? acc[i][j >> 1].y : acc[i][j >> 1].x;
                    else v = acc[i][j];
                    red[(i * 8 + j) * RSTR + threadIdx.x] = v;
                }
        }
        reinterpret_cast<float4*>(red + RSTR * 64)[threadIdx.x] = bq;   // 16-byte aligned: RSTR * 64 % 4 == 0
        __syncthreads();
        for (int s = threadIdx.x; s < NP * 64; s += NT) {
            const int p = s >> 6, ij = s & 63;
            const float* col = red + ij * RSTR + p;
            float t = 0.f;
            for (int gg = 0; gg < NG; ++gg) t += col[gg * NP];
            sum[s] = t;
        }
        for (int r = threadIdx.x; r < RP; r += NT) {
            const int q = r / 4, c = r % 4;
            float t = 0.f;
            for (int th = q; th < NT; th += QPV) t += red[RSTR * 64 + th * 4 + c];
            sum[NP * 64 + r] = t;
        }
        __syncthreads();
    }
};

// Pair index -> (a, b), a <= b, row-major over the upper triangle of T x T blocks.
__device__ __forceinline__ void pair_ab(int T, int p, int* a, int* b) {
    for (int i = 0; i < T; ++i) {
        if (p < T - i) {
            *a = i;
            *b = i + p;
            return;
        }
        p -= T - i;
    }
    *a = 0;
    *b = 0;
}

// Alg. 1 lines 8 and 10-13 for row p, run by one warp: gradient H y - b
// (= W + Z + lambda y), L_p by the power method (v0 = ones/sqrt(R), fixed
// iteration count, Rayleigh quotient), projected step, momentum, extrapolation.
// matvec(x, out) gives this lane's entries (r = lane + 32 t) of H x for x in
// shared memory (RP floats, 16-byte aligned); H is zero outside the leading
// R x R block, so loops run over RP.
template <int RP, class MatVec>
__device__ __forceinline__ void finish_row_mv(const ModeArgs& a, int p, const float* bvec, float* vsh, int lane,
                                              const MatVec& matvec) {
    constexpr int PER = RP > 32 ? RP / 32 : 1;
    const int R = a.rank;
    const size_t base = (size_t)a.inv_self[p] * RP;
    float y[PER], al[PER], grad[PER], v[PER], w[PER];
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        const int r = lane + 32 * t;
        const bool in = r < R;
        al[t] = in ? a.U[base + r] : 0.f;
        y[t] = in ? (a.read_y ? a.Y[base + r] : al[t]) : 0.f;
        v[t] = in ? (a.vwarm ? a.vwarm[base + r] : 1.0f / sqrtf((float)R)) : 0.f;
    }
    // gradient: (H y)_r - b_r
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        const int r = lane + 32 * t;
        if (r < RP) vsh[r] = y[t];
    }
    __syncwarp();
    matvec(vsh, grad);
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        const int r = lane + 32 * t;
        grad[t] = r < R ? grad[t] - bvec[r] : 0.f;
    }
    __syncwarp();
    // power method
    float mu = 0.f;
    for (int it = 0; it < a.power_iters; ++it) {
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int r = lane + 32 * t;
            if (r < RP) vsh[r] = v[t];
        }
        __syncwarp();
        matvec(vsh, w);
        __syncwarp();
        float vw = 0.f, ww = 0.f;
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            vw = fmaf(v[t], w[t], vw);
            ww = fmaf(w[t], w[t], ww);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vw += __shfl_xor_sync(0xffffffffu, vw, o);
            ww += __shfl_xor_sync(0xffffffffu, ww, o);
        }
        mu = vw;
        if (!(ww > 0.f)) {
            mu = 0.f;
            break;
        }
        const float inv = 1.0f / sqrtf(ww);
#pragma unroll
        for (int t = 0; t < PER; ++t) v[t] = w[t] * inv;
    }
    if (a.vwarm) {   // the next update of this row starts from here
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int r = lane + 32 * t;
            if (r < R) a.vwarm[base + r] = v[t];
        }
    }
    const float L = mu;
    if (!(L > 0.f)) return;   // L_p <= 0: the row is skipped
    const double sl = sqrt((double)L), sm = sqrt(a.lambda_d);
    const float beta = (float)((sl - sm) / (sl + sm));
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        const int r = lane + 32 * t;
        if (r < R) {
            const float anew = fmaxf(y[t] - grad[t] / L, 0.f);
            a.U[base + r] = anew;
            if (a.Ub) a.Ub[base + r] = f32_to_bf16_rne(anew);
            if (a.write_y) a.Y[base + r] = anew + beta * (anew - al[t]);
        }
    }
}

// The same with H = G + lambda I given in shared memory (stride RP + 1).
template <int RP>
__device__ __forceinline__ void finish_row_warp(const ModeArgs& a, int p, const float* H, const float* bvec,
                                                float* vsh, int lane) {
    constexpr int PER = RP > 32 ? RP / 32 : 1;
    // for RP <= 32 lane r keeps row r of H in registers; x is read as float4
    // broadcasts (the sums run over c in the same order either way)
    float hrow[RP <= 32 ? RP : 1];
    if constexpr (RP <= 32) {
#pragma unroll
        for (int c = 0; c < RP; ++c) hrow[c] = lane < RP ? H[lane * (RP + 1) + c] : 0.f;
    }
    auto matvec = [&](const float* x, float* out) {
        if constexpr (RP <= 32) {
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < RP; c += 4) {
                const float4 x4 = *reinterpret_cast<const float4*>(x + c);
                s = fmaf(hrow[c], x4.x, s);
                s = fmaf(hrow[c + 1], x4.y, s);
                s = fmaf(hrow[c + 2], x4.z, s);
                s = fmaf(hrow[c + 3], x4.w, s);
            }
            out[0] = s;
        } else {
#pragma unroll
            for (int t = 0; t < PER; ++t) {
                const int r = lane + 32 * t;
                float s = 0.f;
                if (r < RP) {
                    const float* hr = H + r * (RP + 1);
#pragma unroll
                    for (int c = 0; c < RP; ++c) s = fmaf(hr[c], x[c], s);
                }
                out[t] = s;
            }
        }
    };
    finish_row_mv<RP>(a, p, bvec, vsh, lane, matvec);
}

// H = G + lambda I for one row, built by one warp: the reduced tiles of the
// row (global memory) into the warp's own H (full symmetric, stride RP+1) and b.
template <int RP>
__device__ __forceinline__ void build_H_warp(const float* sum, float* H, float* bvec, int R, float lambda,
                                             int lane) {
    constexpr int T = RP / 8, NP = T * (T + 1) / 2, NS = NP * 64 / 32;
    // every load of the row's sums is issued before the first store
    float v[NS];
#pragma unroll
    for (int u = 0; u < NS; ++u) v[u] = sum[u * 32 + lane];
    float bv[(RP + 31) / 32];
#pragma unroll
    for (int u = 0; u < (RP + 31) / 32; ++u) bv[u] = u * 32 + lane < RP ? sum[NP * 64 + u * 32 + lane] : 0.f;
#pragma unroll
    for (int u = 0; u < NS; ++u) {
        const int s = u * 32 + lane;
        const int p = s >> 6, ij = s & 63, i = ij >> 3, j = ij & 7;
        int a, b;
        pair_ab(T, p, &a, &b);
        const int r = 8 * a + i, c = 8 * b + j;
        if (a == b && i > j) continue;
        H[r * (RP + 1) + c] = v[u];
        H[c * (RP + 1) + r] = v[u];
    }
#pragma unroll
    for (int u = 0; u < (RP + 31) / 32; ++u)
        if (u * 32 + lane < RP) bvec[u * 32 + lane] = bv[u];
    __syncwarp();
    for (int r = lane; r < R; r += 32) H[r * (RP + 1) + r] += lambda;
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Light rows (n_p <= kLightMax): one block per row does everything: keys in
// shared memory, exact k-subset selection, Gram/data reduction, row update.
// Shared memory: [visit list u16 x kLightMax | union(keys, Gram pipeline,
// reduction)] + reduced sums, H, b, vectors, histogram.
// Threads per light-row block: 128, so that 4 blocks (rows) share an SM and a
// block barrier waits for 4 warps.
constexpr int kLightThreads = 128;

template <int RP, int EW, bool BF16, int NOR>
struct LightSmem {
    using G = Gram<RP, EW, BF16, kLightThreads, 0, NOR, 24>;
    static constexpr size_t VIS = kLightMax * 2;
    // keys, then the select's histogram and boundary-bin members
    static constexpr size_t KEYS = kLightMax * 4;
    static constexpr size_t SEL = KEYS + (size_t)(kSelPad + 16) * 4 + (size_t)kSelCap * 8;
    __host__ __device__ static constexpr size_t union_bytes(int no) {
        return G::region_bytes(no) > SEL ? G::region_bytes(no) : SEL;
    }
    static constexpr size_t TAIL = (size_t)(kLightThreads / 32 + 16) * 4;
    __host__ __device__ static constexpr size_t bytes(int no) { return VIS + union_bytes(no) + TAIL; }
};

template <int RP, int EW, bool BF16, int NOR>
__global__ void __launch_bounds__(kLightThreads, 4) k_light(ModeArgs a) {
    constexpr int LT = kLightThreads;
    using G = Gram<RP, EW, BF16, LT, 0, NOR, 24>;
    using S = LightSmem<RP, EW, BF16, NOR>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int no = a.n_other;
    uint16_t* vis = reinterpret_cast<uint16_t*>(smem_raw);
    unsigned char* uni = smem_raw + S::VIS;
    uint32_t* keys = reinterpret_cast<uint32_t*>(uni);
    unsigned* hist = reinterpret_cast<unsigned*>(uni + S::KEYS);
    unsigned long long* mem = reinterpret_cast<unsigned long long*>(hist + kSelPad + 16);
    float* red = reinterpret_cast<float*>(uni);
    int* scan_tmp = reinterpret_cast<int*>(uni + S::union_bytes(no));

    const int row = a.light_rows[blockIdx.x];
    const int k = a.light_k[blockIdx.x];
    const int64_t q0 = a.row_ptr[row];
    const int n = (int)(a.row_ptr[row + 1] - q0);
    const uint32_t uq0 = (uint32_t)q0;

    if (a.perm) {
        // epoch-permutation variant: the slot's stretch of the row's permutation
        const PermGen pg(a.ss.k0, a.ss.k1, a.ss.mode, a.perm_epoch, (uint32_t)row, (uint32_t)n);
        const uint32_t s0 = (uint32_t)((a.perm_slot * k) % n);   // stretch start; s0 + j < 2n
        pg.map_range(s0, threadIdx.x, (uint32_t)k, LT, [&](uint32_t j, uint32_t x) { vis[j] = (uint16_t)x; });
        __syncthreads();
        if (a.mask_out) {
            for (int i = threadIdx.x; i < k; i += LT) a.mask_out[q0 + vis[i]] = 1;
            return;
        }
        G gr;
        gr.init();
        auto getpos = [&](int v) -> uint32_t { return uq0 + vis[v]; };
        gr.run(a, getpos, k, uni);
        gr.reduce(red, a.row_sum + (size_t)blockIdx.x * G::PW);
        return;
    }
    // the row's bucket entries (contiguous, 16-byte aligned, a multiple of 16
    // bytes) start toward L2 now, so that the Gram's sampled entry reads after
    // the selection find them there
    if (threadIdx.x == 0) {
        const unsigned char* src = static_cast<const unsigned char*>(a.bucket) + (size_t)q0 * (EW * 4);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(src), "r"((uint32_t)n * (EW * 4))
                     : "memory");
    }
    // Alg. 1 line 5: the k smallest (key, position) of the row's n positions
    unsigned long long T = ~0ull;
    if (k < n) {
        // one Philox block per thread gives the keys of 4 consecutive positions
        const KeyGen kg(a.ss);
        const uint32_t g0 = uq0 >> 2, g1 = (uq0 + (uint32_t)n + 3u) >> 2;
        for (uint32_t g = g0 + threadIdx.x; g < g1; g += LT) {
            const uint4 w = kg.key4(g);
            const uint32_t kw[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (uint32_t t = 0; t < 4; ++t) {
                const uint32_t q = 4u * g + t;
                if (q >= uq0 && q - uq0 < (uint32_t)n) keys[q - uq0] = kw[t];
            }
        }
        __syncthreads();
        auto get = [&](int j) -> unsigned long long {
            return ((unsigned long long)keys[j] << 32) | (unsigned long long)(uq0 + j);
        };
        // digit: the top 12 bits of the key
        auto digit = [](unsigned long long c) -> unsigned { return (unsigned)(c >> 52); };
        auto binmax = [](unsigned b) -> unsigned long long {
            return ((unsigned long long)b << 52) | ((1ull << 52) - 1ull);
        };
        T = block_select_digit<LT>(get, n, k, digit, binmax, hist, mem, scan_tmp);
    }
    // compaction in position order: warp w owns positions [w*seg, (w+1)*seg)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int seg = ((n + LT - 1) / LT) * 32;
    const int wb = warp * seg, we = min(n, wb + seg);
    auto chosen = [&](int j) -> bool {
        return j < we && (k == n || ((((unsigned long long)keys[j] << 32) | (uq0 + j)) <= T));
    };
    // one compare pass: the chosen bits of each 32 positions go to a word of
    // the select's histogram (free now), and the writing pass reads them back
    unsigned* cmask = hist;
    int wcnt = 0;
    for (int j0 = wb; j0 < we; j0 += 32) {
        const unsigned mk = __ballot_sync(0xffffffffu, chosen(j0 + lane));
        if (lane == 0) cmask[j0 >> 5] = mk;
        wcnt += __popc(mk);
    }
    if (lane == 0) scan_tmp[warp] = wcnt;
    __syncthreads();
    int off = 0, nsel = 0;
    for (int w = 0; w < LT / 32; ++w) {
        const int c = scan_tmp[w];
        off += w < warp ? c : 0;
        nsel += c;
    }
    for (int j0 = wb; j0 < we; j0 += 32) {
        const unsigned mk = cmask[j0 >> 5];
        if ((mk >> lane) & 1u) vis[off + __popc(mk & ((1u << lane) - 1u))] = (uint16_t)(j0 + lane);
        off += __popc(mk);
    }
    __syncthreads();
    if (a.mask_out) {
        for (int i = threadIdx.x; i < nsel; i += LT) a.mask_out[q0 + vis[i]] = 1;
        return;
    }
    G gr;
    gr.init();
    auto getpos = [&](int v) -> uint32_t { return uq0 + vis[v]; };
    gr.run(a, getpos, nsel, uni);
    gr.reduce(red, a.row_sum + (size_t)blockIdx.x * G::PW);
}

// Row update of every sampled row (Alg. 1 lines 8, 10-13): one warp per row
// builds H = G + lambda I from the row's reduced sums -- light rows first,
// then split rows -- and runs the power method and the projected momentum
// step, so that the serial part does not hold a whole block.
template <int RP>
struct RowFinish {
    static constexpr int WARPS = RP > 32 ? 4 : 8;
    static constexpr int PERW = RP * (RP + 1) + 2 * RP;   // floats of H, b and v per warp
    static constexpr size_t bytes() { return (size_t)WARPS * PERW * 4; }
};

template <int RP>
__global__ void __launch_bounds__(RowFinish<RP>::WARPS * 32) k_rows_finish(ModeArgs a) {
    using RF = RowFinish<RP>;
    constexpr int T = RP / 8, PW = T * (T + 1) / 2 * 64 + RP;
    extern __shared__ __align__(16) float rf_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * RF::WARPS + warp;
    if (i >= a.n_light + a.n_heavy) return;
    const int row = i < a.n_light ? a.light_rows[i] : a.heavy[i - a.n_light].x;
    float* H = rf_smem + warp * RF::PERW;
    float* bvec = H + RP * (RP + 1);
    float* vsh = bvec + RP;
    build_H_warp<RP>(a.row_sum + (size_t)i * PW, H, bvec, a.rank, a.lambda, lane);
    finish_row_warp<RP>(a, row, H, bvec, vsh, lane);
}

// ---------------------------------------------------------------------------
// Heavy rows, step 1: per chunk of a row, keys of every position; positions
// with key < lo are certainly in the sample and are written, in position
// order; lo <= key < hi are candidates whose fate depends on the whole row.
// Each thread takes 16 consecutive positions per round, the keys of four
// Philox blocks, so one block scan serves 4096 positions (measured with one
// block per key: 8 positions per thread 7.6, 16 per thread 7.1 ms per epoch on
// the Zipf(1.1) 10^4-cube).
constexpr int kSamplePer = 16;   // positions per thread per round of the split-row sampler
constexpr int kResolvePer = 8;   // candidates per thread per round of the resolver's compaction

// Keys of chunk `ch`: certain positions to a.vis[pb ...] in position order,
// candidates to the chunk's candidate slots; returns the certain count (the
// same in every thread).  Rounds start at pb rounded down to a multiple of 4,
// so that a thread's 16 positions are four whole Philox blocks.
__device__ __forceinline__ int sample_chunk(const ModeArgs& a, int ch, int* scan_tmp) {
    static_assert(kSamplePer == 16, "whole Philox blocks per thread, 16-bit position masks");
    const int4 c = a.chunks[ch];
    const int h = c.x;
    const uint32_t pb = (uint32_t)c.y, pe = (uint32_t)c.z;
    const int cand_off = c.w;
    const int cap = a.chunk_caps[ch].x;
    const longlong2 br = a.heavy_bracket[h];
    // 32-bit form of key < lo and key < hi (the bounds may equal 2^32)
    const bool lo_all = br.x > 0xFFFFFFFFll, hi_all = br.y > 0xFFFFFFFFll;
    const uint32_t lo = lo_all ? 0u : (uint32_t)br.x, hi = hi_all ? 0u : (uint32_t)br.y;
    const KeyGen kg(a.ss);
    int nsel = 0, ncand = 0;
    for (uint32_t base = pb & ~3u; base < pe; base += kThreads * kSamplePer) {
        const uint32_t q0 = base + threadIdx.x * kSamplePer;
        // bits of this thread's positions inside the chunk: only the first and
        // the last round of a chunk hold positions outside it
        unsigned vm = 0xFFFFu;
        if (base < pb || base + kThreads * kSamplePer > pe) {
            const unsigned jl = q0 >= pb ? 0u : min(pb - q0, 16u), jh = q0 >= pe ? 0u : min(pe - q0, 16u);
            vm = jh > jl ? (((1u << jh) - 1u) & ~((1u << jl) - 1u)) : 0u;
        }
        // bit j of dm / cm: position q0 + j is certain / a candidate
        uint32_t kv[kSamplePer];
        unsigned dm = 0u, cm = 0u;
        if (lo_all) {
            // k = n: every position, no keys
#pragma unroll
            for (int j = 0; j < kSamplePer; ++j) kv[j] = 0u;
            dm = vm;
        } else {
#pragma unroll
            for (int b = 0; b < kSamplePer / 4; ++b) {
                uint4 w = make_uint4(0u, 0u, 0u, 0u);
                if (q0 + 4u * b < pe) w = kg.key4((q0 >> 2) + b);
                kv[4 * b] = w.x;
                kv[4 * b + 1] = w.y;
                kv[4 * b + 2] = w.z;
                kv[4 * b + 3] = w.w;
            }
            // one compare and one conditional bit set per key and bound
#pragma unroll
            for (int j = 0; j < kSamplePer; ++j) {
                dm = kv[j] < lo ? dm | (1u << j) : dm;
                cm = kv[j] < hi ? cm | (1u << j) : cm;
            }
            if (hi_all) cm = 0xFFFFu;
            dm &= vm;
            cm &= vm & ~dm;
        }
        int tot;
        const int packed = block_exclusive_scan(__popc(dm) | (__popc(cm) << 16), scan_tmp, &tot);
        int od = nsel + (packed & 0xFFFF), oc = ncand + (packed >> 16);
        while (dm) {
            const int j = __ffs(dm) - 1;
            dm &= dm - 1u;
            a.vis[pb + od++] = q0 + j;
        }
        if (cm) {   // about one position in thirty
#pragma unroll
            for (int j = 0; j < kSamplePer; ++j) {
                if ((cm >> j) & 1u) {
                    if (oc < cap) a.cand[cand_off + oc] = ((unsigned long long)kv[j] << 32) | (q0 + j);
                    ++oc;
                }
            }
        }
        nsel += tot & 0xFFFF;
        ncand += tot >> 16;
    }
    // unused candidate slots hold a sentinel larger than any composite
    for (int s = ncand + threadIdx.x; s < cap; s += kThreads) a.cand[cand_off + s] = ~0ull;
    if (threadIdx.x == 0) {
        a.vis_cnt[ch] = nsel;
        a.cand_cnt[ch] = min(ncand, cap);
        if (ncand > cap) atomicOr(&a.flags[h], 1u);
    }
    return nsel;
}

// Epoch-permutation variant for split rows: chunk c of a row writes its share
// [k cl / nch, k (cl+1) / nch) of the row's k visits, the slot's stretch of
// the row's permutation, at the row's start (list of chunk c at vis_off[c]).
// (templated on the entry width only so that each translation unit keeps its own copy)
template <int EW>
__global__ void __launch_bounds__(kThreads) k_perm_visits(ModeArgs a) {
    const int c = blockIdx.x;
    const int h = a.chunks[c].x;
    const int4 hv = a.heavy[h];   // {row, k, first chunk, end chunk}
    const int row = hv.x;
    const int64_t k = hv.y, nch = hv.w - hv.z, cl = c - hv.z;
    const int64_t rp = a.row_ptr[row];
    const int64_t n = a.row_ptr[row + 1] - rp;
    const int64_t jb = k * cl / nch, je = k * (cl + 1) / nch;
    const PermGen pg(a.ss.k0, a.ss.k1, a.ss.mode, a.perm_epoch, (uint32_t)row, (uint32_t)n);
    const uint32_t s0 = (uint32_t)((a.perm_slot * k) % n);   // stretch start; s0 + j < 2n < 2^32
    const uint32_t urp = (uint32_t)rp;
    pg.map_range(s0, (uint32_t)jb + threadIdx.x, (uint32_t)je, kThreads,
                 [&](uint32_t j, uint32_t x) { a.vis[rp + j] = urp + x; });
    if (threadIdx.x == 0) {
        a.vis_cnt[c] = (uint32_t)(je - jb);
        if (cl == 0) a.extra_cnt[h] = 0;
    }
}

template <int EW>
__global__ void __launch_bounds__(kThreads) k_heavy_sample(ModeArgs a) {
    __shared__ int scan_tmp[kThreads / 32 + 1];
    sample_chunk(a, blockIdx.x, scan_tmp);
}

// Heavy rows, step 2: per row, the certain count C plus the m = k - C
// smallest candidates give the exact k-subset.  If the bracket missed (too
// few or too many candidates, or overflow), the row is reselected exactly from
// recomputed keys and its chunk lists are rewritten.
template <int EW>
__global__ void __launch_bounds__(kThreads) k_heavy_resolve(ModeArgs a) {
    __shared__ __align__(16) unsigned hist[kSelPad + 16];
    __shared__ unsigned long long mem[kSelCap];
    __shared__ int scan_tmp[kThreads / 32 + 1];
    __shared__ int red_i[2][kThreads / 32];
    const int h = blockIdx.x;
    const int4 hv = a.heavy[h];
    const int row = hv.x, k = hv.y, cb = hv.z, ce = hv.w;
    const int4 hc = a.heavy_cand[h];
    const int cbeg = hc.x, ccap = hc.y, eoff = hc.z;
    // certain and candidate totals over the row's chunks (fixed order)
    long long s_sel = 0, s_cand = 0;
    for (int ch = cb + threadIdx.x; ch < ce; ch += kThreads) {
        s_sel += a.vis_cnt[ch];
        s_cand += a.cand_cnt[ch];
    }
    int vs = (int)s_sel, vc = (int)s_cand;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        vs += __shfl_xor_sync(0xffffffffu, vs, o);
        vc += __shfl_xor_sync(0xffffffffu, vc, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red_i[0][threadIdx.x >> 5] = vs;
        red_i[1][threadIdx.x >> 5] = vc;
    }
    __syncthreads();
    int C = 0, NC = 0;
    for (int i = 0; i < kThreads / 32; ++i) {
        C += red_i[0][i];
        NC += red_i[1][i];
    }
    const int m = k - C;
    const bool overflow = a.flags[h] != 0u;
    if (!overflow && m >= 0 && m <= NC) {
        if (m == 0) {
            if (threadIdx.x == 0) a.extra_cnt[h] = 0;
            return;
        }
        const unsigned long long* cand = a.cand + cbeg;
        auto get = [&](int j) -> unsigned long long { return cand[j]; };
        // every candidate key lies in the bracket [lo, hi): the digit is the
        // key's offset in the bracket scaled to 12 bits (sentinels are skipped)
        const longlong2 br = a.heavy_bracket[h];
        const unsigned long long lo = (unsigned long long)br.x, w = (unsigned long long)br.y - lo;
        const int sh = w <= 1ull ? 0 : max(0, 64 - __clzll((long long)(w - 1ull)) - 12);
        auto digit = [&](unsigned long long c) -> unsigned { return (unsigned)(((c >> 32) - lo) >> sh); };
        auto binmax = [&](unsigned b) -> unsigned long long {
            const unsigned long long kmax = lo + (((unsigned long long)b + 1ull) << sh) - 1ull;
            return kmax >= 0xFFFFFFFFull ? ~0ull : ((kmax << 32) | 0xFFFFFFFFull);
        };
        const unsigned long long T = block_select_digit(get, ccap, m, digit, binmax, hist, mem, scan_tmp);
        int ne = 0;
        for (int base = 0; base < ccap; base += kThreads * kResolvePer) {
            const int j0 = base + threadIdx.x * kResolvePer;
            unsigned long long cv[kResolvePer];
            int nf = 0;
#pragma unroll
            for (int u = 0; u < kResolvePer; ++u) {
                cv[u] = j0 + u < ccap ? cand[j0 + u] : ~0ull;
                nf += (cv[u] != ~0ull && cv[u] <= T) ? 1 : 0;
            }
            int tot;
            int off = ne + block_exclusive_scan(nf, scan_tmp, &tot);
#pragma unroll
            for (int u = 0; u < kResolvePer; ++u)
                if (cv[u] != ~0ull && cv[u] <= T) a.extra[eoff + off++] = (uint32_t)(cv[u] & 0xFFFFFFFFull);
            ne += tot;
        }
        if (threadIdx.x == 0) a.extra_cnt[h] = ne;
        return;
    }
    // exact fallback over the whole row
    if (threadIdx.x == 0 && a.stat_fallback) atomicAdd(a.stat_fallback, 1ull);
    const int64_t q0 = a.row_ptr[row];
    const int n = (int)(a.row_ptr[row + 1] - q0);
    const uint32_t uq0 = (uint32_t)q0;
    const KeyGen kg(a.ss);
    auto getf = [&](int j) -> unsigned long long {
        return ((unsigned long long)kg.key(uq0 + j) << 32) | (unsigned long long)(uq0 + j);
    };
    const unsigned long long T = block_select_kth(getf, n, k, hist);
    for (int ch = cb; ch < ce; ++ch) {
        const int4 c = a.chunks[ch];
        const uint32_t pb = (uint32_t)c.y, pe = (uint32_t)c.z;
        int nsel = 0;
        for (uint32_t base = pb; base < pe; base += kThreads) {
            const uint32_t q = base + threadIdx.x;
            bool f = false;
            if (q < pe) f = ((((unsigned long long)kg.key(q)) << 32) | q) <= T;
            int tot;
            const int off = block_exclusive_scan(f ? 1 : 0, scan_tmp, &tot);
            if (f) a.vis[pb + nsel + off] = q;
            nsel += tot;
        }
        if (threadIdx.x == 0) a.vis_cnt[ch] = nsel;
    }
    if (threadIdx.x == 0) a.extra_cnt[h] = 0;
}

// Heavy rows, step 3: Gram/data partials of each chunk's certain visits and of
// each row's chosen candidates.
// Split-row Gram block shape per padded rank: threads, blocks per SM for the
// register budget, and packed FP32 FMA.  At R = 32 the packed form needs about
// 150 registers; measured on the Zipf(1.1) 10^4-cube (ms/epoch of this
// kernel): packed 128 threads x 3 blocks 16.3, packed 192 x 2 17.1, scalar
// 256 x 2 18.0, scalar 160 x 3 18.4, scalar 128 x 4 19.2.  Deeper row
// prefetch pays: 5 row slots per thread (40 registers, 154 in all) 15.7,
// 6 slots 16.1, 2 slots with 4 blocks per SM 22.7.
template <int RP>
struct GramNT {
    static constexpr bool packed = RP == 32;
    static constexpr int value = packed ? 128 : 256;
    static constexpr int blocks = packed ? 3 : 2;
    static constexpr int rreg = packed ? 40 : 32;   // registers for factor rows loaded one tile ahead
};
// Resident most-frequent rows per other mode in the split-row Gram.  Off:
// measured on the Zipf(1.1) 10^4-cube, R = 32, the copies it saves cost less
// than the per-visit selection it adds (28.4 vs 32.5 ms/epoch); the L1-cached
// row copies already serve the hot rows.
template <int RP>
struct HotRows {
    static constexpr int value = 0;
};

template <int RP, int EW, bool BF16, int NOR>
struct HeavyGramSmem {
    using G = Gram<RP, EW, BF16, GramNT<RP>::value, HotRows<RP>::value, NOR, GramNT<RP>::rreg, GramNT<RP>::packed>;
    __host__ __device__ static constexpr size_t bytes(int no) { return G::total_bytes(no) + (size_t)G::PW * 4; }
};

template <int RP, int EW, bool BF16, int NOR>
__global__ void __launch_bounds__(GramNT<RP>::value, GramNT<RP>::blocks) k_heavy_gram(ModeArgs a) {
    using G = Gram<RP, EW, BF16, GramNT<RP>::value, HotRows<RP>::value, NOR, GramNT<RP>::rreg, GramNT<RP>::packed>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* pipe = smem_raw;
    float* red = reinterpret_cast<float*>(smem_raw);
    float* sum = reinterpret_cast<float*>(smem_raw + G::total_bytes(a.n_other));
    const int item = blockIdx.x;
    const uint32_t* list;
    int cnt;
    if (item < a.n_chunks) {
        list = a.vis + (a.vis_off ? a.vis_off[item] : a.chunks[item].y);
        cnt = (int)a.vis_cnt[item];
    } else {
        const int h = item - a.n_chunks;
        list = a.extra + a.heavy_cand[h].z;
        cnt = (int)a.extra_cnt[h];
    }
    G gr;
    gr.init();
    auto getpos = [&](int v) -> uint32_t { return list[v]; };
    gr.run(a, getpos, cnt, pipe);
    gr.reduce(red, sum);
    float* out = a.partial + (size_t)item * G::PW;
    for (int s = threadIdx.x; s < G::PW; s += GramNT<RP>::value) out[s] = sum[s];
}

// Heavy rows, step 4a: a row's items (its chunks in order, then its chosen
// candidates) are summed in fixed groups of kReduceGroup consecutive items,
// one block per group, so that long rows are not summed by a single block.

template <int RP>
__global__ void __launch_bounds__(kThreads) k_heavy_reduce(ModeArgs a) {
    constexpr int T = RP / 8, NP = T * (T + 1) / 2, PW = NP * 64 + RP;
    const int4 gr = a.groups[blockIdx.x];   // {heavy row, first item, end item, 0}
    const int h = gr.x;
    const int4 hv = a.heavy[h];
    const int nitems = hv.w - hv.z + 1;
    // a row with a single group has its final sum here
    const int2 gg = a.heavy_groups[h];
    float* out = gg.y - gg.x == 1 ? a.row_sum + (size_t)(a.n_light + h) * PW : a.partial2 + (size_t)blockIdx.x * PW;
    for (int s = threadIdx.x; s < PW; s += kThreads) {
        float v[kReduceGroup];
#pragma unroll
        for (int u = 0; u < kReduceGroup; ++u) {
            const int i = gr.y + u;
            const int it = i < nitems - 1 ? hv.z + i : a.n_chunks + h;
            v[u] = i < gr.z ? a.partial[(size_t)it * PW + s] : 0.f;
        }
        float t = 0.f;
#pragma unroll
        for (int u = 0; u < kReduceGroup; ++u) t += v[u];
        out[s] = t;
    }
}

// Heavy rows, step 4b: fixed-order sum of the row's group sums into the row's
// slot of the reduced-sum buffer (the update itself is k_rows_finish).
template <int RP>
__global__ void __launch_bounds__(kThreads) k_heavy_rowsum(ModeArgs a) {
    constexpr int T = RP / 8, NP = T * (T + 1) / 2, PW = NP * 64 + RP;
    const int h = blockIdx.x;
    const int2 gg = a.heavy_groups[h];   // {first group, end group}
    if (gg.y - gg.x == 1) return;        // written by k_heavy_reduce
    float* out = a.row_sum + (size_t)(a.n_light + h) * PW;
    for (int s = threadIdx.x; s < PW; s += kThreads) {
        float t = 0.f;
        int g = gg.x;
        for (; g + 8 <= gg.y; g += 8) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = a.partial2[(size_t)(g + u) * PW + s];
#pragma unroll
            for (int u = 0; u < 8; ++u) t += v[u];
        }
        for (; g < gg.y; ++g) t += a.partial2[(size_t)g * PW + s];
        out[s] = t;
    }
}

// Sampler-only mode for heavy rows: mark the chosen positions.
template <int EW>
__global__ void k_heavy_mask(ModeArgs a) {
    const int item = blockIdx.x;
    const uint32_t* list;
    int cnt;
    if (item < a.n_chunks) {
        list = a.vis + (a.vis_off ? a.vis_off[item] : a.chunks[item].y);
        cnt = (int)a.vis_cnt[item];
    } else {
        const int h = item - a.n_chunks;
        list = a.extra + a.heavy_cand[h].z;
        cnt = (int)a.extra_cnt[h];
    }
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) a.mask_out[list[i]] = 1;
}


}  // namespace ntc
