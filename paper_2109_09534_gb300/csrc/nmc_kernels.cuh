// nmc_kernels.cuh -- device side of Algorithm 1 (accelerated stochastic
// gradient for NMC, Sec. II-B) for one mode: per-row sampling, Khatri-Rao row
// gathers, the row Gram/data reductions, the power method for L_p and the
// projected momentum step.  Instantiated from nmc.cu.
#pragma once

#include "ntc_internal.cuh"

namespace ntc {

// ---------------------------------------------------------------------------
// Block radix select.  Items are unique 64-bit composites (key << 32 | bucket
// position).  Returns T such that exactly k items satisfy composite <= T
// (1 <= k <= n): the k-th smallest composite, or, when a whole radix bucket
// completes the count early, the largest composite that bucket can hold.
// This is how "the k_p positions with the smallest (key, position)" of the
// sampling rule (Sec. II-B, Alg. 1 line 5) are found without a sort.
// `hist` holds 256 + 8 unsigned ints of shared memory.
template <class Get>
__device__ unsigned long long block_select_kth(const Get& get, int n, int k, unsigned* hist) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long prefix = 0ull;
    int remaining = k;
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 56 - 8 * pass;
        for (int i = tid; i < 256; i += kThreads) hist[i] = 0u;
        __syncthreads();
        for (int j = tid; j < n; j += kThreads) {
            const unsigned long long c = get(j);
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
// Gram / data reduction over a list of sampled observations of one row:
//   G = sum_e k_e k_e^T  (upper triangle),  b = sum_e x_e k_e
// k_e is the Khatri-Rao row of observation e (Hadamard product of the other
// modes' factor rows, Sec. II unfolding with K of Sec. III), so that
// H_{l,p} = G + lambda I (Alg. 1 line 9) and W_l(p,:) = -b (line 6).
// Threads own 8x8 tiles (a, b), a <= b, of G; NG groups of NP threads take
// interleaved visits of each staged tile of VT gathered rows.
template <int RP, int EW, bool BF16>
struct Gram {
    static constexpr int T = RP / 8;
    static constexpr int NP = T * (T + 1) / 2;
    static constexpr int NG = kThreads / NP;
    static constexpr int NACT = NG * NP;
    static constexpr int VPG = (96 + NG - 1) / NG;
    static constexpr int VT = NG * VPG;           // visits per staged tile
    static constexpr int QPV = RP / 4;            // float4 per k row
    static constexpr int KST = RP + 4;            // staged row stride (floats)
    static constexpr int PW = NP * 72;            // reduced floats: 64 tile + 8 of b per pair
    // shared memory (floats)
    static constexpr int SM_TILE = VT * KST + VT;
    static constexpr int SM_RED = NACT * 72;
    static constexpr int SM_SUM = PW;

    float acc[8][8];
    float bacc[8];
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
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            bacc[i] = 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
        }
    }

    // Gather the Khatri-Rao rows of visits [v0, v0 + nv) into the staged tile.
    template <class GetPos>
    __device__ __forceinline__ void gather(const ModeArgs& a, const GetPos& getpos, int v0, int nv,
                                           float* tile) {
        const Entry<EW>* bucket = reinterpret_cast<const Entry<EW>*>(a.bucket);
        float* xt = tile + VT * KST;
        for (int s = threadIdx.x; s < nv * QPV; s += kThreads) {
            const int v = s / QPV, qd = s - v * QPV;
            const uint32_t pos = getpos(v0 + v);
            const Entry<EW> e = bucket[pos];
            float4 prod = make_float4(1.f, 1.f, 1.f, 1.f);
            for (int o = 0; o < a.n_other; ++o) {
                const size_t off = (size_t)e.w[o] * RP + 4 * qd;
                float4 u;
                if (BF16) {
                    const uint2 raw = *reinterpret_cast<const uint2*>(
                        static_cast<const uint16_t*>(a.other[o]) + off);
                    u = bf16x4_to_f32(raw);
                } else {
                    u = *reinterpret_cast<const float4*>(static_cast<const float*>(a.other[o]) + off);
                }
                prod.x *= u.x;
                prod.y *= u.y;
                prod.z *= u.z;
                prod.w *= u.w;
            }
            *reinterpret_cast<float4*>(tile + v * KST + 4 * qd) = prod;
            if (qd == 0) xt[v] = __int_as_float(e.w[EW - 1]);
        }
    }

    __device__ __forceinline__ void accumulate(const float* tile, int nv) {
        if (!active) return;
        const float* xt = tile + VT * KST;
        for (int v = g; v < nv; v += NG) {
            const float* kv = tile + v * KST;
            const float4 a0 = *reinterpret_cast<const float4*>(kv + 8 * pa);
            const float4 a1 = *reinterpret_cast<const float4*>(kv + 8 * pa + 4);
            const float4 b0 = *reinterpret_cast<const float4*>(kv + 8 * pb);
            const float4 b1 = *reinterpret_cast<const float4*>(kv + 8 * pb + 4);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
            if (pa == pb) {
                const float x = xt[v];
#pragma unroll
                for (int i = 0; i < 8; ++i) bacc[i] = fmaf(x, av[i], bacc[i]);
            }
        }
    }

    // Whole list: staged tiles of VT visits.
    template <class GetPos>
    __device__ __forceinline__ void run(const ModeArgs& a, const GetPos& getpos, int nvis, float* tile) {
        for (int v0 = 0; v0 < nvis; v0 += VT) {
            const int nv = min(VT, nvis - v0);
            gather(a, getpos, v0, nv, tile);
            __syncthreads();
            accumulate(tile, nv);
            __syncthreads();
        }
    }

    // Fixed-order reduction over the NG groups into sum[PW] (shared).
    __device__ __forceinline__ void reduce(float* red, float* sum) {
        if (active) {
            float* r = red + (size_t)threadIdx.x * 72;
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) r[i * 8 + j] = acc[i][j];
#pragma unroll
            for (int i = 0; i < 8; ++i) r[64 + i] = bacc[i];
        }
        __syncthreads();
        for (int s = threadIdx.x; s < PW; s += kThreads) {
            float t = 0.f;
            for (int gg = 0; gg < NG; ++gg) t += red[(size_t)gg * PW + s];
            sum[s] = t;
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

// Expand the reduced tiles into H = G + lambda I (full symmetric, stride RP+1)
// and b (Alg. 1 lines 6 and 9).
template <int RP>
__device__ __forceinline__ void build_H(const float* sum, float* H, float* bvec, int R, float lambda) {
    constexpr int T = RP / 8, NP = T * (T + 1) / 2;
    for (int s = threadIdx.x; s < NP * 64; s += kThreads) {
        const int p = s >> 6, ij = s & 63, i = ij >> 3, j = ij & 7;
        int a, b;
        pair_ab(T, p, &a, &b);
        const int r = 8 * a + i, c = 8 * b + j;
        if (a == b && i > j) continue;
        const float v = sum[p * 72 + ij];
        H[r * (RP + 1) + c] = v;
        H[c * (RP + 1) + r] = v;
    }
    for (int s = threadIdx.x; s < NP * 8; s += kThreads) {
        const int p = s >> 3, i = s & 7;
        int a, b;
        pair_ab(T, p, &a, &b);
        if (a == b) bvec[8 * a + i] = sum[p * 72 + 64 + i];
    }
    __syncthreads();
    if (threadIdx.x < R) H[threadIdx.x * (RP + 1) + threadIdx.x] += lambda;
    __syncthreads();
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Alg. 1 lines 8 and 10-13 for row p, run by warp 0: gradient H y - b
// (= W + Z + lambda y), L_p by the power method (v0 = ones/sqrt(R), fixed
// iteration count, Rayleigh quotient), projected step, momentum, extrapolation.
template <int RP>
__device__ __forceinline__ void finish_row(const ModeArgs& a, int p, const float* H, const float* bvec,
                                           float* vsh) {
    if (threadIdx.x >= 32) return;
    constexpr int PER = RP > 32 ? RP / 32 : 1;
    const int lane = threadIdx.x;
    const int R = a.rank;
    const size_t base = (size_t)p * RP;
    float y[PER], al[PER], grad[PER], v[PER], w[PER];
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        const int r = lane + 32 * t;
        const bool in = r < R;
        al[t] = in ? a.U[base + r] : 0.f;
        y[t] = in ? (a.read_y ? a.Y[base + r] : al[t]) : 0.f;
        v[t] = in ? 1.0f / sqrtf((float)R) : 0.f;
    }
    // gradient: (H y)_r - b_r
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        const int r = lane + 32 * t;
        if (r < RP) vsh[r] = y[t];
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        const int r = lane + 32 * t;
        float s = 0.f;
        if (r < R) {
            for (int c = 0; c < R; ++c) s = fmaf(H[r * (RP + 1) + c], vsh[c], s);
            s -= bvec[r];
        }
        grad[t] = s;
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
        float vw = 0.f, ww = 0.f;
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int r = lane + 32 * t;
            float s = 0.f;
            if (r < R)
                for (int c = 0; c < R; ++c) s = fmaf(H[r * (RP + 1) + c], vsh[c], s);
            w[t] = s;
            vw = fmaf(v[t], s, vw);
            ww = fmaf(s, s, ww);
        }
        __syncwarp();
        vw = warp_sum(vw);
        ww = warp_sum(ww);
        mu = vw;
        if (!(ww > 0.f)) {
            mu = 0.f;
            break;
        }
        const float inv = 1.0f / sqrtf(ww);
#pragma unroll
        for (int t = 0; t < PER; ++t) v[t] = w[t] * inv;
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

// ---------------------------------------------------------------------------
// Light rows (n_p <= kLightMax): one block per row does everything: keys in
// shared memory, exact k-subset selection, Gram/data reduction, row update.
template <int RP, int EW, bool BF16>
struct LightSmem {
    using G = Gram<RP, EW, BF16>;
    // region A: selection (keys + visit list) and gather tile, later the reduction buffer
    static constexpr int A_SEL = kLightMax + kLightMax / 2;   // keys (u32) + visits (u16), in floats
    static constexpr int A_FLOATS = (A_SEL + G::SM_TILE) > G::SM_RED ? (A_SEL + G::SM_TILE) : G::SM_RED;
    static constexpr int B_FLOATS = G::SM_SUM + RP * (RP + 1) + 2 * RP + 8;
    static constexpr int MISC_U32 = 256 + 8 + 16;
    static constexpr size_t BYTES = (size_t)(A_FLOATS + B_FLOATS + MISC_U32) * 4;
};

template <int RP, int EW, bool BF16>
__global__ void __launch_bounds__(kThreads, 2) k_light(ModeArgs a) {
    using G = Gram<RP, EW, BF16>;
    using S = LightSmem<RP, EW, BF16>;
    extern __shared__ __align__(16) float smem[];
    float* regA = smem;
    uint32_t* keys = reinterpret_cast<uint32_t*>(regA);
    uint16_t* vis = reinterpret_cast<uint16_t*>(regA + kLightMax);
    float* tile = regA + S::A_SEL;
    float* red = regA;
    float* sum = smem + S::A_FLOATS;
    float* H = sum + G::SM_SUM;
    float* bvec = H + RP * (RP + 1);
    float* vsh = bvec + RP;
    unsigned* hist = reinterpret_cast<unsigned*>(vsh + RP + 8);
    int* scan_tmp = reinterpret_cast<int*>(hist + 256 + 8);

    const int row = a.light_rows[blockIdx.x];
    const int k = a.light_k[blockIdx.x];
    const int64_t q0 = a.row_ptr[row];
    const int n = (int)(a.row_ptr[row + 1] - q0);
    const uint32_t uq0 = (uint32_t)q0;

    // Alg. 1 line 5: the k smallest (key, position) of the row's n positions
    unsigned long long T = ~0ull;
    if (k < n) {
        for (int j = threadIdx.x; j < n; j += kThreads) keys[j] = a.ss.key(uq0 + j);
        __syncthreads();
        auto get = [&](int j) -> unsigned long long {
            return ((unsigned long long)keys[j] << 32) | (unsigned long long)(uq0 + j);
        };
        T = block_select_kth(get, n, k, hist);
    }
    int nsel = 0;
    for (int base = 0; base < n; base += kThreads) {
        const int j = base + threadIdx.x;
        bool f = false;
        if (j < n) f = k == n || ((((unsigned long long)keys[j] << 32) | (uq0 + j)) <= T);
        int tot;
        const int off = block_exclusive_scan(f ? 1 : 0, scan_tmp, &tot);
        if (f) vis[nsel + off] = (uint16_t)j;
        nsel += tot;
    }
    __syncthreads();
    if (a.mask_out) {
        for (int i = threadIdx.x; i < nsel; i += kThreads) a.mask_out[q0 + vis[i]] = 1;
        return;
    }
    G gr;
    gr.init();
    auto getpos = [&](int v) -> uint32_t { return uq0 + vis[v]; };
    gr.run(a, getpos, nsel, tile);
    gr.reduce(red, sum);
    build_H<RP>(sum, H, bvec, a.rank, a.lambda);
    finish_row<RP>(a, row, H, bvec, vsh);
}

// ---------------------------------------------------------------------------
// Heavy rows, step 1: per chunk of a row, keys of every position; positions
// with key < lo are certainly in the sample (written in position order);
// lo <= key < hi are candidates whose fate depends on the whole row.
__global__ void __launch_bounds__(kThreads) k_heavy_sample(ModeArgs a) {
    __shared__ int scan_tmp[kThreads / 32 + 1];
    const int ch = blockIdx.x;
    const int4 c = a.chunks[ch];
    const int h = c.x;
    const uint32_t pb = (uint32_t)c.y, pe = (uint32_t)c.z;
    const int cand_off = c.w;
    const int cap = a.chunk_caps[ch].x;
    const longlong2 br = a.heavy_bracket[h];
    const unsigned long long lo = (unsigned long long)br.x, hi = (unsigned long long)br.y;
    int nsel = 0, ncand = 0;
    for (uint32_t base = pb; base < pe; base += kThreads) {
        const uint32_t q = base + threadIdx.x;
        bool d = false, cn = false;
        unsigned long long key = 0;
        if (q < pe) {
            key = a.ss.key(q);
            d = key < lo;
            cn = !d && key < hi;
        }
        int tot;
        const int packed = block_exclusive_scan((d ? 1 : 0) | (cn ? 0x10000 : 0), scan_tmp, &tot);
        const int od = packed & 0xFFFF, oc = packed >> 16;
        if (d) a.vis[pb + nsel + od] = q;
        if (cn && ncand + oc < cap) a.cand[cand_off + ncand + oc] = (key << 32) | q;
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
}

// Heavy rows, step 2: per row, the certain count C plus the m = k - C
// smallest candidates give the exact k-subset.  If the bracket missed (too
// few or too many candidates, or overflow), the row is reselected exactly from
// recomputed keys and its chunk lists are rewritten.
__global__ void __launch_bounds__(kThreads) k_heavy_resolve(ModeArgs a) {
    __shared__ unsigned hist[256 + 8];
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
        // sentinels sort after every real composite, so the m-th smallest over
        // the whole region is the m-th smallest real candidate
        const unsigned long long T = block_select_kth(get, ccap, m, hist);
        int ne = 0;
        for (int base = 0; base < ccap; base += kThreads) {
            const int j = base + threadIdx.x;
            const unsigned long long cv = j < ccap ? cand[j] : ~0ull;
            const bool f = cv <= T;
            int tot;
            const int off = block_exclusive_scan(f ? 1 : 0, scan_tmp, &tot);
            if (f) a.extra[eoff + ne + off] = (uint32_t)(cv & 0xFFFFFFFFull);
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
    auto getf = [&](int j) -> unsigned long long {
        return ((unsigned long long)a.ss.key(uq0 + j) << 32) | (unsigned long long)(uq0 + j);
    };
    const unsigned long long T = block_select_kth(getf, n, k, hist);
    for (int ch = cb; ch < ce; ++ch) {
        const int4 c = a.chunks[ch];
        const uint32_t pb = (uint32_t)c.y, pe = (uint32_t)c.z;
        int nsel = 0;
        for (uint32_t base = pb; base < pe; base += kThreads) {
            const uint32_t q = base + threadIdx.x;
            bool f = false;
            if (q < pe) f = ((((unsigned long long)a.ss.key(q)) << 32) | q) <= T;
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
template <int RP, int EW, bool BF16>
__global__ void __launch_bounds__(kThreads, 2) k_heavy_gram(ModeArgs a) {
    using G = Gram<RP, EW, BF16>;
    extern __shared__ __align__(16) float smem[];
    float* tile = smem;
    float* red = smem;
    constexpr int A = G::SM_TILE > G::SM_RED ? G::SM_TILE : G::SM_RED;
    float* sum = smem + A;
    const int item = blockIdx.x;
    const uint32_t* list;
    int cnt;
    if (item < a.n_chunks) {
        list = a.vis + a.chunks[item].y;
        cnt = (int)a.vis_cnt[item];
    } else {
        const int h = item - a.n_chunks;
        list = a.extra + a.heavy_cand[h].z;
        cnt = (int)a.extra_cnt[h];
    }
    G gr;
    gr.init();
    auto getpos = [&](int v) -> uint32_t { return list[v]; };
    gr.run(a, getpos, cnt, tile);
    gr.reduce(red, sum);
    float* out = a.partial + (size_t)item * G::PW;
    for (int s = threadIdx.x; s < G::PW; s += kThreads) out[s] = sum[s];
}

// Heavy rows, step 4: fixed-order sum of a row's partials, then the row update.
template <int RP>
__global__ void __launch_bounds__(kThreads) k_heavy_finish(ModeArgs a) {
    constexpr int T = RP / 8, NP = T * (T + 1) / 2, PW = NP * 72;
    extern __shared__ __align__(16) float smem[];
    float* sum = smem;
    float* H = sum + PW;
    float* bvec = H + RP * (RP + 1);
    float* vsh = bvec + RP;
    const int h = blockIdx.x;
    const int4 hv = a.heavy[h];
    for (int s = threadIdx.x; s < PW; s += kThreads) {
        float t = 0.f;
        for (int ch = hv.z; ch < hv.w; ++ch) t += a.partial[(size_t)ch * PW + s];
        t += a.partial[(size_t)(a.n_chunks + h) * PW + s];
        sum[s] = t;
    }
    __syncthreads();
    build_H<RP>(sum, H, bvec, a.rank, a.lambda);
    finish_row<RP>(a, hv.x, H, bvec, vsh);
}

// Sampler-only mode for heavy rows: mark the chosen positions.
__global__ void k_heavy_mask(ModeArgs a) {
    const int item = blockIdx.x;
    const uint32_t* list;
    int cnt;
    if (item < a.n_chunks) {
        list = a.vis + a.chunks[item].y;
        cnt = (int)a.vis_cnt[item];
    } else {
        const int h = item - a.n_chunks;
        list = a.extra + a.heavy_cand[h].z;
        cnt = (int)a.extra_cnt[h];
    }
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) a.mask_out[list[i]] = 1;
}

template <int RP>
constexpr size_t heavy_finish_smem() {
    return (size_t)((RP / 8) * (RP / 8 + 1) / 2 * 72 + RP * (RP + 1) + 2 * RP + 8) * 4;
}

template <int RP, int EW, bool BF16>
constexpr size_t heavy_gram_smem() {
    using G = Gram<RP, EW, BF16>;
    return (size_t)((G::SM_TILE > G::SM_RED ? G::SM_TILE : G::SM_RED) + G::SM_SUM) * 4;
}

}  // namespace ntc
