// tiny_rows.cuh -- Algorithm 1 for rows with few observations (n_p <= 509),
// one warp per row from the sample to the updated factor row: keys of the
// row's positions in registers, the exact k_p-subset of the sampling rule by a
// byte-wise radix select of the k_p-th key (a 256-bin warp histogram per
// byte), ties taken in position order, the Gram/data sums accumulated in
// registers, then H, the gradient, L_p and the projected momentum step
// (finish_row_warp) on the warp's own H in shared memory; at R_pad = 64 and
// k_p <= 32 the warp keeps the k_p gathered rows K instead and applies H as
// K^T K + lambda I (finish_row_mv).  Rating-shaped
// tensors have hundreds of thousands of such rows per mode (users or items
// with a handful of ratings); a block per row with a 4096-bin histogram select
// and a reduced-sum round trip through global memory cost them far more than
// their few visits.
#pragma once

#include "nmc_kernels.cuh"

namespace ntc {

// KONLY: the launch that takes only rows of at most kTinyKForm visits at
// R_pad = 64, whose area holds the visit list and K instead of H.
template <int RP, bool KONLY = false>
struct TinyShape {
    static constexpr int WARPS = RP > 32 ? 4 : 8;
    static constexpr int RPL = RP > 32 ? 2 : 1;      // H rows owned per lane (rank r = lane + 32 t)
    static constexpr int ND = RP / 2 + 1;            // stored diagonals of each owned row
    static constexpr int KST = RP + 4;               // K row stride (floats)
    // per warp: H (RP x (RP+1); the visit list, 512 u16, lives there until H
    // is written, so the area holds at least 256 floats) or, with KONLY, the
    // visit list then K; b, the power-method vector, k of one visit, and the
    // select's 256-bin histogram
    static constexpr int HA = KONLY ? 256 + kTinyKForm * KST : (RP * (RP + 1) > 256 ? RP * (RP + 1) : 256);
    static constexpr int PERW = HA + 3 * RP + 256;
    static constexpr size_t bytes() { return (size_t)WARPS * PERW * 4; }
};

template <int RP, int EW, bool BF16, int NOR, bool KONLY = false>
__global__ void __launch_bounds__(TinyShape<RP>::WARPS * 32) k_tiny_rows(ModeArgs a) {
    using TS = TinyShape<RP, KONLY>;
    static_assert(!KONLY || RP == 64, "the K-only launch is the rank-64 one");
    static_assert(EW == 4 && NOR >= 1 && NOR <= 3, "orders 2-4");
    extern __shared__ __align__(16) float tiny_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* H = tiny_smem + warp * TS::PERW;
    float* bvec = H + TS::HA;
    float* vsh = bvec + RP;
    float* ksh = vsh + RP;
    unsigned* hist = reinterpret_cast<unsigned*>(ksh + RP);
    uint16_t* vis = reinterpret_cast<uint16_t*>(H);
    const int i = a.tiny_begin + blockIdx.x * TS::WARPS + warp;
    if (i >= a.tiny_end) return;   // the same in every lane of the warp
    const int row = a.tiny_rows[i];
    const int k = a.tiny_k[i];
    const int64_t q0 = a.row_ptr[row];
    const int n = (int)(a.row_ptr[row + 1] - q0);
    const uint32_t uq0 = (uint32_t)q0;

    // ---- Alg. 1 line 5: the k smallest (key, position) of the row's positions
    int nsel = k;
    if (a.perm) {
        // epoch-permutation variant: the slot's stretch of the row's permutation
        const PermGen pg(a.ss.k0, a.ss.k1, a.ss.mode, a.perm_epoch, (uint32_t)row, (uint32_t)n);
        const uint32_t s0 = (uint32_t)((a.perm_slot * k) % n);   // stretch start; s0 + j < 2n
        pg.map_range(s0, lane, (uint32_t)k, 32, [&](uint32_t j, uint32_t x) { vis[j] = (uint16_t)x; });
    } else {
        // lane L: positions a0 + 16 L + j, j < 16 (four Philox blocks), a0 = q0 rounded down to 4
        const uint32_t a0 = uq0 & ~3u;
        const uint32_t qb = a0 + 16u * (uint32_t)lane;
        const KeyGen kg(a.ss);
        uint32_t kv[16];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const uint4 w = kg.key4((qb >> 2) + b);
            kv[4 * b] = w.x;
            kv[4 * b + 1] = w.y;
            kv[4 * b + 2] = w.z;
            kv[4 * b + 3] = w.w;
        }
        unsigned valid = 0u;
#pragma unroll
        for (int j = 0; j < 16; ++j) valid |= (unsigned)(qb + j >= uq0 && qb + j - uq0 < (uint32_t)n) << j;
        unsigned sel = valid;
        if (k < n) {
            // T = the k-th smallest key (the smallest key value with #(key <= T)
            // >= k), one byte per pass from the top: a 256-bin histogram of the
            // keys that match the digits found so far, and the bin where the
            // running count reaches k
            uint32_t prefix = 0u;
            int rem = k;
#pragma unroll 1
            for (int shift = 24; shift >= 0; shift -= 8) {
#pragma unroll
                for (int b = 0; b < 8; ++b) hist[lane * 8 + b] = 0u;
                __syncwarp();
                const uint32_t hmask = shift == 24 ? 0u : (0xFFFFFFFFu << (shift + 8));
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (((valid >> j) & 1u) && (kv[j] & hmask) == (prefix & hmask))
                        atomicAdd(&hist[(kv[j] >> shift) & 255u], 1u);
                __syncwarp();
                unsigned c[8], own = 0u;
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    c[b] = hist[lane * 8 + b];
                    own += c[b];
                }
                unsigned incl = own;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const unsigned excl = incl - own;
                unsigned found = 0u;   // lane holding the bin: 1 + digit in bits 0-8, count below in 9-31
                if (excl < (unsigned)rem && (unsigned)rem <= incl) {
                    unsigned cum = excl;
#pragma unroll
                    for (int b = 0; b < 8; ++b) {
                        if (!found && cum + c[b] >= (unsigned)rem) found = (1u + lane * 8 + b) | (cum << 9);
                        cum += c[b];
                    }
                }
                found = __reduce_or_sync(0xffffffffu, found);
                prefix |= (((found & 511u) - 1u) & 255u) << shift;
                rem -= (int)(found >> 9);
                __syncwarp();
            }
            const uint32_t lo = prefix;
            unsigned lt = 0u, eq = 0u;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const bool v = (valid >> j) & 1u;
                lt |= (unsigned)(v && kv[j] < lo) << j;
                eq |= (unsigned)(v && kv[j] == lo) << j;
            }
            // keys equal to T are taken in position order (lane, then j) until k
            const int need = k - (int)__reduce_add_sync(0xffffffffu, (unsigned)__popc(lt));
            const int ce = __popc(eq);
            int incl = ce;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            int take = need - (incl - ce);
            unsigned keep = 0u;
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (((eq >> j) & 1u) && take > 0) {
                    keep |= 1u << j;
                    --take;
                }
            sel = lt | keep;
        }
        // visit list in position order
        const int cnt = __popc(sel);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        int off = incl - cnt;
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if ((sel >> j) & 1u) vis[off++] = (uint16_t)(qb + j - uq0);
        nsel = __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    if (a.mask_out) {
        for (int v = lane; v < nsel; v += 32) a.mask_out[q0 + vis[v]] = 1;
        return;
    }

    // K form (R_pad = 64, at most KMAX visits): the visits' k rows go to shared
    // memory (after the visit list, stride RP + 4) instead of being summed into
    // G, and the finish evaluates H x = K^T (K x) + lambda x.  For k_p < R_pad
    // that is less arithmetic and far less shared-memory traffic than forming H
    // and reading all R_pad^2 entries in each of the power method's matvecs;
    // the iteration and its result are those of H x (up to rounding order).
    constexpr bool KFORM = RP == 64;
    constexpr int KMAX = kTinyKForm, KST = TS::KST;
    static_assert(!KFORM || 256 + KMAX * KST <= TS::HA, "K rows fit after the visit list");
    // the host gives the K-only launch rows of k_p <= kTinyKForm (nsel = k_p)
    if (KONLY && nsel > KMAX) return;
    const bool kform = KONLY || (KFORM && nsel <= KMAX);   // the same in every lane
    float* Km = H + 256;

    // ---- Gram / data sums (Alg. 1 lines 6, 7, 9): lane owns H rows r = lane + 32 t
    // and keeps H[r][(r + d) mod RP] for d = 0 .. RP/2 (each unordered pair once,
    // the pairs at distance RP/2 twice with identical sums)
    float acc[TS::RPL][TS::ND];
    float bacc[TS::RPL];
#pragma unroll
    for (int t = 0; t < TS::RPL; ++t) {
        bacc[t] = 0.f;
#pragma unroll
        for (int d = 0; d < TS::ND; ++d) acc[t][d] = 0.f;
    }
    const Entry<EW>* bucket = reinterpret_cast<const Entry<EW>*>(a.bucket);
    auto elem = [&](int o, int idx, int r) -> float {
        if constexpr (BF16) {
            const uint16_t u = static_cast<const uint16_t*>(a.other[o])[(size_t)idx * RP + r];
            return __uint_as_float((uint32_t)u << 16);
        } else {
            return static_cast<const float*>(a.other[o])[(size_t)idx * RP + r];
        }
    };
    for (int vb = 0; vb < nsel; vb += 32) {
        const int nb = min(32, nsel - vb);
        uint4 e = make_uint4(0u, 0u, 0u, 0u);   // lane v: the entry of visit vb + v
        if (lane < nb) e = __ldg(reinterpret_cast<const uint4*>(bucket + q0 + vis[vb + lane]));
        for (int v = 0; v < nb; ++v) {
            const int i0 = (int)__shfl_sync(0xffffffffu, e.x, v);
            const int i1 = NOR > 1 ? (int)__shfl_sync(0xffffffffu, e.y, v) : 0;
            const int i2 = NOR > 2 ? (int)__shfl_sync(0xffffffffu, e.z, v) : 0;
            const float x = __uint_as_float(__shfl_sync(0xffffffffu, e.w, v));
            float kk[TS::RPL];
#pragma unroll
            for (int t = 0; t < TS::RPL; ++t) {
                const int r = lane + 32 * t;
                float p = 0.f;
                if (r < RP) {
                    p = elem(0, i0, r);
                    if (NOR > 1) p *= elem(1, i1, r);
                    if (NOR > 2) p *= elem(2, i2, r);
                    if (kform) Km[(vb + v) * KST + r] = p;
                    else ksh[r] = p;
                }
                kk[t] = p;
                bacc[t] = fmaf(x, p, bacc[t]);
            }
            if (kform) continue;
            __syncwarp();
#pragma unroll
            for (int t = 0; t < TS::RPL; ++t) {
                const int r = lane + 32 * t;
                if (r < RP) {
#pragma unroll
                    for (int d = 0; d < TS::ND; ++d) acc[t][d] = fmaf(kk[t], ksh[(r + d) & (RP - 1)], acc[t][d]);
                }
            }
            __syncwarp();
        }
    }
    if (kform) {
#pragma unroll
        for (int t = 0; t < TS::RPL; ++t) {
            const int r = lane + 32 * t;
            if (r < RP) bvec[r] = bacc[t];
        }
        __syncwarp();
        const int R = a.rank;
        const float lam = a.lambda;
        auto matvec = [&](const float* x, float* out) {
            // u_j = K[j] . x in lane j (rows 16-byte aligned; a quarter warp's
            // row starts fall in distinct banks), then out_r = sum_j K[j][r] u_j
            float u = 0.f;
            if (lane < nsel) {
                const float4* kr = reinterpret_cast<const float4*>(Km + lane * KST);
                const float4* x4 = reinterpret_cast<const float4*>(x);
#pragma unroll
                for (int c = 0; c < RP / 4; ++c) {
                    const float4 kq = kr[c], xq = x4[c];
                    u = fmaf(kq.x, xq.x, u);
                    u = fmaf(kq.y, xq.y, u);
                    u = fmaf(kq.z, xq.z, u);
                    u = fmaf(kq.w, xq.w, u);
                }
            }
#pragma unroll
            for (int t = 0; t < TS::RPL; ++t) out[t] = 0.f;
            for (int j = 0; j < nsel; ++j) {
                const float uj = __shfl_sync(0xffffffffu, u, j);
#pragma unroll
                for (int t = 0; t < TS::RPL; ++t) out[t] = fmaf(Km[j * KST + lane + 32 * t], uj, out[t]);
            }
#pragma unroll
            for (int t = 0; t < TS::RPL; ++t) {
                const int r = lane + 32 * t;
                if (r < R) out[t] = fmaf(lam, x[r], out[t]);
            }
        };
        finish_row_mv<RP>(a, row, bvec, vsh, lane, matvec);
        return;
    }
    if constexpr (!KONLY) {
        // H = G + lambda I (line 9), full symmetric, stride RP + 1; b
#pragma unroll
        for (int t = 0; t < TS::RPL; ++t) {
            const int r = lane + 32 * t;
            if (r < RP) {
#pragma unroll
                for (int d = 0; d < TS::ND; ++d) {
                    const int c = (r + d) & (RP - 1);
                    H[r * (RP + 1) + c] = acc[t][d];
                    H[c * (RP + 1) + r] = acc[t][d];
                }
                bvec[r] = bacc[t];
            }
        }
        __syncwarp();
        for (int r = lane; r < a.rank; r += 32) H[r * (RP + 1) + r] += a.lambda;
        __syncwarp();
        // lines 8, 10-13
        finish_row_warp<RP>(a, row, H, bvec, vsh, lane);
    }
}

}  // namespace ntc
