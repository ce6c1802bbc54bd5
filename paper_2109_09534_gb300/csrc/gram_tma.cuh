// gram_tma.cuh -- split-row Gram/data partials on the tensor cores with the
// factor rows gathered by the Tensor Memory Accelerator: the same unit of work,
// arithmetic (TF32 big + small split, one tcgen05.mma kind::tf32 per 8 visits,
// D restarted every tile and folded into FP32 registers by alternating warp
// pairs) and output layout as k_heavy_gram_tc (gram_tc.cuh), with a warp-
// specialised pipeline in place of the register prefetch and the block
// barrier (Alg. 1 lines 6 and 9).
//
// Block = 4 consumer warps (0-3) + 1 producer warp (4).
//   producer: per tile of VT visits, the visits' 16-byte bucket entries are
//     loaded into registers four tiles ahead (their positions eight ahead)
//     and stored in the tile's stage;
//     one lane arms the stage's `full` mbarrier with the byte count, and the
//     lanes issue cp.async.bulk.tensor.2d.tile::gather4 copies: each brings 4
//     factor rows (4 row coordinates of one other mode's factor matrix, a box
//     of one row of R_pad elements) into the stage.  NS stages are in flight.
//   consumers: wait for the stage, form k_e = Hadamard product of the gathered
//     rows (4 ranks per thread, 8 threads per visit), b += x k, split k into
//     big + small and store S = [big; small] for the MMA, release the stage
//     (`empty` mbarrier); a named barrier among the consumers hands S to the
//     MMA-issuing thread, which commits the tile's MMAs to an mbarrier that
//     both frees S and marks D ready for the fold.
// Every mbarrier wait is bounded; a wait that gives up stops the block's work
// (the producer also stops when the consumers have), the block waits (again
// bounded) for the copies and MMAs it issued, frees its tensor memory, writes
// no partial and counts the timeout, which the host reports.
#pragma once

#include <cuda.h>

#include "gram_tc.cuh"
#include "ntc_host.h"

namespace ntc {

// GatherMaps (ntc_host.h): TMA descriptors of the other modes' factor matrices
// (float32 masters or bfloat16 copies, rows of R_pad elements) in increasing
// mode order, the updated mode left out: a 2-D tensor {R_pad, rows}, box
// {R_pad, 1}.

namespace tc {

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}
// Arrive once and add `bytes` to the phase's expected transaction count.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// Four rows (row coordinates r0..r3, all columns of the box from column 0) of
// a 2-D tensor into dst (4 consecutive boxes); completion counted on bar.
__device__ __forceinline__ void tma_gather4(void* dst, const CUtensorMap* map, int r0, int r1, int r2, int r3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];\n" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(smem_addr(bar))
        : "memory");
}
// Barrier `id` among the first `nthreads` threads (whole warps) with an OR of `pred`.
__device__ __forceinline__ bool bar_or(int id, int nthreads, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}
// Bounded wait that also ends, without counting as a timeout, once *stop is set.
// Returns 1 on completion, 0 on stop, -1 on timeout.
__device__ __forceinline__ int mbar_wait_or_stop(uint64_t* bar, uint32_t parity, const volatile int* stop) {
    const long long t0 = clock64();
    while (!mbar_test(bar, parity)) {
        if (*stop) return 0;
        if (clock64() - t0 > kWaitCycles) return -1;
    }
    return 1;
}

}  // namespace tc

// Shape and shared-memory map.  S buffers as in GramTC (same descriptors);
// behind them the NS stages of gathered rows ([mode][visit][row], 128-byte
// aligned) and of bucket entries.
template <int EW, bool BF16, int NOR, int VT, int NS>
struct GramTMA {
    using TC = GramTC<EW, VT, 1, 128>;
    static constexpr int RP = 32;
    static constexpr int NC = 128;                 // consumer threads (warps 0-3)
    static constexpr int NT = NC + 32;             // + the producer warp
    static constexpr int SPV = 8;                  // consumer threads per visit: 4 ranks each
    static constexpr int RS = VT * SPV / NC;       // visits (slots) per consumer thread and tile
    static constexpr int RB = RP * (BF16 ? 2 : 4); // bytes per factor row
    static constexpr int ROWS_STAGE = NOR * VT * RB;
    static constexpr int ENT_STAGE = VT * 16;
    // [full NS][empty NS][mma 2] mbarriers, TMEM slot, stop flag; then S0, S1
    static constexpr int BAR_BYTES = (2 * NS + 2) * 8;
    static constexpr int S_OFF = ((BAR_BYTES + 16 + 127) / 128) * 128;
    static constexpr int S_END = S_OFF + 2 * TC::SB;
    // the tensor core's reads of the odd tiles' shifted A operand reach this far
    // past S_OFF + SB (see GramTC::REACH): the row stages lie within that reach,
    // which only feeds ignored rows of D
    static constexpr int R_OFF = ((S_END + 127) / 128) * 128;
    static constexpr int E_OFF = R_OFF + NS * ROWS_STAGE;
    static constexpr int USED = E_OFF + NS * ENT_STAGE;
    static constexpr int REACH = S_OFF + TC::SB + (VT / 4 - 2) * TC::KGB + 15 * TC::SBO + TC::KGB + 128;
    // + 128: the kernel rounds the dynamic shared-memory base up to 128 bytes
    static constexpr int BYTES = ((USED > REACH ? USED : REACH) + 127) / 128 * 128 + 128;
    static constexpr int PW = 10 * 64 + RP;
    static constexpr int TSTR = RP + 1;
    static_assert(RS * NC == VT * SPV && VT % 8 == 0 && VT <= 64, "tile shape");
    static_assert(NOR >= 1 && NOR <= 3 && EW == 4, "orders 2-4");
    static_assert(4 * RP * TSTR * 4 + NC * 16 <= 2 * TC::SB, "epilogue fits in S0 and S1");
    static_assert(ROWS_STAGE % 128 == 0 && ENT_STAGE % 16 == 0, "stage alignment");
};

template <int EW, bool BF16, int NOR, int VT, int NS, int BPS>
__global__ void __launch_bounds__(GramTMA<EW, BF16, NOR, VT, NS>::NT, BPS)
    k_heavy_gram_tma(ModeArgs a, const __grid_constant__ GatherMaps maps) {
    using G = GramTMA<EW, BF16, NOR, VT, NS>;
    using TC = typename G::TC;
    constexpr int NC = G::NC, RS = G::RS, RP = G::RP, RB = G::RB;
    extern __shared__ __align__(16) unsigned char smem_tma_raw[];
    // TMA destinations (the row stages) must be 128-byte aligned
    unsigned char* smem_raw = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_tma_raw) + 127) & ~static_cast<uintptr_t>(127));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);   // [NS]: rows and entries of a stage landed
    uint64_t* empty = full + NS;                               // [NS]: consumers released a stage
    uint64_t* mma = empty + NS;                                // [2]: MMAs of even / odd tiles done
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem_raw + G::BAR_BYTES);
    volatile int* stop = reinterpret_cast<volatile int*>(smem_raw + G::BAR_BYTES + 4);
    unsigned char* S = smem_raw + G::S_OFF;
    unsigned char* rows = smem_raw + G::R_OFF;
    Entry<EW>* ents = reinterpret_cast<Entry<EW>*>(smem_raw + G::E_OFF);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

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
    const int ntiles = (cnt + VT - 1) / VT;
    auto tile_n = [&](int t) { return min(VT, cnt - t * VT); };

    if (warp == 0) tc::tmem_alloc(tslot, TC::TCOLS);
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], NC / 32);
        }
        tc::mbar_init(&mma[0], 1);
        tc::mbar_init(&mma[1], 1);
        *stop = 0;
        tc::mbar_init_fence();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    bool ok = true;

    if (warp == NC / 32) {
        // ---------------- producer warp ----------------
        const Entry<EW>* bucket = reinterpret_cast<const Entry<EW>*>(a.bucket);
        auto load_pos = [&](int t, int h) -> int {
            const int v = t * VT + lane + 32 * h;
            return (t < ntiles && lane + 32 * h < VT && v < cnt) ? (int)__ldg(list + v) : -1;
        };
        auto load_ent = [&](int pos) -> uint4 {
            return pos >= 0 ? __ldg(reinterpret_cast<const uint4*>(bucket + pos)) : make_uint4(0, 0, 0, 0);
        };
        // register rings: entries of tiles t .. t+3, positions of tiles t+4 ..
        // t+7, so that an entry load waits for a position loaded four tiles
        // earlier and a stage's entries were loaded four tiles before
        constexpr int AH = 4;
        uint4 E[AH][2];
        int P[AH][2];
#pragma unroll
        for (int i = 0; i < AH; ++i)
#pragma unroll
            for (int h = 0; h < 2; ++h) P[i][h] = load_pos(i, h);
#pragma unroll
        for (int i = 0; i < AH; ++i)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                E[i][h] = load_ent(P[i][h]);
                P[i][h] = load_pos(AH + i, h);
            }
        int issued = 0;
        for (int t = 0; t < ntiles; ++t) {
            const int s = t % NS;
            if (t >= NS) {
                const int w = tc::mbar_wait_or_stop(&empty[s], (uint32_t)(((t / NS) - 1) & 1), stop);
                if (w <= 0) {
                    if (w < 0) ok = false;
                    break;
                }
            }
            const int nv = tile_n(t);
            Entry<EW>* es = ents + s * VT;
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (lane + 32 * h < nv) *reinterpret_cast<uint4*>(es + lane + 32 * h) = E[0][h];
            __syncwarp();
            const int ng = (nv + 3) >> 2;   // groups of 4 visits
            if (lane == 0) tc::mbar_arrive_expect_tx(&full[s], (uint32_t)(NOR * ng * 4 * RB));
            __syncwarp();
            unsigned char* rs = rows + (size_t)s * G::ROWS_STAGE;
            for (int i = lane; i < NOR * ng; i += 32) {
                const int o = i / ng, g = i - o * ng;
                int r[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) r[k] = es[min(4 * g + k, nv - 1)].w[o];
                tc::tma_gather4(rs + (size_t)(o * VT + 4 * g) * RB, &maps.m[o], r[0], r[1], r[2], r[3], &full[s]);
            }
            issued = t + 1;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
#pragma unroll
                for (int i = 0; i + 1 < AH; ++i) E[i][h] = E[i + 1][h];
                E[AH - 1][h] = load_ent(P[0][h]);   // tile t + AH
#pragma unroll
                for (int i = 0; i + 1 < AH; ++i) P[i][h] = P[i + 1][h];
                P[AH - 1][h] = load_pos(t + 2 * AH, h);
            }
        }
        // copies issued but not consumed (only after a stop or a timeout): wait for them
        for (int t = max(0, issued - NS); t < issued; ++t) tc::mbar_wait(&full[t % NS], (uint32_t)((t / NS) & 1));
    } else {
        // ---------------- consumer warps ----------------
        const int c = tid & 7;   // ranks 4c .. 4c+3
        float bq[4] = {0.f, 0.f, 0.f, 0.f};
        auto load4 = [&](const unsigned char* row) -> float4 {
            if constexpr (BF16) return bf16x4_to_f32(*reinterpret_cast<const uint2*>(row + c * 8));
            else return *reinterpret_cast<const float4*>(row + c * 16);
        };
        // k rows of tile t -> S buffer (zero past nv, so a partial K step adds nothing); b += x k
        auto product = [&](int t, unsigned char* buf) {
            const int s = t % NS, nv = tile_n(t);
            const unsigned char* rs = rows + (size_t)s * G::ROWS_STAGE;
            const Entry<EW>* es = ents + s * VT;
#pragma unroll
            for (int j = 0; j < RS; ++j) {
                const int v = (tid >> 3) + j * (NC / 8);
                float k[4] = {0.f, 0.f, 0.f, 0.f};
                if (v < nv) {
                    float4 p = load4(rs + (size_t)v * RB);
#pragma unroll
                    for (int o = 1; o < NOR; ++o) {
                        const float4 u = load4(rs + (size_t)(o * VT + v) * RB);
                        p.x *= u.x;
                        p.y *= u.y;
                        p.z *= u.z;
                        p.w *= u.w;
                    }
                    k[0] = p.x;
                    k[1] = p.y;
                    k[2] = p.z;
                    k[3] = p.w;
                    const float x = __int_as_float(es[v].w[EW - 1]);
#pragma unroll
                    for (int i = 0; i < 4; ++i) bq[i] = fmaf(x, k[i], bq[i]);
                }
                // rows 4c+i (big) and R + 4c+i (small) of visit v
                float* p = reinterpret_cast<float*>(buf + (v >> 2) * TC::KGB + (c >> 1) * TC::SBO + (c & 1) * 64 +
                                                    (v & 3) * 4);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float big = tc::round_tf32(k[i]);
                    p[i * 4] = big;
                    p[i * 4 + TC::SBO] = k[i] - big;   // 4 SBO bytes = SBO floats on
                }
            }
        };
        const int fpar = (warp & 3) >> 1;
        const uint32_t fofs = (uint32_t)(32 * (warp & 3)) << 16;
        float acc[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = 0.f;
        auto fold = [&](uint32_t taddr) {
            float v[32];
            tc::tmem_ld32(taddr + fofs, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[j] += v[j];
        };
        auto dbuf = [&](int t) -> uint32_t { return tmem + (uint32_t)((t & 1) * TC::N); };
        auto consume = [&](int t) {   // wait for tile t's stage, form its S, release the stage
            ok &= tc::mbar_wait(&full[t % NS], (uint32_t)((t / NS) & 1));
            if (ok) product(t, S + (t & 1) * TC::SB);
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&empty[t % NS]);
        };
        if (a.test_stall_cycles > 0 && blockIdx.x == 0) {
            // test hook: block 0 waits on a phase that no MMA was committed to
            ok = tc::mbar_wait(&mma[0], 0u, a.test_stall_cycles);
        }
        if (ntiles > 0 && ok) consume(0);
        const uint32_t s_base = tc::smem_addr(S);
        int issued = 0;   // tiles whose MMAs were committed
        for (int t = 0; t < ntiles; ++t) {
            tc::fence_async_smem();   // this thread's S stores of tile t
            tc::fence_before();       // and its reads of the D buffer tile t may overwrite
            if (tc::bar_or(1, NC, !ok)) break;   // a wait gave up: issue nothing more
            issued = t + 1;
            if (tid == 0) {
                tc::fence_after();
                const uint32_t buf = s_base + (uint32_t)((t & 1) * TC::SB);
                const uint32_t ashift = (t & 1) ? 8u * TC::SBO : 0u;   // odd tiles: S rows -> D lanes 64..127
                const int nks = (tile_n(t) + 7) >> 3;
                for (int ks = 0; ks < nks; ++ks) {
                    const uint32_t kaddr = buf + (uint32_t)(ks * 2 * TC::KGB);
                    const uint64_t adesc = tc::smem_desc(kaddr - ashift, TC::KGB, TC::SBO);
                    const uint64_t bdesc = tc::smem_desc(kaddr, TC::KGB, TC::SBO);
                    tc::mma_tf32(dbuf(t), adesc, bdesc, TC::IDESC, ks > 0 ? 1u : 0u);
                }
                tc::mma_commit(&mma[t & 1]);
            }
            if (t >= 1) {
                // tile t-1's MMAs have finished: its S buffer is free and its D is folded
                ok &= tc::mbar_wait(&mma[(t - 1) & 1], (uint32_t)(((t - 1) >> 1) & 1));
                tc::fence_after();
                if (ok && fpar == ((t - 1) & 1)) fold(dbuf(t - 1));
            }
            if (t + 1 < ntiles && ok) consume(t + 1);
        }
        if (!ok) *stop = 1;   // the producer stops at its next wait
        if (issued > 0) {
            // the last commit covers every MMA this block issued
            const bool last = tc::mbar_wait(&mma[(issued - 1) & 1], (uint32_t)(((issued - 1) >> 1) & 1));
            tc::fence_after();
            if (ok && last && issued == ntiles && fpar == ((ntiles - 1) & 1)) fold(dbuf(ntiles - 1));
            ok &= last;
        }
        tc::bar_or(1, NC, false);   // every MMA has finished: S0 becomes the epilogue buffer
        float* T4 = reinterpret_cast<float*>(S);          // [warp][RP][TSTR]: bb even, sb even, bb odd, sb odd
        float* bred = T4 + 4 * RP * G::TSTR;              // [NC][4]
        {
            float* T = T4 + warp * RP * G::TSTR;
#pragma unroll
            for (int j = 0; j < 32; ++j) T[lane * G::TSTR + j] = acc[j];
        }
        reinterpret_cast<float4*>(bred)[tid] = make_float4(bq[0], bq[1], bq[2], bq[3]);
    }
    tc::fence_before();
    const int any_timeout = __syncthreads_or(ok ? 0 : 1);   // a wait that gave up in any thread
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_free(tmem, TC::TCOLS);
    }
    if (any_timeout) {
        // the partial is not valid: leave it unwritten and count the block
        if (tid == 0 && a.stat_wait) {
            atomicAdd(a.stat_wait, 1ull);
            atomicAdd(a.stat_wait + 1, 1ull);
        }
        return;
    }
    const float* T4 = reinterpret_cast<const float*>(S);
    const float* bred = T4 + 4 * RP * G::TSTR;
    float* out = a.partial + (size_t)item * G::PW;
    for (int s = tid; s < 10 * 64; s += G::NT) {
        int pa, pb;
        pair_ab(4, s >> 6, &pa, &pb);
        int gi = 8 * pa + ((s >> 3) & 7), gj = 8 * pb + (s & 7);
        if (gi > gj) {
            const int t = gi;
            gi = gj;
            gj = t;
        }
        const int ij = gi * G::TSTR + gj, ji = gj * G::TSTR + gi, L = RP * G::TSTR;
        const float bb = T4[ij] + T4[2 * L + ij];
        const float sb = (T4[L + ij] + T4[3 * L + ij]) + (T4[L + ji] + T4[3 * L + ji]);
        out[s] = bb + sb;
    }
    // b[r]: threads with r / 4 == tid % 8, in increasing order
    for (int r = tid; r < RP; r += G::NT) {
        float t = 0.f;
        for (int th = r >> 2; th < NC; th += 8) t += bred[th * 4 + (r & 3)];
        out[640 + r] = t;
    }
}

}  // namespace ntc
