// gram_tc64.cuh -- split-row Gram/data partials on the tensor cores at padded
// rank 64: the same unit of work, split arithmetic and output layout as the
// FP32 FMA kernel k_heavy_gram<64> (one chunk's certain visits, or one split
// row's chosen candidates -> G and b partials, Alg. 1 lines 6 and 9).
//
// As at rank 32 (gram_tc.cuh), each k is split into big = TF32(k) and small =
// k - big, a tile of VT visits is staged as S = [big; small] in shared memory
// (here 2 R = 128 rows, so M = 128 has no ignored rows), and one tcgen05.mma
// kind::tf32 per 8 visits accumulates D = S big^T (M = 128, N = 64) in tensor
// memory: rows 0..63 of D are bb = sum big big^T, rows 64..127 sb = sum small
// big^T, and G = bb + sb + sb^T.  D restarts every tile in one of two buffers
// (the tensor core's FP32 accumulation is biased over long sums) and all eight
// warps fold the finished tile into FP32 registers: warp w holds TMEM lanes
// 32 (w mod 4) .. + 31 and columns 32 (w / 4) .. + 31.  b stays on FP32 FMA.
#pragma once

#include "gram_tc.cuh"

namespace ntc {

template <int EW, int VT>
struct GramTC64 {
    static constexpr int RP = 64;
    static constexpr int NT = 256;
    static constexpr int BLOCKS = 2;              // resident blocks per SM (shared memory)
    static constexpr int SPV = RP / 8;            // product slots per visit: 8 ranks each
    static constexpr int RS = VT * SPV / NT;      // product slots per thread and tile
    static constexpr int SROWS = 2 * RP;          // S rows: big, then small
    // S element (row r, visit v) at (v/4) KGB + (r/8) SBO + (r%8) 16 + (v%4) 4:
    // K-major 8 x 16-byte core matrices; SBO = 144 puts the 32 stores of a warp
    // (8 row groups x 4 visits) in distinct banks
    static constexpr int SBO = 144;
    static constexpr int KGB = SROWS / 8 * SBO + 64;   // one 4-visit column of core matrices (= LBO)
    static constexpr int SB = VT / 4 * KGB;       // one S buffer
    static constexpr int M = 128;
    static constexpr int N = RP;
    static constexpr uint32_t IDESC = tc::idesc_tf32(M, N);
    static constexpr int TCOLS = 2 * N;           // two D buffers (tiles alternate)
    static constexpr int SE = 5;                  // entry stages
    static constexpr int ENTB = EW * 4;
    static constexpr int NP = 36;                 // 8x8 tiles of the upper triangle
    static constexpr int PW = NP * 64 + RP;       // partial: the tiles, then b
    static constexpr int S_OFF = 64;
    static constexpr int E_OFF = S_OFF + 2 * SB;
    static constexpr int USED = E_OFF + SE * VT * ENTB;
    // the operand reads of the last K step end inside their S buffer
    static constexpr int REACH = S_OFF + SB + (VT / 4 - 2) * KGB + KGB + 15 * SBO + 128;
    static constexpr int BYTES = ((USED > REACH ? USED : REACH) + 127) / 128 * 128;
    static constexpr int TSTR = RP + 1;           // epilogue: D rows [128][TSTR], then b partials [NT][8]
    static_assert(VT % 8 == 0 && (VT * SPV) % NT == 0 && NT % SPV == 0 && VT <= NT, "tile shape");
    static_assert(S_OFF + SB + (VT / 4 - 1) * KGB + 15 * SBO + 128 <= S_OFF + 2 * SB, "reads stay in S1");
    static_assert(SROWS * TSTR * 4 + NT * 32 <= 2 * SB, "epilogue fits in S0 and S1");
    static_assert(SBO % 16 == 0 && KGB % 16 == 0, "descriptor offsets are 16-byte multiples");
    static_assert(EW == 4, "orders 2-4");
};

template <int EW, bool BF16, int NOR, int VT>
__global__ void __launch_bounds__(GramTC64<EW, VT>::NT, GramTC64<EW, VT>::BLOCKS) k_heavy_gram_tc64(ModeArgs a) {
    using G = GramTC64<EW, VT>;
    using RowT = std::conditional_t<BF16, uint2, float4>;   // 4 factor elements
    constexpr int NT = G::NT, SPV = G::SPV, RS = G::RS, RP = G::RP, ROWB = RP * (BF16 ? 2 : 4);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw);   // [2]: MMAs of even / odd tiles
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem_raw + 16);
    unsigned char* S = smem_raw + G::S_OFF;
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

    if (warp == 0) tc::tmem_alloc(tslot, G::TCOLS);
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        tc::mbar_init_fence();
    }

    const Entry<EW>* bucket = reinterpret_cast<const Entry<EW>*>(a.bucket);
    const int ntiles = (cnt + VT - 1) / VT;
    auto tile_n = [&](int t) { return min(VT, cnt - t * VT); };
    auto pos_of = [&](int t) -> uint32_t { return (t < ntiles && tid < tile_n(t)) ? list[t * VT + tid] : 0u; };
    auto issue_entries = [&](int t, uint32_t pos) {
        if (t < ntiles && tid < tile_n(t)) {
            const unsigned char* src = reinterpret_cast<const unsigned char*>(bucket + pos);
            unsigned char* dst = reinterpret_cast<unsigned char*>(ents + (t % G::SE) * VT + tid);
#pragma unroll
            for (int c = 0; c < G::ENTB / 16; ++c) cp_async16(dst + 16 * c, src + 16 * c);
        }
    };
    // this thread's 8 ranks (8q .. 8q+7) of every k row it forms; slot j of a
    // tile is visit (tid + j NT) / SPV
    const int q = tid % SPV;
    RowT rb[RS][NOR][2];
    auto load_rows = [&](const Entry<EW>* e, int nv) {
#pragma unroll
        for (int j = 0; j < RS; ++j) {
            const int v = (tid + j * NT) / SPV;
            if (v < nv) {
#pragma unroll
                for (int o = 0; o < NOR; ++o) {
                    const RowT* src = reinterpret_cast<const RowT*>(static_cast<const unsigned char*>(a.other[o]) +
                                                                    (size_t)e[v].w[o] * ROWB) + 2 * q;
                    rb[j][o][0] = __ldg(src);
                    rb[j][o][1] = __ldg(src + 1);
                }
            }
        }
    };
    float bq[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) bq[c] = 0.f;
    // k rows of the tile -> S (zero past nv, so a partial K step adds nothing); b += x k
    auto product = [&](const Entry<EW>* e, unsigned char* buf, int nv) {
        unsigned char* qb = buf + q * G::SBO;
#pragma unroll
        for (int j = 0; j < RS; ++j) {
            const int v = (tid + j * NT) / SPV;
            float k[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) k[c] = 0.f;
            if (v < nv) {
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    float4 p = Gram<32, EW, BF16>::to_f4(rb[j][0][hh]);
#pragma unroll
                    for (int o = 1; o < NOR; ++o) {
                        const float4 u = Gram<32, EW, BF16>::to_f4(rb[j][o][hh]);
                        p.x *= u.x;
                        p.y *= u.y;
                        p.z *= u.z;
                        p.w *= u.w;
                    }
                    k[4 * hh] = p.x;
                    k[4 * hh + 1] = p.y;
                    k[4 * hh + 2] = p.z;
                    k[4 * hh + 3] = p.w;
                }
                const float x = __int_as_float(e[v].w[EW - 1]);
#pragma unroll
                for (int c = 0; c < 8; ++c) bq[c] = fmaf(x, k[c], bq[c]);
            }
            float* p = reinterpret_cast<float*>(qb + (v >> 2) * G::KGB + (v & 3) * 4);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float big = tc::round_tf32(k[c]);
                p[c * 4] = big;                           // row 8q + c
                p[c * 4 + 2 * G::SBO] = k[c] - big;       // row R + 8q + c: 8 SBO bytes = 2 SBO floats on
            }
        }
    };
    // this warp's part of D: lanes 32 (warp % 4) .., columns 32 (warp / 4) ..
    const uint32_t fofs = ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * 32);
    float acc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = 0.f;
    auto fold = [&](uint32_t taddr) {
        float v[32];
        tc::tmem_ld32(taddr + fofs, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] += v[j];
    };

    issue_entries(0, pos_of(0));
    issue_entries(1, pos_of(1));
    issue_entries(2, pos_of(2));
    cp_async_commit();
    const uint32_t p3 = pos_of(3);
    cp_async_wait<0>();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    auto dbuf = [&](int t) -> uint32_t { return tmem + (uint32_t)((t & 1) * G::N); };
    bool ok = true;
    if (a.test_stall_cycles > 0 && blockIdx.x == 0) {
        // test hook: block 0 waits on a phase that no MMA was committed to
        ok = tc::mbar_wait(&mbar[0], 0u, a.test_stall_cycles);
    }
    if (ntiles > 0) {
        load_rows(ents, tile_n(0));
        product(ents, S, tile_n(0));
    }
    if (ntiles > 1) load_rows(ents + VT, tile_n(1));
    issue_entries(3, p3);
    cp_async_commit();
    uint32_t pos_next = pos_of(4);
    const uint32_t s_base = tc::smem_addr(S);
    int issued = 0;   // tiles whose MMAs were committed
    for (int t = 0; t < ntiles; ++t) {
        cp_async_wait<1>();      // entries of t+2
        tc::fence_async_smem();  // this thread's S stores of tile t
        tc::fence_before();      // and its reads of the D buffer tile t overwrites
        if (__syncthreads_or(ok ? 0 : 1)) break;   // a wait gave up: issue nothing more
        issued = t + 1;
        if (tid == 0) {
            tc::fence_after();
            const uint32_t buf = s_base + (uint32_t)((t & 1) * G::SB);
            const int nks = (tile_n(t) + 7) >> 3;
            for (int ks = 0; ks < nks; ++ks) {
                const uint32_t kaddr = buf + (uint32_t)(ks * 2 * G::KGB);
                const uint64_t adesc = tc::smem_desc(kaddr, G::KGB, G::SBO);
                const uint64_t bdesc = tc::smem_desc(kaddr, G::KGB, G::SBO);
                tc::mma_tf32(dbuf(t), adesc, bdesc, G::IDESC, ks > 0 ? 1u : 0u);
            }
            tc::mma_commit(&mbar[t & 1]);
        }
        if (t >= 1) {
            // tile t-1's MMAs have finished: its S buffer is free and its D is folded
            ok &= tc::mbar_wait(&mbar[(t - 1) & 1], (uint32_t)(((t - 1) >> 1) & 1));
            tc::fence_after();
            if (ok) fold(dbuf(t - 1));
        }
        if (t + 1 < ntiles) product(ents + ((t + 1) % G::SE) * VT, S + ((t + 1) & 1) * G::SB, tile_n(t + 1));
        if (t + 2 < ntiles) load_rows(ents + ((t + 2) % G::SE) * VT, tile_n(t + 2));
        issue_entries(t + 4, pos_next);
        pos_next = pos_of(t + 5);
        cp_async_commit();
    }
    cp_async_wait<0>();
    if (issued > 0) {
        // the last commit covers every MMA this block issued
        const bool last = tc::mbar_wait(&mbar[(issued - 1) & 1], (uint32_t)(((issued - 1) >> 1) & 1));
        tc::fence_after();
        if (ok && last && issued == ntiles) fold(dbuf(ntiles - 1));
        ok &= last;
    }
    __syncthreads();   // every MMA has finished: S0 becomes the epilogue buffer
    float* T = reinterpret_cast<float*>(S);           // [128][TSTR]: bb rows, then sb rows
    float* bred = T + G::SROWS * G::TSTR;             // [NT][8]
#pragma unroll
    for (int j = 0; j < 32; ++j) T[(32 * (warp & 3) + lane) * G::TSTR + (warp >> 2) * 32 + j] = acc[j];
    reinterpret_cast<float4*>(bred)[2 * tid] = make_float4(bq[0], bq[1], bq[2], bq[3]);
    reinterpret_cast<float4*>(bred)[2 * tid + 1] = make_float4(bq[4], bq[5], bq[6], bq[7]);
    tc::fence_before();
    const int any_timeout = __syncthreads_or(ok ? 0 : 1);   // a wait that gave up in any thread
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_free(tmem, G::TCOLS);
    }
    if (any_timeout) {
        // the partial is not valid: leave it unwritten and count the block
        if (tid == 0 && a.stat_wait) {
            atomicAdd(a.stat_wait, 1ull);
            atomicAdd(a.stat_wait + 1, 1ull);
        }
        return;
    }
    // G[i][j] = bb[i][j] + (sb[i][j] + sb[j][i]) from the upper triangle, so
    // that the diagonal tiles are exactly symmetric
    float* out = a.partial + (size_t)item * G::PW;
    for (int s = tid; s < G::NP * 64; s += NT) {
        int pa, pb;
        pair_ab(8, s >> 6, &pa, &pb);
        int gi = 8 * pa + ((s >> 3) & 7), gj = 8 * pb + (s & 7);
        if (gi > gj) {
            const int t = gi;
            gi = gj;
            gj = t;
        }
        const float bb = T[gi * G::TSTR + gj];
        const float sb = T[(RP + gi) * G::TSTR + gj] + T[(RP + gj) * G::TSTR + gi];
        out[s] = bb + sb;
    }
    // b[r]: slot-owner threads th = r/8 (mod SPV), in increasing order
    for (int r = tid; r < RP; r += NT) {
        float t = 0.f;
        for (int th = r >> 3; th < NT; th += SPV) t += bred[th * 8 + (r & 7)];
        out[G::NP * 64 + r] = t;
    }
}

}  // namespace ntc
