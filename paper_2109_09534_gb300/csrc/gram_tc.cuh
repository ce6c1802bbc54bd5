// gram_tc.cuh -- split-row Gram/data partials on the fifth-generation tensor
// cores (tcgen05.mma, kind::tf32) at padded rank 32: the same unit of work and
// the same output layout as k_heavy_gram (one chunk's certain visits, or one
// split row's chosen candidates -> G and b partials, Alg. 1 lines 6 and 9).
//
// G = sum_e k_e k_e^T over the sampled visits is a dense contraction.  FP32
// accuracy from TF32 operands by splitting: each k is written as big + small,
// big = k rounded to TF32 (10 explicit mantissa bits, half away from zero) and
// small = k - big (exact in FP32; read as TF32 by the tensor core, an error of
// at most 2^-21 |k| of either sign).  Per tile of VT visits the block stages
// S = [big; small] (2R rows x VT visits) in shared memory, and one MMA per 8
// visits (M = 64 = 2R, N = R) accumulates D = S big^T in tensor memory: rows
// 0..R-1 give bb = sum big big^T, rows R..2R-1 give sb = sum small big^T, and
// G = bb + sb + sb^T (the dropped small small^T is about 2^-24 of G).
// The tensor core's FP32 accumulation is biased (measured: accumulating a
// whole chunk in tensor memory moved G by up to 3e-5 relative), so D restarts
// every tile (VT/8 MMAs) and every warp adds its slice of each finished tile
// into FP32 registers: with M = 64, D row r sits in TMEM lane 32 (r / 16) +
// r % 16, so warp w holds rows 16 w .. 16 w + 15 in its lanes 0-15, and the
// 16x32bx2 load shape hands its 32 threads one row and 16 columns each.
// b = sum x_e k_e stays on the FP32 FMA path.
#pragma once

#include "nmc_kernels.cuh"

namespace ntc {
namespace tc {

// An mbarrier wait gives up after this many SM clock cycles (about one second
// at 2 GHz); the block then stops issuing work, waits (again bounded) for the
// MMAs it has committed, frees its tensor memory, writes no partial and
// records the timeout in the handle's counters, which the host reports.
constexpr long long kWaitCycles = 2000000000ll;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the completion of the phase with parity `parity`: false
// once `limit` SM clock cycles have passed without it.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit = kWaitCycles) {
    const long long t0 = clock64();
    while (!mbar_test(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}
// Generic-proxy shared-memory stores -> visible to the tensor core's reads.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// Tensor-memory allocation by one whole warp: ncols columns (a power of two,
// 32..512) of all 128 lanes; the base address is written to *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
// D (+)= A B^T with A (M x K) and B (N x K) described in shared memory, TF32
// inputs, FP32 accumulators in tensor memory; accum = 0 overwrites D.
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
// The mbarrier completes a phase once every MMA issued so far by this thread
// has finished (its shared-memory reads included).
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_addr(bar))
                 : "memory");
}
// 32 consecutive FP32 columns of this thread's lane (shape 32x32b: warp w reads
// lanes 32(w%4)..32(w%4)+31), waited for before returning.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor, no swizzle: start address, leading byte
// offset (between the two 16-byte core-matrix columns of one K = 8 step) and
// stride byte offset (between 8-row groups along M or N), descriptor version 1.
__host__ __device__ constexpr uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::tf32: FP32 accumulators (bits 4-5 = 1), TF32
// A and B (bits 7-9, 10-12 = 2), both K-major, N/8 in bits 17-22, M/16 in 24-28.
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// TF32 rounding of an FP32 value: the 13 low mantissa bits rounded half away
// from zero into the upper bits (finite inputs of the Gram are far from the
// overflow boundary).
__device__ __forceinline__ float round_tf32(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

}  // namespace tc

// Block shape and shared-memory map of the tensor-core Gram.  FW = tiles per
// tensor-memory accumulation window (D restarts, and is folded into the
// registers, every FW tiles); only 1 is valid.  k_heavy_gram_tc issues M = 64
// MMAs (IDESC64); the M = 128 form with the alternating lane placement
// described below (IDESC, odd tiles' A started 8 row groups early) is the one
// the TMA-gather kernel (gram_tma.cuh) uses, and the shared-memory reach below
// covers it.
template <int EW, int VT, int FW, int NT_>
struct GramTC {
    static constexpr int RP = 32;
    static constexpr int NT = NT_;                // threads: 128 or 256
    // resident blocks per SM: five of 128 threads (at most 102 registers; 5 x
    // (BYTES + 1 KB reserved) = 221 KB of the SM's 228 KB of shared memory;
    // 5 x 64 TMEM columns of 512)
    static constexpr int BLOCKS = NT == 128 ? 5 : 3;
    // (M = 128 form, TMA-gather kernel: D's 2R useful rows sit in TMEM lanes
    // 0..63 for even tiles and, with A's descriptor started 8 row groups early,
    // in lanes 64..127 for odd tiles, so the folding warps alternate)
    static constexpr int SPV = RP / 8;            // product slots per visit: 8 ranks each
    static constexpr int RS = VT * SPV / NT;      // product slots per thread and tile
    static constexpr int SROWS = 2 * RP;          // S rows: big, then small
    // S element (row r, visit v) at (v/4) KGB + (r/8) SBO + (r%8) 16 + (v%4) 4:
    // 8 x 16-byte core matrices, K-major.  A slot's 8 ranks are one row group;
    // SBO = 144 and KGB = 8 SBO + 64 put the 32 stores of a warp (4 row groups
    // x 8 visits) in distinct banks.
    static constexpr int SBO = 144;
    static constexpr int KGB = SROWS / 8 * SBO + 64;   // one 4-visit column of core matrices (= LBO)
    static constexpr int SB = VT / 4 * KGB;       // one S buffer
    static constexpr int M = 128;                 // A = S: rows 2R..127 are ignored rows of D
    static constexpr int N = RP;                  // B = big
    static constexpr uint32_t IDESC = tc::idesc_tf32(M, N);
    // M = 64 form: A = S rows 0..63 only; D row r in TMEM lane 32 (r / 16) + r % 16
    static constexpr uint32_t IDESC64 = tc::idesc_tf32(64, N);
    static constexpr int TCOLS = 2 * N;           // two D buffers (windows alternate)
    static constexpr int SE = 5;                  // entry stages
    static constexpr int ENTB = EW * 4;
    static constexpr int PW = 10 * 64 + RP;       // partial: ten 8x8 upper tiles, then b
    // shared memory: [mbarriers, TMEM slot][S0][S1][entries][reach pad]; odd
    // tiles (always S1) start A's reads 8 SBO early, inside S0
    static constexpr int S_OFF = 64;
    static_assert(8 * SBO <= SB, "odd tiles' shifted A reads stay inside S0");
    static constexpr int E_OFF = S_OFF + 2 * SB;
    static constexpr int USED = E_OFF + SE * VT * ENTB;
    // Furthest byte an operand read of the last K step of S1 can touch (16 row
    // groups of A, two core-matrix columns): the allocation covers it.
    static constexpr int LAST = S_OFF + SB + (VT / 4 - 2) * KGB;
    static constexpr int REACH = LAST + 15 * SBO + KGB + 128;
    static constexpr int BYTES = ((USED > REACH ? USED : REACH) + 127) / 128 * 128;
    // epilogue buffers alias S0 and S1 once every MMA has completed: the bb
    // and sb sums [2 RP][RP + 1] (the TMA-gather kernel: [4][RP][RP + 1], even
    // and odd tiles), then the b partials [NT][8]
    static constexpr int TSTR = RP + 1;
    static_assert(VT % 8 == 0 && VT <= NT && (VT * SPV) % NT == 0 && NT % SPV == 0, "tile shape");
    static_assert(FW == 1, "one tile per accumulation window (alternating lane placement)");
    static_assert(NT == 128 || NT == 256, "block");
    static_assert(4 * RP * TSTR * 4 + NT * 32 <= 2 * SB, "epilogue fits in S0 and S1");
    static_assert(SBO % 16 == 0 && KGB % 16 == 0, "descriptor offsets are 16-byte multiples");
    static_assert(EW == 4, "orders 2-4");
    static_assert(NT != 128 || BLOCKS * (BYTES + 1024) <= 228 * 1024, "the resident blocks' shared memory fits an SM");
    static_assert(BLOCKS * TCOLS <= 512, "the resident blocks' tensor memory fits an SM");
};

template <int EW, bool BF16, int NOR, int VT, int FW, int NTB>
__global__ void __launch_bounds__(NTB, GramTC<EW, VT, FW, NTB>::BLOCKS) k_heavy_gram_tc(ModeArgs a) {
    using G = GramTC<EW, VT, FW, NTB>;
    using RowT = std::conditional_t<BF16, uint2, float4>;   // 4 factor elements
    constexpr int NT = G::NT, SPV = G::SPV, RS = G::RS, RP = G::RP, ROWB = RP * (BF16 ? 2 : 4);
    static_assert(NT == 128, "four warps: one 16-row slice of D each");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw);   // [2]: MMAs of even / odd tiles
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem_raw + 16);
    unsigned char* S = smem_raw + G::S_OFF;
    Entry<EW>* ents = reinterpret_cast<Entry<EW>*>(smem_raw + G::E_OFF);
    const int tid = threadIdx.x, warp = tid >> 5;

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
                    float4 p = Gram<RP, EW, BF16>::to_f4(rb[j][0][hh]);
#pragma unroll
                    for (int o = 1; o < NOR; ++o) {
                        const float4 u = Gram<RP, EW, BF16>::to_f4(rb[j][o][hh]);
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
                p[c * 4 + G::SBO] = k[c] - big;           // row R + 8q + c: 4 SBO bytes = SBO floats on
            }
        }
    };
    // fold: warp w holds D rows 16 w .. 16 w + 15 in its lanes 0-15; thread l
    // adds row 16 w + l % 16, columns 16 (l / 16) .. + 15 (shape 16x32bx2)
    const uint32_t fofs = (uint32_t)(32 * warp) << 16;
    float acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = 0.f;
    auto fold = [&](uint32_t taddr) {
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.16x32bx2.x16.b32 "
            "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16], 16;\n\t"
            "tcgen05.wait::ld.sync.aligned;\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr + fofs)
            : "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] += __uint_as_float(r[j]);
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
    // D buffer of tile t: windows of FW tiles alternate between the two
    auto dbuf = [&](int t) -> uint32_t { return tmem + (uint32_t)(((t / FW) & 1) * G::N); };
    bool ok = true;
    if (a.test_stall_cycles > 0 && blockIdx.x == 0) {
        // test hook: block 0 waits on a phase that no MMA was committed to, so
        // that the wait runs out with nothing in flight
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
        tc::fence_before();      // and its reads of the D buffer tile t may overwrite
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
                tc::mma_tf32(dbuf(t), adesc, bdesc, G::IDESC64, (ks > 0 || t % FW != 0) ? 1u : 0u);
            }
            tc::mma_commit(&mbar[t & 1]);
        }
        if (t >= 1) {
            // tile t-1's MMAs have finished: its S buffer is free, and a window
            // that ended with it is folded
            ok &= tc::mbar_wait(&mbar[(t - 1) & 1], (uint32_t)(((t - 1) >> 1) & 1));
            tc::fence_after();
            if (t % FW == 0) fold(dbuf(t - 1));
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
    float* T2 = reinterpret_cast<float*>(S);          // [2 RP][TSTR]: bb rows, then sb rows
    float* bred = T2 + 2 * RP * G::TSTR;              // [NT][8]
    {
        const int l = tid & 31;
        float* T = T2 + (16 * warp + (l & 15)) * G::TSTR + 16 * (l >> 4);
#pragma unroll
        for (int j = 0; j < 16; ++j) T[j] = acc[j];
    }
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
        // (per call and since the handle was created; the host reports it)
        if (tid == 0 && a.stat_wait) {
            atomicAdd(a.stat_wait, 1ull);
            atomicAdd(a.stat_wait + 1, 1ull);
        }
        return;
    }
    // G[i][j] = bb[i][j] + (sb[i][j] + sb[j][i]) from the upper triangle, so
    // that the diagonal tiles are exactly symmetric
    float* out = a.partial + (size_t)item * G::PW;
    for (int s = tid; s < 10 * 64; s += NT) {
        int pa, pb;
        pair_ab(4, s >> 6, &pa, &pb);
        int gi = 8 * pa + ((s >> 3) & 7), gj = 8 * pb + (s & 7);
        if (gi > gj) {
            const int t = gi;
            gi = gj;
            gj = t;
        }
        const int ij = gi * G::TSTR + gj, ji = gj * G::TSTR + gi, L = RP * G::TSTR;
        const float bb = T2[ij];
        const float sb = T2[L + ij] + T2[L + ji];
        out[s] = bb + sb;
    }
    // b[r]: slot-owner threads th = r/8 (mod SPV), in increasing order
    for (int r = tid; r < RP; r += NT) {
        float t = 0.f;
        for (int th = r >> 3; th < NT; th += SPV) t += bred[th * 8 + (r & 7)];
        out[640 + r] = t;
    }
}

}  // namespace ntc
