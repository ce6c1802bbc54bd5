// launch_rp.cuh -- enqueue one inner iteration of Algorithm 1 on one mode for
// a given padded rank: light rows (side stream) and split rows (sample,
// resolve, Gram partials, reduce, finish).  Included once per rank by
// nmc_rp*.cu so that the instantiations compile in parallel.
#pragma once

#include "gram_tc.cuh"
#include "gram_tc64.cuh"
#include "gram_tma.cuh"
#include "nmc_kernels.cuh"
#include "ntc_host.h"
#include "tiny_rows.cuh"

namespace ntc {

// The split-row Gram runs on the tensor cores (gram_tc.cuh) at padded rank
// 32 with the other modes' count fixed at compile time (orders 2-4), unless
// the handle's "gram_tc" is 0; visits per staged tile:
template <int RP, int EW, int NOR>
constexpr bool kTensorGram = RP == 32 && EW == 4 && NOR > 0;
// and at padded rank 64 (gram_tc64.cuh: M = 128 = 2 R, N = 64)
template <int RP, int EW, int NOR>
constexpr bool kTensorGram64 = RP == 64 && EW == 4 && NOR > 0;
constexpr int kTcTile = 64;
constexpr int kTcWindow = 1;   // tiles per tensor-memory accumulation window
constexpr int kTcThreads = 128;
// TMA-gather form ("gram_tc" 2): row stages in flight per block (the gathered
// rows of a stage take NOR * 8 KB at float32) and blocks per SM
template <int NOR>
constexpr int kTmaStages = NOR == 3 ? 2 : 4;
constexpr int kTmaBlocks = 2;
template <int EW, bool BF, int NOR>
using TmaG = GramTMA<EW, BF, NOR, kTcTile, kTmaStages<NOR>>;
// ("gram_tc" 3: two stages, three blocks per SM)
template <int EW, bool BF, int NOR>
using TmaG3 = GramTMA<EW, BF, NOR, kTcTile, 2>;

template <int RP, int EW, bool BF, int NOR>
cudaError_t launch_mode_t(const ModeArgs& a, const ModePlan& p, Launcher& L, bool mask_only) {
    cudaStream_t s = L.s;
    // kernel attributes once per process (handles may run on several threads)
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [] {
        constexpr int nomax = Gram<RP, EW, BF>::NOMAX;
        cudaError_t e = set_smem(k_light<RP, EW, BF, NOR>, LightSmem<RP, EW, BF, NOR>::bytes(nomax));
        if (e == cudaSuccess) e = set_smem(k_heavy_gram<RP, EW, BF, NOR>, HeavyGramSmem<RP, EW, BF, NOR>::bytes(nomax));
        if (e == cudaSuccess) e = set_smem(k_rows_finish<RP>, RowFinish<RP>::bytes());
        if constexpr (EW == 4 && NOR > 0)
            if (e == cudaSuccess) e = set_smem(k_tiny_rows<RP, EW, BF, NOR>, TinyShape<RP>::bytes());
        if constexpr (EW == 4 && NOR > 0 && RP == 64)
            if (e == cudaSuccess) e = set_smem(k_tiny_rows<RP, EW, BF, NOR, true>, TinyShape<RP, true>::bytes());
        if constexpr (kTensorGram64<RP, EW, NOR>)
            if (e == cudaSuccess) e = set_smem(k_heavy_gram_tc64<EW, BF, NOR, kTcTile>, GramTC64<EW, kTcTile>::BYTES);
        if constexpr (kTensorGram<RP, EW, NOR>) {
            if (e == cudaSuccess) e = set_smem(k_heavy_gram_tc<EW, BF, NOR, kTcTile, kTcWindow, kTcThreads>, GramTC<EW, kTcTile, kTcWindow, kTcThreads>::BYTES);
            if (e == cudaSuccess)
                e = set_smem(k_heavy_gram_tma<EW, BF, NOR, kTcTile, kTmaStages<NOR>, kTmaBlocks>, TmaG<EW, BF, NOR>::BYTES);
            if (e == cudaSuccess)
                e = set_smem(k_heavy_gram_tma<EW, BF, NOR, kTcTile, 2, 3>, TmaG3<EW, BF, NOR>::BYTES);

        }
        attr_err = e;
    });
    if (attr_err != cudaSuccess) return attr_err;
    const bool fork = p.n_light + p.n_tiny > 0 && p.n_heavy > 0 && L.h->overlap;
    // light rows: in stream order, or on the side stream (forked here for
    // overlap 1, beside the split-row sampler; after the sampler for overlap
    // 2, beside the split-row Gram)
    auto launch_light = [&]() -> cudaError_t {
        cudaError_t e = cudaSuccess;
        if (fork) {
            ntc_handle* h = L.h;
            if (!h->side) {
                if ((e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking)) != cudaSuccess) return e;
                if ((e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming)) != cudaSuccess) return e;
                if ((e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming)) != cudaSuccess) return e;
            }
            if ((e = cudaEventRecord(h->ev_fork, s)) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(h->side, h->ev_fork, 0)) != cudaSuccess) return e;
        }
        if (p.n_light + p.n_tiny > 0) {
            const int64_t bytes = (p.visits - p.visits_heavy) * L.bpv;   // light and one-warp rows
            cudaStream_t ls = fork ? L.h->side : s;
            e = L.run_on(ls, NTC_K_LIGHT, mask_only ? 0 : bytes, [&] {
                if constexpr (EW == 4 && NOR > 0) {
                    if (p.n_tiny > 0) {
                        constexpr int W = TinyShape<RP>::WARPS;
                        // at R_pad 64 the rows of at most kTinyKForm visits (the
                        // tail: rows are longest first) take the K-only launch
                        const int nbig = RP == 64 ? p.n_tiny_big : p.n_tiny;
                        int nl = 0;
                        if (nbig > 0) {
                            ModeArgs ab = a;
                            ab.tiny_end = nbig;
                            k_tiny_rows<RP, EW, BF, NOR><<<(nbig + W - 1) / W, W * 32, TinyShape<RP>::bytes(), ls>>>(ab);
                            ++nl;
                        }
                        if constexpr (RP == 64) {
                            if (nbig < p.n_tiny) {
                                ModeArgs ak = a;
                                ak.tiny_begin = nbig;
                                const int nk = p.n_tiny - nbig;
                                k_tiny_rows<RP, EW, BF, NOR, true>
                                    <<<(nk + W - 1) / W, W * 32, TinyShape<RP, true>::bytes(), ls>>>(ak);
                                ++nl;
                            }
                        }
                        // run_on counts one launch
                        *L.launches += nl - 1 + (p.n_light > 0 ? 1 : 0);
                    }
                }
                if (p.n_light > 0)
                    k_light<RP, EW, BF, NOR><<<p.n_light, kLightThreads, LightSmem<RP, EW, BF, NOR>::bytes(a.n_other), ls>>>(a);
            });
            if (e != cudaSuccess) return e;
            if (fork && (e = cudaEventRecord(L.h->ev_join, ls)) != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    cudaError_t e = cudaSuccess;
    const bool light_late = fork && L.h->overlap == 2;
    if (!light_late && (e = launch_light()) != cudaSuccess) return e;
    // split-row sampling: on the sampling stream when pipelined, so that it can
    // run beside the previous update's Gram; its scratch set (a.sset) is free
    // once the Gram two updates back has read it
    ntc_handle* h = L.h;
    const bool pipe = h->pipeline && p.n_heavy > 0;
    cudaStream_t ss = s;
    if (pipe) {
        if (!h->samp) {
            if ((e = cudaStreamCreateWithFlags(&h->samp, cudaStreamNonBlocking)) != cudaSuccess) return e;
            for (int q = 0; q < 2; ++q) {
                if ((e = cudaEventCreateWithFlags(&h->ev_sampled[q], cudaEventDisableTiming)) != cudaSuccess) return e;
                if ((e = cudaEventCreateWithFlags(&h->ev_free[q], cudaEventDisableTiming)) != cudaSuccess) return e;
            }
        }
        ss = h->samp;
        if ((e = cudaStreamWaitEvent(ss, h->ev_free[a.sset], 0)) != cudaSuccess) return e;
    }
    if (p.n_heavy > 0 && a.perm) {
        // epoch-permutation variant: visits straight from the permutation
        e = L.run_on(ss, NTC_K_HEAVY_SAMPLE, 0, [&] { k_perm_visits<EW><<<p.n_chunks, kThreads, 0, ss>>>(a); });
        if (e != cudaSuccess) return e;
    }
    if (p.n_heavy > 0) {
        if (!a.perm) {
            e = cudaMemsetAsync(a.flags, 0, sizeof(uint32_t) * p.n_heavy, ss);
            if (e != cudaSuccess) return e;
            e = L.run_on(ss, NTC_K_HEAVY_SAMPLE, 0, [&] { k_heavy_sample<EW><<<p.n_chunks, kThreads, 0, ss>>>(a); });
            if (e != cudaSuccess) return e;
            e = L.run_on(ss, NTC_K_HEAVY_RESOLVE, 0, [&] { k_heavy_resolve<EW><<<p.n_heavy, kThreads, 0, ss>>>(a); });
            if (e != cudaSuccess) return e;
        }
        if (pipe) {
            if ((e = cudaEventRecord(h->ev_sampled[a.sset], ss)) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(s, h->ev_sampled[a.sset], 0)) != cudaSuccess) return e;
        }
        if (light_late && (e = launch_light()) != cudaSuccess) return e;
        if (mask_only) {
            k_heavy_mask<EW><<<p.n_chunks + p.n_heavy, kThreads, 0, s>>>(a);
            ++*L.launches;
            if (pipe && (e = cudaEventRecord(h->ev_free[a.sset], s)) != cudaSuccess) return e;
        } else {
            const GatherMaps* gm = nullptr;
            if constexpr (kTensorGram<RP, EW, NOR>)
                if (h->gram_tc >= 2 && (e = gather_maps(h, (int)a.ss.mode, &gm)) != cudaSuccess) return e;
            e = L.run(NTC_K_HEAVY_GRAM, p.visits_heavy * L.bpv, [&] {
                bool tensor = false;
                if constexpr (kTensorGram<RP, EW, NOR>) {
                    if (h->gram_tc == 2) {
                        using T = TmaG<EW, BF, NOR>;
                        k_heavy_gram_tma<EW, BF, NOR, kTcTile, kTmaStages<NOR>, kTmaBlocks>
                            <<<p.n_chunks + p.n_heavy, T::NT, T::BYTES, s>>>(a, *gm);
                        tensor = true;
                    } else if (h->gram_tc == 3) {
                        using T = TmaG3<EW, BF, NOR>;
                        k_heavy_gram_tma<EW, BF, NOR, kTcTile, 2, 3><<<p.n_chunks + p.n_heavy, T::NT, T::BYTES, s>>>(a, *gm);
                        tensor = true;
                    } else if (h->gram_tc) {
                        using T = GramTC<EW, kTcTile, kTcWindow, kTcThreads>;
                        k_heavy_gram_tc<EW, BF, NOR, kTcTile, kTcWindow, kTcThreads><<<p.n_chunks + p.n_heavy, T::NT, T::BYTES, s>>>(a);
                        tensor = true;
                    }
                }
                if constexpr (kTensorGram64<RP, EW, NOR>) {
                    if (h->gram_tc) {
                        using T = GramTC64<EW, kTcTile>;
                        k_heavy_gram_tc64<EW, BF, NOR, kTcTile><<<p.n_chunks + p.n_heavy, T::NT, T::BYTES, s>>>(a);
                        tensor = true;
                    }
                }
                if (!tensor)
                    k_heavy_gram<RP, EW, BF, NOR><<<p.n_chunks + p.n_heavy, GramNT<RP>::value,
                                               HeavyGramSmem<RP, EW, BF, NOR>::bytes(a.n_other), s>>>(a);
            });
            if (e != cudaSuccess) return e;
            // the Gram was the last reader of this sampling set
            if (pipe && (e = cudaEventRecord(h->ev_free[a.sset], s)) != cudaSuccess) return e;
            e = L.run(NTC_K_FINISH, 0, [&] {
                k_heavy_reduce<RP><<<p.n_groups, kThreads, 0, s>>>(a);
                k_heavy_rowsum<RP><<<p.n_heavy, kThreads, 0, s>>>(a);
            });
            ++*L.launches;
            if (e != cudaSuccess) return e;
        }
    }
    if (fork && (e = cudaStreamWaitEvent(s, L.h->ev_join, 0)) != cudaSuccess) return e;
    const int nrows = p.n_light + p.n_heavy;
    if (!mask_only && nrows > 0) {
        constexpr int W = RowFinish<RP>::WARPS;
        e = L.run(NTC_K_FINISH, (int64_t)nrows * L.bpr, [&] {
            k_rows_finish<RP><<<(nrows + W - 1) / W, W * 32, RowFinish<RP>::bytes(), s>>>(a);
        });
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// Orders 2-4 take the register-row Gram with the number of other modes fixed
// at compile time; orders 5-8 stage factor rows in shared memory.
template <int RP, bool BF>
cudaError_t launch_mode_bf(int ew, const ModeArgs& a, const ModePlan& p, Launcher& L, bool mo) {
    if (ew == 8) return launch_mode_t<RP, 8, BF, 0>(a, p, L, mo);
    switch (a.n_other) {
        case 1: return launch_mode_t<RP, 4, BF, 1>(a, p, L, mo);
        case 2: return launch_mode_t<RP, 4, BF, 2>(a, p, L, mo);
        default: return launch_mode_t<RP, 4, BF, 3>(a, p, L, mo);
    }
}

template <int RP>
cudaError_t launch_mode_rp(int ew, bool bf, const ModeArgs& a, const ModePlan& p, Launcher& L, bool mo) {
    return bf ? launch_mode_bf<RP, true>(ew, a, p, L, mo) : launch_mode_bf<RP, false>(ew, a, p, L, mo);
}

}  // namespace ntc
