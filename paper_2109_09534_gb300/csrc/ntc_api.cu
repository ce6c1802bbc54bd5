// ntc_api.cu -- host orchestrator and C ABI (include/ntc.h) of the GB300
// library for AO accelerated stochastic nonnegative tensor completion
// (arXiv 2109.09534).  The handle owns device memory, buckets the observed
// entries, plans the per-mode row work (light rows: one block each; heavy
// rows: split into chunks) and enqueues Algorithm 2 around Algorithm 1 on one
// CUDA stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "aux_kernels.cuh"
#include "ntc_host.h"
#include "tiny_rows.cuh"

using namespace ntc;

namespace {

ntc_status fail(ntc_handle* h, ntc_status s, const std::string& msg) {
    if (h) h->err = msg;
    return s;
}

#define NTC_CUDA(h, call)                                                                   \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            return fail((h), e_ == cudaErrorMemoryAllocation ? NTC_ERR_OOM : NTC_ERR_CUDA,  \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                \
        }                                                                                   \
    } while (0)

int ew_of(int order) { return order <= 4 ? 4 : 8; }

int grid_for(int64_t n, int per_block = 256, int cap = 152 * 16) {
    int64_t g = (n + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

cudaError_t launch_mode(int rp, int ew, bool bf, const ModeArgs& a, const ModePlan& p, Launcher& L, bool mo) {
    switch (rp) {
        case 8: return launch_mode_rp<8>(ew, bf, a, p, L, mo);
        case 16: return launch_mode_rp<16>(ew, bf, a, p, L, mo);
        case 32: return launch_mode_rp<32>(ew, bf, a, p, L, mo);
        default: return launch_mode_rp<64>(ew, bf, a, p, L, mo);
    }
}

int partial_width(int rp) {
    const int T = rp / 8;
    return T * (T + 1) / 2 * 64 + rp;
}

// ---- per-(mode, c) plan ------------------------------------------------------
ntc_status build_plan(ntc_handle* h, int mode, double c) {
    ModePlan& p = h->plan[mode];
    const bool tiny = h->tiny_rows && ew_of(h->order) == 4;
    if (p.valid && p.c == c && p.heavy_threshold == h->heavy_threshold && p.chunk == h->chunk &&
        p.bracket_z == h->bracket_z && p.tiny == tiny)
        return NTC_OK;
    p.valid = false;
    const std::vector<int64_t>& rp = h->row_ptr_h[mode];
    const int64_t P = h->dims[mode];
    std::vector<std::pair<int64_t, int32_t>> light, tinyv;   // (n, row)
    std::vector<int32_t> light_k;
    std::vector<int4> chunks, caps, heavy, hcand, groups;
    std::vector<int32_t> voff;   // epoch-permutation variant: chunk list starts
    std::vector<int2> heavy_groups;
    std::vector<longlong2> brk;
    int64_t visits = 0, visits_heavy = 0, updated = 0, skipped = 0, cand_total = 0, extra_total = 0;
    // rows in descending order of observations (ties by row), so that the
    // per-row blocks of the longest split rows start first
    std::vector<int32_t> order((size_t)P);
    for (int64_t r = 0; r < P; ++r) order[(size_t)r] = (int32_t)r;
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
        return rp[(size_t)x + 1] - rp[(size_t)x] > rp[(size_t)y + 1] - rp[(size_t)y];
    });
    for (const int32_t r : order) {
        const int64_t n = rp[r + 1] - rp[r];
        const int64_t k = (int64_t)std::floor(c * (double)n);   // B_{l,p} = floor(c ||M(p,:)||_0)
        if (k == 0) {
            ++skipped;
            continue;
        }
        ++updated;
        visits += k;
        if (n <= h->heavy_threshold) {
            if (tiny && n <= kTinyMax) tinyv.push_back({n, (int32_t)r});
            else light.push_back({n, (int32_t)r});
            continue;
        }
        visits_heavy += k;
        const int hidx = (int)heavy.size();
        const int64_t nch = (n + h->chunk - 1) / h->chunk;
        long long lo, hi;
        if (k == n) {
            lo = hi = 1ll << 32;
        } else {
            const double q = (double)k / (double)n;
            const double sd = std::sqrt(q * (1.0 - q) / (double)n);
            const double delta = h->bracket_z * sd;
            const double two32 = 4294967296.0;
            double l = std::max(0.0, q - delta) * two32, u = std::min(1.0, q + delta) * two32;
            lo = (long long)std::floor(l);
            hi = (long long)std::ceil(u);
            if (h->bracket_z <= 0.0) lo = hi = (long long)std::floor(q * two32);
            lo = std::max(0ll, std::min(lo, 1ll << 32));
            hi = std::max(lo, std::min(hi, 1ll << 32));
        }
        const int cb = (int)chunks.size();
        const int64_t cbeg = cand_total;
        for (int64_t j = 0; j < nch; ++j) {
            const int64_t pb = rp[r] + (j * n) / nch, pe = rp[r] + ((j + 1) * n) / nch;
            const double expect = (double)(pe - pb) * (double)(hi - lo) / 4294967296.0;
            int cap = hi > lo ? (int)std::ceil(expect + 8.0 * std::sqrt(expect) + 8.0) : 0;
            cap = (cap + 3) & ~3;
            chunks.push_back(make_int4(hidx, (int)pb, (int)pe, (int)cand_total));
            voff.push_back((int32_t)(rp[r] + (k * j) / nch));
            caps.push_back(make_int4(cap, 0, 0, 0));
            cand_total += cap;
        }
        heavy.push_back(make_int4((int)r, (int)k, cb, (int)chunks.size()));
        {
            const int nitems = (int)chunks.size() - cb + 1;   // chunks, then the chosen candidates
            const int g0 = (int)groups.size();
            for (int i = 0; i < nitems; i += kReduceGroup)
                groups.push_back(make_int4(hidx, i, std::min(nitems, i + kReduceGroup), 0));
            heavy_groups.push_back(make_int2(g0, (int)groups.size()));
        }
        brk.push_back(make_longlong2(lo, hi));
        const int ccap = (int)(cand_total - cbeg);
        hcand.push_back(make_int4((int)cbeg, ccap, (int)extra_total, ccap));
        extra_total += ccap;
    }
    // longest light rows first: better tail behaviour, same results
    std::stable_sort(light.begin(), light.end(),
                     [](const std::pair<int64_t, int32_t>& x, const std::pair<int64_t, int32_t>& y) {
                         return x.first > y.first;
                     });
    std::vector<int32_t> lrows(light.size());
    light_k.resize(light.size());
    for (size_t i = 0; i < light.size(); ++i) {
        lrows[i] = light[i].second;
        light_k[i] = (int32_t)std::floor(c * (double)light[i].first);
    }
    // rows of one warp each, in the same order (longest first)
    std::vector<int32_t> trows(tinyv.size()), tk(tinyv.size());
    for (size_t i = 0; i < tinyv.size(); ++i) {
        trows[i] = tinyv[i].second;
        tk[i] = (int32_t)std::floor(c * (double)tinyv[i].first);
    }
    if (cand_total >= (1ll << 31) || extra_total >= (1ll << 31))
        return fail(h, NTC_ERR_ARG, "sampler bracket too wide for this row size");
    auto up = [&](DevMem& m, const void* src, size_t bytes) -> cudaError_t {
        cudaError_t e = m.ensure(bytes);
        if (e != cudaSuccess || bytes == 0) return e;
        return cudaMemcpyAsync(m.p, src, bytes, cudaMemcpyHostToDevice, h->stream);
    };
    NTC_CUDA(h, up(p.light_rows, lrows.data(), lrows.size() * 4));
    NTC_CUDA(h, up(p.light_k, light_k.data(), light_k.size() * 4));
    NTC_CUDA(h, up(p.tiny_rows, trows.data(), trows.size() * 4));
    NTC_CUDA(h, up(p.tiny_k, tk.data(), tk.size() * 4));
    NTC_CUDA(h, up(p.chunks, chunks.data(), chunks.size() * sizeof(int4)));
    NTC_CUDA(h, up(p.vis_off, voff.data(), voff.size() * sizeof(int32_t)));
    NTC_CUDA(h, up(p.chunk_caps, caps.data(), caps.size() * sizeof(int4)));
    NTC_CUDA(h, up(p.heavy, heavy.data(), heavy.size() * sizeof(int4)));
    NTC_CUDA(h, up(p.bracket, brk.data(), brk.size() * sizeof(longlong2)));
    NTC_CUDA(h, up(p.heavy_cand, hcand.data(), hcand.size() * sizeof(int4)));
    NTC_CUDA(h, up(p.groups, groups.data(), groups.size() * sizeof(int4)));
    NTC_CUDA(h, up(p.heavy_groups, heavy_groups.data(), heavy_groups.size() * sizeof(int2)));
    NTC_CUDA(h, cudaStreamSynchronize(h->stream));   // host vectors go out of scope
    p.c = c;
    p.heavy_threshold = h->heavy_threshold;
    p.chunk = h->chunk;
    p.bracket_z = h->bracket_z;
    p.visits = visits;
    p.visits_heavy = visits_heavy;
    p.rows_updated = updated;
    p.rows_skipped = skipped;
    p.n_light = (int)light.size();
    p.n_tiny = (int)tinyv.size();
    p.n_tiny_big = 0;
    while (p.n_tiny_big < p.n_tiny && tk[(size_t)p.n_tiny_big] > kTinyKForm) ++p.n_tiny_big;
    p.tiny = tiny;
    p.n_heavy = (int)heavy.size();
    p.n_chunks = (int)chunks.size();
    p.n_groups = (int)groups.size();
    p.cand_total = cand_total;
    p.extra_total = extra_total;
    // scratch sized for this plan
    for (int b = 0; b < (h->pipeline ? 2 : 1); ++b) {
        NTC_CUDA(h, h->vis[b].ensure(sizeof(uint32_t) * (size_t)std::max<int64_t>(h->nnz, 1)));
        NTC_CUDA(h, h->vis_cnt[b].ensure(sizeof(uint32_t) * (size_t)std::max(p.n_chunks, 1)));
        NTC_CUDA(h, h->cand_cnt[b].ensure(sizeof(uint32_t) * (size_t)std::max(p.n_chunks, 1)));
        NTC_CUDA(h, h->cand[b].ensure(sizeof(unsigned long long) * (size_t)std::max<int64_t>(cand_total, 1)));
        NTC_CUDA(h, h->extra[b].ensure(sizeof(uint32_t) * (size_t)std::max<int64_t>(extra_total, 1)));
        NTC_CUDA(h, h->extra_cnt[b].ensure(sizeof(uint32_t) * (size_t)std::max(p.n_heavy, 1)));
        NTC_CUDA(h, h->flags[b].ensure(sizeof(uint32_t) * (size_t)std::max(p.n_heavy, 1)));
    }
    NTC_CUDA(h, h->partial.ensure(sizeof(float) * (size_t)partial_width(h->rp) *
                                  (size_t)std::max(p.n_chunks + p.n_heavy, 1)));
    NTC_CUDA(h, h->partial2.ensure(sizeof(float) * (size_t)partial_width(h->rp) * (size_t)std::max(p.n_groups, 1)));
    NTC_CUDA(h, h->row_sum.ensure(sizeof(float) * (size_t)partial_width(h->rp) *
                                  (size_t)std::max(p.n_light + p.n_heavy, 1)));
    p.valid = true;
    return NTC_OK;
}

ModeArgs mode_args(ntc_handle* h, int mode, int inner, uint64_t seed, uint64_t ao_iter) {
    ModeArgs a;
    memset(&a, 0, sizeof(a));
    const ModePlan& p = h->plan[mode];
    int o = 0;
    for (int i = 0; i < h->order; ++i) {
        if (i == mode) continue;
        a.other[o++] = h->storage_bf16 ? (const void*)h->Ub[i].p : (const void*)h->U[i].p;
    }
    a.n_other = h->order - 1;
    int64_t nh = 64;   // the kernels cap this at their own resident-row count
    for (int i = 0; i < h->order; ++i)
        if (i != mode) nh = std::min<int64_t>(nh, h->dims[i]);
    a.nhot = (int)nh;
    a.rank = h->rank;
    a.rp = h->rp;
    a.lambda = (float)h->lambda;
    a.lambda_d = h->lambda;
    a.power_iters = h->power_iters;
    a.U = h->U[mode].as<float>();
    a.inv_self = h->inv_dev[mode].as<int32_t>();
    a.Ub = h->storage_bf16 ? h->Ub[mode].as<uint16_t>() : nullptr;
    a.Y = h->max_inner > 1 ? h->Y.as<float>() : nullptr;
    a.read_y = inner > 0 ? 1 : 0;
    a.write_y = inner + 1 < h->max_inner ? 1 : 0;
    a.row_ptr = h->row_ptr[mode].as<int64_t>();
    a.bucket = h->bucket[mode].p;
    a.ss.mode = (uint32_t)mode;
    a.ss.iter = (uint32_t)ao_iter;
    a.ss.inner = (uint32_t)inner;
    a.ss.k0 = (uint32_t)seed;
    a.ss.k1 = (uint32_t)(seed >> 32);
    a.light_rows = p.light_rows.as<int32_t>();
    a.light_k = p.light_k.as<int32_t>();
    a.tiny_rows = p.tiny_rows.as<int32_t>();
    a.tiny_k = p.tiny_k.as<int32_t>();
    a.n_tiny = p.n_tiny;
    a.tiny_begin = 0;
    a.tiny_end = p.n_tiny;
    a.chunks = p.chunks.as<int4>();
    a.chunk_caps = p.chunk_caps.as<int4>();
    a.heavy = p.heavy.as<int4>();
    a.heavy_bracket = p.bracket.as<longlong2>();
    a.heavy_cand = p.heavy_cand.as<int4>();
    a.n_chunks = p.n_chunks;
    a.n_heavy = p.n_heavy;
    const int sb = h->pipeline ? (int)(h->upd & 1) : 0;   // sampling set of this update
    a.vis = h->vis[sb].as<uint32_t>();
    a.vis_cnt = h->vis_cnt[sb].as<uint32_t>();
    a.cand = h->cand[sb].as<unsigned long long>();
    a.cand_cnt = h->cand_cnt[sb].as<uint32_t>();
    a.extra = h->extra[sb].as<uint32_t>();
    a.extra_cnt = h->extra_cnt[sb].as<uint32_t>();
    a.flags = h->flags[sb].as<uint32_t>();
    a.sset = sb;
    a.partial = h->partial.as<float>();
    a.groups = p.groups.as<int4>();
    a.heavy_groups = p.heavy_groups.as<int2>();
    a.n_groups = p.n_groups;
    a.partial2 = h->partial2.as<float>();
    a.row_sum = h->row_sum.as<float>();
    a.n_light = p.n_light;
    a.stat_fallback = h->stat.as<unsigned long long>();
    a.stat_wait = h->stat.as<unsigned long long>() + 1;
    a.test_stall_cycles = h->test_stall_cycles;
    a.mask_out = nullptr;
    return a;
}

// Algorithmic bytes (the model of the sampled visits): per visit the other
// modes' indices, the value and the other modes' factor rows; per row update
// the row pointer, the master row read and written (plus the bfloat16 copy
// and the extrapolation row when they exist).
Launcher make_launcher(ntc_handle* h) {
    const int64_t N = h->order, R = h->rank, sz = h->storage_bf16 ? 2 : 4;
    Launcher L;
    L.h = h;
    L.s = h->stream;
    L.launches = &h->stats.kernel_launches;
    L.bpv = (N - 1) * 4 + 4 + (N - 1) * R * sz;
    L.bpr = 8 + 4 * R + 4 * R + (h->storage_bf16 ? 2 * R : 0) + (h->max_inner > 1 ? 8 * R : 0);
    return L;
}

// Algorithm 1 on one mode at AO iteration ao_iter.
// Epoch-permutation variant: epoch floor(k / T) and slot (k mod T) * MAX_INNER
// + inner of AO iteration k, T = ceil(1/c) AO iterations per epoch.
void set_perm(const ntc_handle* h, ModeArgs& a, const ModePlan& p, double c, uint64_t ao_iter, int inner) {
    if (!h->sampler) return;
    const uint64_t T = (uint64_t)std::ceil(1.0 / c - 1e-12);
    a.perm = 1;
    a.perm_epoch = (uint32_t)(ao_iter / T);
    a.perm_slot = (int64_t)(ao_iter % T) * h->max_inner + inner;
    a.vis_off = p.vis_off.as<int32_t>();
}

ntc_status run_snmc(ntc_handle* h, int mode, double c, uint64_t seed, uint64_t ao_iter) {
    ntc_status st = build_plan(h, mode, c);
    if (st != NTC_OK) return st;
    const ModePlan& p = h->plan[mode];
    Launcher L = make_launcher(h);
    if (h->power_warm && !h->warm_ready[mode]) {   // first warm use: v0 = ones/sqrt(R)
        NTC_CUDA(h, h->vwarm[mode].ensure(sizeof(float) * (size_t)(h->dims[mode] * h->rp)));
        k_fill_warm<<<grid_for(h->dims[mode] * h->rp), 256, 0, h->stream>>>(h->vwarm[mode].as<float>(), h->dims[mode],
                                                                             h->rank, h->rp);
        NTC_CUDA(h, cudaGetLastError());
        h->warm_ready[mode] = true;
    }
    for (int l = 0; l < h->max_inner; ++l) {
        ModeArgs a = mode_args(h, mode, l, seed, ao_iter);
        a.vwarm = h->power_warm ? h->vwarm[mode].as<float>() : nullptr;
        set_perm(h, a, p, c, ao_iter, l);
        NTC_CUDA(h, launch_mode(h->rp, ew_of(h->order), h->storage_bf16 != 0, a, p, L, false));
        h->upd += 1;
        h->stats.visits += p.visits;
        h->stats.visits_heavy += p.visits_heavy;
        h->stats.rows_updated += p.rows_updated;
        h->stats.rows_skipped += p.rows_skipped;
        h->stats.alg_bytes += p.visits * L.bpv + p.rows_updated * L.bpr;
    }
    return NTC_OK;
}

ntc_status check_ready(ntc_handle* h) {
    if (!h) return NTC_ERR_ARG;
    if (h->nnz < 0) return fail(h, NTC_ERR_STATE, "ntc_set_observed has not been called");
    return NTC_OK;
}

// Device counters: [0] rows that used the exact fallback selector and [1]
// tensor-core Gram blocks whose bounded wait gave up, both for the current
// call; [2] the latter since the handle was created (never cleared).
ntc_status reset_stats(ntc_handle* h) {
    h->stats = ntc_stats{};
    if (!h->stat.p) {
        NTC_CUDA(h, h->stat.ensure(3 * sizeof(unsigned long long)));
        NTC_CUDA(h, cudaMemsetAsync(h->stat.p, 0, 3 * sizeof(unsigned long long), h->stream));
        return NTC_OK;
    }
    NTC_CUDA(h, cudaMemsetAsync(h->stat.p, 0, 2 * sizeof(unsigned long long), h->stream));
    return NTC_OK;
}

// After the handle's stream has been synchronised: a tensor-core Gram block
// that gave up waiting since the last check left a partial unwritten, so the
// updates enqueued since then are not valid.  Reported once per new timeout.
ntc_status check_faults(ntc_handle* h) {
    if (!h->stat.p) return NTC_OK;
    unsigned long long total = 0;
    NTC_CUDA(h, cudaMemcpyAsync(&total, h->stat.as<unsigned long long>() + 2, sizeof(total),
                                cudaMemcpyDeviceToHost, h->stream));
    NTC_CUDA(h, cudaStreamSynchronize(h->stream));
    if (total > h->faults_seen) {
        const unsigned long long fresh = total - h->faults_seen;
        h->faults_seen = total;
        return fail(h, NTC_ERR_CUDA,
                    "tensor-core Gram: " + std::to_string(fresh) +
                        " block(s) gave up a bounded wait for their MMAs; the factors updated since the last "
                        "successful check are not valid");
    }
    return NTC_OK;
}

// Stable LSD radix sort of (key = row index of `mode`, payload = entry index).
// Bucket of `mode` by a stable LSD radix sort of (row, entry) pairs: the
// first pass builds the 16-byte entries from the COO, the last writes them in
// bucket order (passes alternate between entry_tmp and the bucket so that the
// last lands in the bucket).  *keys_out: the sorted rows.
ntc_status sort_mode_entries(ntc_handle* h, int mode, const RowMaps& maps, DevMem& k0, DevMem& k1, DevMem& hist,
                             DevMem& sums, uint32_t** keys_out) {
    const int64_t n = h->nnz;
    cudaStream_t s = h->stream;
    // once per process (admissions of a server may bucket on several threads)
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [] { attr_err = set_smem(k_radix_scatter_ent, kEntScatterSmem); });
    NTC_CUDA(h, attr_err);
    NTC_CUDA(h, h->entry_tmp.ensure(sizeof(uint4) * (size_t)std::max<int64_t>(n, 1)));
    int bits = 1;
    while (bits < 31 && (1ll << bits) < h->dims[mode]) ++bits;
    const int passes = (bits + 7) / 8;
    const int ntiles = (int)((n + kSortTile - 1) / kSortTile);
    const int64_t nh = (int64_t)ntiles * 256;
    const int nb = (int)((nh + kScanBlock - 1) / kScanBlock);
    uint32_t *kin = k0.as<uint32_t>(), *kout = k1.as<uint32_t>();
    uint4* bucket = h->bucket[mode].as<uint4>();
    uint4* tmp = h->entry_tmp.as<uint4>();
    // keys and entries in input order first (coalesced), into the buffer that
    // leaves the last pass's output in the bucket
    uint4* pin = passes % 2 == 1 ? tmp : bucket;
    uint4* pout = pin == bucket ? tmp : bucket;
    k_build_keys_entries<<<grid_for(n), 256, 0, s>>>(h->coo_idx.as<int32_t>(), h->coo_val.as<float>(), n, h->order, mode,
                                                     maps, k0.as<uint32_t>(), pin);
    for (int pass = 0; pass < passes && n > 0; ++pass) {
        const int shift = 8 * pass;
        k_radix_hist<<<ntiles, kThreads, 0, s>>>(kin, n, shift, hist.as<uint32_t>(), ntiles);
        k_scan_sums<<<nb, kThreads, 0, s>>>(hist.as<uint32_t>(), nh, sums.as<uint32_t>());
        k_scan_top<<<1, kThreads, 0, s>>>(sums.as<uint32_t>(), nb);
        k_scan_apply<<<nb, kThreads, 0, s>>>(hist.as<uint32_t>(), nh, sums.as<uint32_t>(), hist.as<uint32_t>() + nh);
        k_radix_scatter_ent<<<ntiles, kThreads, kEntScatterSmem, s>>>(kin, pin, kout, pout, n, shift,
                                                                      hist.as<uint32_t>() + nh, ntiles);
        std::swap(kin, kout);
        pin = pout;
        pout = pout == bucket ? tmp : bucket;
    }
    NTC_CUDA(h, cudaGetLastError());
    *keys_out = kin;
    return NTC_OK;
}

ntc_status sort_mode(ntc_handle* h, int mode, DevMem& k0, DevMem& k1, DevMem& v0, DevMem& v1, DevMem& hist,
                     DevMem& sums, uint32_t** keys_out, uint32_t** perm_out) {
    const int64_t n = h->nnz;
    cudaStream_t s = h->stream;
    k_extract_keys<<<grid_for(n), 256, 0, s>>>(h->coo_idx.as<int32_t>(), n, h->order, mode, k0.as<uint32_t>(),
                                               v0.as<uint32_t>());
    int bits = 1;
    while (bits < 31 && (1ll << bits) < h->dims[mode]) ++bits;
    const int passes = (bits + 7) / 8;
    const int ntiles = (int)((n + kSortTile - 1) / kSortTile);
    const int64_t nh = (int64_t)ntiles * 256;
    const int nb = (int)((nh + kScanBlock - 1) / kScanBlock);
    uint32_t *kin = k0.as<uint32_t>(), *vin = v0.as<uint32_t>(), *kout = k1.as<uint32_t>(), *vout = v1.as<uint32_t>();
    for (int pass = 0; pass < passes && n > 0; ++pass) {
        const int shift = 8 * pass;
        k_radix_hist<<<ntiles, kThreads, 0, s>>>(kin, n, shift, hist.as<uint32_t>(), ntiles);
        k_scan_sums<<<nb, kThreads, 0, s>>>(hist.as<uint32_t>(), nh, sums.as<uint32_t>());
        k_scan_top<<<1, kThreads, 0, s>>>(sums.as<uint32_t>(), nb);
        k_scan_apply<<<nb, kThreads, 0, s>>>(hist.as<uint32_t>(), nh, sums.as<uint32_t>(),
                                             hist.as<uint32_t>() + nh);
        k_radix_scatter<<<ntiles, kThreads, 0, s>>>(kin, vin, kout, vout, n, shift, hist.as<uint32_t>() + nh, ntiles);
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    NTC_CUDA(h, cudaGetLastError());
    *keys_out = kin;
    *perm_out = vin;
    return NTC_OK;
}

// Factor `mode` in original row order, [dims][rank] float32 (host).
ntc_status download_factor(ntc_handle* h, int mode, float* out) {
    const int64_t I = h->dims[mode];
    const int R = h->rank, RP = h->rp;
    std::vector<float> tmp((size_t)I * RP);
    NTC_CUDA(h, cudaMemcpyAsync(tmp.data(), h->U[mode].p, sizeof(float) * tmp.size(), cudaMemcpyDeviceToHost,
                                h->stream));
    NTC_CUDA(h, cudaStreamSynchronize(h->stream));
    const std::vector<int32_t>& inv = h->inv_h[mode];
    for (int64_t r = 0; r < I; ++r) memcpy(out + r * R, tmp.data() + (size_t)inv[(size_t)r] * RP, sizeof(float) * R);
    return check_faults(h);
}

// Store `in` ([dims][rank], original row order, host) as factor `mode`.
ntc_status upload_factor(ntc_handle* h, int mode, const float* in) {
    const int64_t I = h->dims[mode];
    const int R = h->rank, RP = h->rp;
    std::vector<float> tmp((size_t)I * RP, 0.f);
    const std::vector<int32_t>& inv = h->inv_h[mode];
    for (int64_t r = 0; r < I; ++r) memcpy(tmp.data() + (size_t)inv[(size_t)r] * RP, in + r * R, sizeof(float) * R);
    NTC_CUDA(h, cudaMemcpyAsync(h->U[mode].p, tmp.data(), sizeof(float) * tmp.size(), cudaMemcpyHostToDevice,
                                h->stream));
    if (h->storage_bf16) {
        const int64_t m = I * RP;
        k_to_bf16<<<grid_for(m), 256, 0, h->stream>>>(h->U[mode].as<float>(), h->Ub[mode].as<uint16_t>(), m);
        NTC_CUDA(h, cudaGetLastError());
    }
    NTC_CUDA(h, cudaStreamSynchronize(h->stream));
    return NTC_OK;
}

ntc_status upload_maps(ntc_handle* h, int mode) {
    const size_t I = (size_t)h->dims[mode];
    NTC_CUDA(h, h->inv_dev[mode].ensure(sizeof(int32_t) * I));
    NTC_CUDA(h, h->rows_dev[mode].ensure(sizeof(int32_t) * I));
    NTC_CUDA(h, cudaMemcpyAsync(h->inv_dev[mode].p, h->inv_h[mode].data(), sizeof(int32_t) * I,
                                cudaMemcpyHostToDevice, h->stream));
    NTC_CUDA(h, cudaMemcpyAsync(h->rows_dev[mode].p, h->rows_h[mode].data(), sizeof(int32_t) * I,
                                cudaMemcpyHostToDevice, h->stream));
    NTC_CUDA(h, cudaStreamSynchronize(h->stream));
    return NTC_OK;
}

ntc_status set_observed_impl(ntc_handle* h, int64_t nnz, const int32_t* idx, const float* vals, bool dev) {
    if (!h) return NTC_ERR_ARG;
    if (nnz < 0 || nnz >= (1ll << 31) || (nnz > 0 && (!idx || !vals)))
        return fail(h, NTC_ERR_ARG, "nnz must be in [0, 2^31) with non-null idx and vals");
    cudaStream_t s = h->stream;
    const int N = h->order;
    // stage and validate before touching the handle's current data
    DevMem& cidx = h->stage_idx;
    DevMem& cval = h->stage_val;
    NTC_CUDA(h, cidx.ensure(sizeof(int32_t) * (size_t)std::max<int64_t>(nnz * N, 1)));
    NTC_CUDA(h, cval.ensure(sizeof(float) * (size_t)std::max<int64_t>(nnz, 1)));
    if (nnz > 0) {
        const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        NTC_CUDA(h, cudaMemcpyAsync(cidx.p, idx, sizeof(int32_t) * nnz * N, kind, s));
        NTC_CUDA(h, cudaMemcpyAsync(cval.p, vals, sizeof(float) * nnz, kind, s));
    }
    DevMem& bad = h->bad_flag;
    NTC_CUDA(h, bad.ensure(sizeof(unsigned)));
    NTC_CUDA(h, cudaMemsetAsync(bad.p, 0, sizeof(unsigned), s));
    if (nnz > 0) k_validate<<<grid_for(nnz), 256, 0, s>>>(cidx.as<int32_t>(), nnz, N, h->dims_dev.as<int64_t>(),
                                                         bad.as<unsigned>());
    unsigned bad_h = 0;
    NTC_CUDA(h, cudaMemcpyAsync(&bad_h, bad.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    NTC_CUDA(h, cudaStreamSynchronize(s));
    if (bad_h) return fail(h, NTC_ERR_INDEX, "an observed index is out of range");
    // commit (the previous COO becomes the next call's staging buffer)
    std::swap(h->coo_idx.p, cidx.p);
    std::swap(h->coo_idx.bytes, cidx.bytes);
    std::swap(h->coo_val.p, cval.p);
    std::swap(h->coo_val.bytes, cval.bytes);
    h->nnz = nnz;
    h->ao_iter = 0;
    for (int i = 0; i < N; ++i) h->warm_ready[i] = false;   // new observations: cold power method again
    for (int i = 0; i < N; ++i) h->plan[i].valid = false;
    // factors set by the caller keep their values across the renumbering
    std::vector<std::vector<float>> kept(N);
    for (int i = 0; i < N; ++i) {
        if (!h->factor_set[i]) continue;
        kept[i].resize((size_t)h->dims[i] * h->rank);
        ntc_status st = download_factor(h, i, kept[i].data());
        if (st != NTC_OK) return st;
    }
    // observation counts per row -> storage order (most frequent first, ties by row)
    for (int i = 0; i < N; ++i) {
        const int64_t I = h->dims[i];
        DevMem& cnt = h->row_cnt;
        NTC_CUDA(h, cnt.ensure(sizeof(uint32_t) * (size_t)I));
        NTC_CUDA(h, cudaMemsetAsync(cnt.p, 0, sizeof(uint32_t) * (size_t)I, s));
        // (few blocks when each flushes a shared histogram of the whole mode)
        const int cgrid = I <= kCountSmemRows ? grid_for(nnz, 256, 152 * 2) : grid_for(nnz);
        if (nnz > 0)
            k_count_rows<<<cgrid, 256, 0, s>>>(h->coo_idx.as<int32_t>(), nnz, N, i, I, cnt.as<uint32_t>());
        NTC_CUDA(h, cudaGetLastError());
        std::vector<uint32_t> c((size_t)I);
        NTC_CUDA(h, cudaMemcpyAsync(c.data(), cnt.p, sizeof(uint32_t) * (size_t)I, cudaMemcpyDeviceToHost, s));
        NTC_CUDA(h, cudaStreamSynchronize(s));
        std::vector<int32_t>& rows = h->rows_h[i];
        rows.resize((size_t)I);
        for (int64_t r = 0; r < I; ++r) rows[(size_t)r] = (int32_t)r;
        std::stable_sort(rows.begin(), rows.end(), [&](int32_t x, int32_t y) { return c[(size_t)x] > c[(size_t)y]; });
        h->inv_h[i].resize((size_t)I);
        for (int64_t j = 0; j < I; ++j) h->inv_h[i][(size_t)rows[(size_t)j]] = (int32_t)j;
        ntc_status st = upload_maps(h, i);
        if (st != NTC_OK) return st;
    }
    RowMaps maps;
    for (int i = 0; i < N; ++i) maps.inv[i] = h->inv_dev[i].as<int32_t>();
    // per-mode buckets
    DevMem &k0 = h->sort_k0, &k1 = h->sort_k1, &v0 = h->sort_v0, &v1 = h->sort_v1, &hist = h->sort_hist,
           &sums = h->sort_sums;
    const size_t nb4 = sizeof(uint32_t) * (size_t)std::max<int64_t>(nnz, 1);
    NTC_CUDA(h, k0.ensure(nb4));
    NTC_CUDA(h, k1.ensure(nb4));
    if (!(ew_of(N) == 4 && !h->keep_perm)) {   // the permutation path (orders > 4 or a kept permutation)
        NTC_CUDA(h, v0.ensure(nb4));
        NTC_CUDA(h, v1.ensure(nb4));
    }
    const int64_t ntiles = (nnz + kSortTile - 1) / kSortTile;
    NTC_CUDA(h, hist.ensure(sizeof(uint32_t) * (size_t)std::max<int64_t>(2 * ntiles * 256, 1)));
    NTC_CUDA(h, sums.ensure(sizeof(uint32_t) * (size_t)std::max<int64_t>(ntiles * 256 / kScanBlock + 2, 1)));
    const int EW = ew_of(N);
    for (int i = 0; i < N; ++i) {
        uint32_t *keys = nullptr, *perm = nullptr;
        NTC_CUDA(h, h->bucket[i].ensure((size_t)EW * 4 * (size_t)std::max<int64_t>(nnz, 1)));
        // orders 2-4 without a kept permutation: entries ride through the sort
        const bool ride = EW == 4 && !h->keep_perm;
        ntc_status st = ride ? sort_mode_entries(h, i, maps, k0, k1, hist, sums, &keys)
                             : sort_mode(h, i, k0, k1, v0, v1, hist, sums, &keys, &perm);
        if (st != NTC_OK) return st;
        NTC_CUDA(h, h->row_ptr[i].ensure(sizeof(int64_t) * (size_t)(h->dims[i] + 1)));
        k_row_ptr<<<grid_for(nnz + 1), 256, 0, s>>>(keys, nnz, h->dims[i], h->row_ptr[i].as<int64_t>());
        if (nnz > 0 && !ride) {
            NTC_CUDA(h, h->entry_tmp.ensure((size_t)EW * 4 * (size_t)nnz));
            if (EW == 4) {
                k_build_entries<4><<<grid_for(nnz), 256, 0, s>>>(h->coo_idx.as<int32_t>(), h->coo_val.as<float>(), nnz,
                                                                 N, i, maps, h->entry_tmp.as<Entry<4>>());
                k_gather_entries<4><<<grid_for(nnz), 256, 0, s>>>(h->entry_tmp.as<Entry<4>>(), perm, nnz,
                                                                  h->bucket[i].as<Entry<4>>());
            } else {
                k_build_entries<8><<<grid_for(nnz), 256, 0, s>>>(h->coo_idx.as<int32_t>(), h->coo_val.as<float>(), nnz,
                                                                 N, i, maps, h->entry_tmp.as<Entry<8>>());
                k_gather_entries<8><<<grid_for(nnz), 256, 0, s>>>(h->entry_tmp.as<Entry<8>>(), perm, nnz,
                                                                  h->bucket[i].as<Entry<8>>());
            }
        }
        if (h->keep_perm) {
            NTC_CUDA(h, h->perm[i].ensure(nb4));
            NTC_CUDA(h, cudaMemcpyAsync(h->perm[i].p, perm, nb4, cudaMemcpyDeviceToDevice, s));
        } else {
            h->perm[i].release();
        }
        h->row_ptr_h[i].resize((size_t)h->dims[i] + 1);
        NTC_CUDA(h, cudaMemcpyAsync(h->row_ptr_h[i].data(), h->row_ptr[i].p, sizeof(int64_t) * (h->dims[i] + 1),
                                    cudaMemcpyDeviceToHost, s));
        NTC_CUDA(h, cudaGetLastError());
    }
    // initial factors for modes not set by the caller
    DevMem part, tot;
    NTC_CUDA(h, part.ensure(sizeof(double) * 1024));
    NTC_CUDA(h, tot.ensure(sizeof(double)));
    const int gb = grid_for(nnz, 256, 1024);
    k_sum_f32<<<gb, kThreads, 0, s>>>(h->coo_val.as<float>(), nnz, part.as<double>());
    k_sum_partials<<<1, kThreads, 0, s>>>(part.as<double>(), gb, tot.as<double>());
    for (int i = 0; i < N; ++i) {
        if (h->factor_set[i]) {
            ntc_status st = upload_factor(h, i, kept[i].data());
            if (st != NTC_OK) return st;
            continue;
        }
        k_init_factor<<<grid_for(h->dims[i] * h->rp), 256, 0, s>>>(
            h->U[i].as<float>(), h->storage_bf16 ? h->Ub[i].as<uint16_t>() : nullptr, h->dims[i], h->rank, h->rp, i,
            tot.as<double>(), nnz, N, (uint32_t)h->init_seed, (uint32_t)(h->init_seed >> 32),
            h->rows_dev[i].as<int32_t>());
    }
    NTC_CUDA(h, cudaGetLastError());
    NTC_CUDA(h, cudaStreamSynchronize(s));
    if (!h->cache_staging) {
        for (DevMem* m : {&h->stage_idx, &h->stage_val, &h->sort_k0, &h->sort_k1, &h->sort_v0, &h->sort_v1,
                          &h->sort_hist, &h->sort_sums, &h->row_cnt, &h->entry_tmp})
            m->release();
    }
    return NTC_OK;
}

FactorSet factor_set(ntc_handle* h) {
    FactorSet f;
    for (int i = 0; i < h->order; ++i) {
        f.U[i] = h->U[i].as<float>();
        f.inv[i] = h->inv_dev[i].as<int32_t>();
    }
    for (int i = 0; i < kMaxOrder; ++i) f.dims[i] = i < h->order ? h->dims[i] : 0;
    f.order = h->order;
    f.R = h->rank;
    f.rp = h->rp;
    return f;
}

}  // namespace

// ---- serving-runtime entry points (declared in ntc_host.h) ---------------------
namespace ntc {

cudaError_t rmse_enqueue(ntc_handle* h, const int32_t* idx, const float* vals, int64_t n, double* scratch,
                         double* host_sum) {
    const int gb = grid_for(n, 256, kRmseScratch - 1);
    k_sq_resid<<<gb, kThreads, 0, h->stream>>>(factor_set(h), idx, vals, n, scratch);
    k_sum_partials<<<1, kThreads, 0, h->stream>>>(scratch, gb, scratch + (kRmseScratch - 1));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(host_sum, scratch + (kRmseScratch - 1), sizeof(double), cudaMemcpyDeviceToHost,
                           h->stream);
}

size_t factor_table_bytes() { return sizeof(FactorSet); }

int64_t snapshot_floats(const ntc_handle* h) {
    int64_t n = 0;
    for (int i = 0; i < h->order; ++i) n += h->dims[i] * h->rp;
    return n;
}

cudaError_t snapshot_factors(ntc_handle* h, float* dst) {
    for (int i = 0; i < h->order; ++i) {
        const size_t b = sizeof(float) * (size_t)(h->dims[i] * h->rp);
        const cudaError_t e = cudaMemcpyAsync(dst, h->U[i].p, b, cudaMemcpyDeviceToDevice, h->stream);
        if (e != cudaSuccess) return e;
        dst += h->dims[i] * h->rp;
    }
    return cudaSuccess;
}

cudaError_t predict_multi(ntc_handle* const* handles, const float* const* snaps, int nh, const int32_t* slot,
                          const int32_t* idx, int64_t n, float* out, void* table, cudaStream_t s) {
    std::vector<FactorSet> t((size_t)nh);
    for (int j = 0; j < nh; ++j) {
        t[(size_t)j] = factor_set(handles[j]);
        if (snaps[j]) {
            const float* p = snaps[j];
            for (int i = 0; i < handles[j]->order; ++i) {
                t[(size_t)j].U[i] = p;
                p += handles[j]->dims[i] * handles[j]->rp;
            }
        }
    }
    // pageable source: the copy is staged before the call returns
    cudaError_t e = cudaMemcpyAsync(table, t.data(), sizeof(FactorSet) * (size_t)nh, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess || n == 0) return e;
    k_predict_multi<<<grid_for(n), 256, 0, s>>>(static_cast<const FactorSet*>(table), slot, idx, n, out);
    return cudaGetLastError();
}

ntc_status prepare_epoch(ntc_handle* h, double c) {
    ntc_status st = check_ready(h);
    if (st != NTC_OK) return st;
    if (!(c > 0.0 && c <= 1.0)) return fail(h, NTC_ERR_ARG, "c must be in (0, 1]");
    for (int i = 0; i < h->order; ++i)
        if ((st = build_plan(h, i, c)) != NTC_OK) return st;
    return reset_stats(h);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (the
// library links only the CUDA runtime).
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encode_tiled() {
    static std::once_flag once;
    static EncodeTiled fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}

cudaError_t gather_maps(ntc_handle* h, int mode, const GatherMaps** out) {
    const int want = h->storage_bf16 ? 2 : 1;
    if (h->gmaps_state[mode] != want) {
        EncodeTiled enc = encode_tiled();
        if (!enc) return cudaErrorNotSupported;
        int o = 0;
        for (int i = 0; i < h->order; ++i) {
            if (i == mode) continue;
            if (o >= 3) return cudaErrorInvalidValue;
            void* base = h->storage_bf16 ? h->Ub[i].p : h->U[i].p;
            const cuuint64_t dims[2] = {(cuuint64_t)h->rp, (cuuint64_t)h->dims[i]};
            const cuuint64_t strides[1] = {(cuuint64_t)h->rp * (h->storage_bf16 ? 2u : 4u)};
            const cuuint32_t box[2] = {(cuuint32_t)h->rp, 1u};
            const cuuint32_t es[2] = {1u, 1u};
            const CUresult r = enc(&h->gmaps[mode].m[o], h->storage_bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                                         : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                                   2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
            ++o;
        }
        h->gmaps_state[mode] = want;
    }
    *out = &h->gmaps[mode];
    return cudaSuccess;
}

cudaError_t fault_count_enqueue(ntc_handle* h, unsigned long long* host) {
    if (!h->stat.p) {
        *host = 0;
        return cudaSuccess;
    }
    return cudaMemcpyAsync(host, h->stat.as<unsigned long long>() + 2, sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, h->stream);
}

int64_t handle_device_bytes(const ntc_handle* h) {
    int64_t b = 0;
    for (int i = 0; i < kMaxOrder; ++i) {
        b += (int64_t)(h->U[i].bytes + h->Ub[i].bytes + h->row_ptr[i].bytes + h->bucket[i].bytes + h->perm[i].bytes +
                       h->inv_dev[i].bytes + h->rows_dev[i].bytes);
        const ModePlan& p = h->plan[i];
        b += (int64_t)(p.tiny_rows.bytes + p.tiny_k.bytes);
        b += (int64_t)(p.light_rows.bytes + p.light_k.bytes + p.chunks.bytes + p.chunk_caps.bytes + p.heavy.bytes +
                       p.bracket.bytes + p.heavy_cand.bytes + p.groups.bytes + p.heavy_groups.bytes);
    }
    for (int q = 0; q < 2; ++q)
        b += (int64_t)(h->vis[q].bytes + h->vis_cnt[q].bytes + h->cand[q].bytes + h->cand_cnt[q].bytes +
                       h->extra[q].bytes + h->extra_cnt[q].bytes + h->flags[q].bytes);
    b += (int64_t)(h->Y.bytes + h->coo_idx.bytes + h->coo_val.bytes + h->dims_dev.bytes +
                   h->partial.bytes + h->partial2.bytes + h->row_sum.bytes + h->stat.bytes +
                   h->red.bytes + h->mask.bytes + h->stage_idx.bytes + h->stage_val.bytes + h->sort_k0.bytes +
                   h->sort_k1.bytes + h->sort_v0.bytes + h->sort_v1.bytes + h->sort_hist.bytes + h->sort_sums.bytes +
                   h->bad_flag.bytes + h->row_cnt.bytes + h->entry_tmp.bytes);
    for (int i = 0; i < kMaxOrder; ++i) b += (int64_t)h->vwarm[i].bytes;
    return b;
}

}  // namespace ntc

// ---- allocation-free RMSE -----------------------------------------------------
// One double of partial sum per block of kNoAllocPerBlock queries, then the
// final sum and the out-of-range flag, in a file-scope device array: every GPU
// that loads the library holds these 32 KB until the process exits, and every
// call shares them.
constexpr int kNoAllocPerBlock = 2048;
constexpr int kNoAllocMaxBlocks = 4096;
constexpr int64_t kNoAllocMaxQueries = (int64_t)kNoAllocPerBlock * kNoAllocMaxBlocks;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxBlocks + 2];

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kNoAllocMaxDevices];

// Device address of the scratch array on the current device `dev` (the
// array's name in host code is only a host-side stand-in).  Only a successful
// lookup is kept, so a call after a failed one (e.g. one made during stream
// capture) looks it up again.
cudaError_t noalloc_scratch(int dev, double** out) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}
}  // namespace

extern "C" {

ntc_status ntc_create(int order, const int64_t* dims, int rank, double lambda, ntc_handle** out) {
    if (!out) return NTC_ERR_ARG;
    *out = nullptr;
    if (order < 2 || order > kMaxOrder || !dims || rank < 1 || rank > 64 || !(lambda >= 0.0) || std::isinf(lambda))
        return NTC_ERR_ARG;
    for (int i = 0; i < order; ++i)
        if (dims[i] < 1 || dims[i] >= (1ll << 31)) return NTC_ERR_ARG;
    ntc_handle* h = new (std::nothrow) ntc_handle();
    if (!h) return NTC_ERR_OOM;
    h->order = order;
    h->rank = rank;
    h->rp = pad_rank(rank);
    h->lambda = lambda;
    cudaGetDevice(&h->device);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < order && e == cudaSuccess; ++i) {
        h->dims[i] = dims[i];
        const size_t bytes = sizeof(float) * (size_t)dims[i] * h->rp;
        e = h->U[i].ensure(bytes);
        if (e == cudaSuccess) e = cudaMemset(h->U[i].p, 0, bytes);
    }
    for (int i = 0; i < order && e == cudaSuccess; ++i) {
        h->inv_h[i].resize((size_t)dims[i]);
        h->rows_h[i].resize((size_t)dims[i]);
        for (int64_t r = 0; r < dims[i]; ++r) h->inv_h[i][(size_t)r] = h->rows_h[i][(size_t)r] = (int32_t)r;
        e = h->inv_dev[i].ensure(sizeof(int32_t) * (size_t)dims[i]);
        if (e == cudaSuccess) e = h->rows_dev[i].ensure(sizeof(int32_t) * (size_t)dims[i]);
        if (e == cudaSuccess)
            e = cudaMemcpy(h->inv_dev[i].p, h->inv_h[i].data(), sizeof(int32_t) * dims[i], cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(h->rows_dev[i].p, h->rows_h[i].data(), sizeof(int32_t) * dims[i], cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = h->dims_dev.ensure(sizeof(int64_t) * kMaxOrder);
    if (e == cudaSuccess) e = cudaMemcpy(h->dims_dev.p, h->dims, sizeof(int64_t) * kMaxOrder, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        const ntc_status s = e == cudaErrorMemoryAllocation ? NTC_ERR_OOM : NTC_ERR_CUDA;
        delete h;
        return s;
    }
    *out = h;
    return NTC_OK;
}

ntc_status ntc_set_param(ntc_handle* h, const char* key, double v) {
    if (!h || !key) return NTC_ERR_ARG;
    h->err.clear();
    const std::string k(key);
    if (k == "max_inner") {
        if (!(v >= 1 && v <= 1e6)) return fail(h, NTC_ERR_ARG, "max_inner must be >= 1");
        h->max_inner = (int)v;
        if (h->max_inner > 1) {
            int64_t mx = 0;
            for (int i = 0; i < h->order; ++i) mx = std::max(mx, h->dims[i]);
            NTC_CUDA(h, h->Y.ensure(sizeof(float) * (size_t)mx * h->rp));
        }
    } else if (k == "power_iters") {
        if (!(v >= 1 && v <= 1e4)) return fail(h, NTC_ERR_ARG, "power_iters must be in [1, 10000]");
        h->power_iters = (int)v;
    } else if (k == "storage_bf16") {
        const int b = v != 0.0;
        if (b && !h->storage_bf16) {
            for (int i = 0; i < h->order; ++i) {
                const int64_t n = h->dims[i] * h->rp;
                NTC_CUDA(h, h->Ub[i].ensure(sizeof(uint16_t) * (size_t)n));
                k_to_bf16<<<grid_for(n), 256, 0, h->stream>>>(h->U[i].as<float>(), h->Ub[i].as<uint16_t>(), n);
            }
            NTC_CUDA(h, cudaGetLastError());
        }
        h->storage_bf16 = b;
    } else if (k == "init_seed") {
        if (!(v >= 0)) return fail(h, NTC_ERR_ARG, "init_seed must be >= 0");
        h->init_seed = (uint64_t)v;
    } else if (k == "overlap") {
        if (v != 0.0 && v != 1.0 && v != 2.0) return fail(h, NTC_ERR_ARG, "overlap must be 0, 1 or 2");
        h->overlap = (int)v;
    } else if (k == "profile") {
        h->profile = v != 0.0;
    } else if (k == "keep_perm") {
        h->keep_perm = v != 0.0;
    } else if (k == "pipeline") {
        if (h->nnz >= 0) return fail(h, NTC_ERR_STATE, "pipeline must be set before ntc_set_observed");
        h->pipeline = v != 0.0 ? 1 : 0;
    } else if (k == "power_warm") {
        h->power_warm = v != 0.0 ? 1 : 0;
    } else if (k == "sampler") {
        if (v != 0.0 && v != 1.0) return fail(h, NTC_ERR_ARG, "sampler must be 0 (independent) or 1 (epoch permutation)");
        h->sampler = (int)v;
    } else if (k == "gram_tc") {
        if (!(v == 0.0 || v == 1.0 || v == 2.0 || v == 3.0))
            return fail(h, NTC_ERR_ARG, "gram_tc must be 0, 1, 2 or 3");
        h->gram_tc = (int)v;
    } else if (k == "tiny_rows") {
        h->tiny_rows = v != 0.0 ? 1 : 0;
    } else if (k == "test_gram_stall") {
        if (!(v >= 0 && v <= 1e9)) return fail(h, NTC_ERR_ARG, "test_gram_stall must be in [0, 1e9] cycles");
        h->test_stall_cycles = (long long)v;
    } else if (k == "cache_staging") {
        h->cache_staging = v != 0.0 ? 1 : 0;
    } else if (k == "bracket_z") {
        if (!(v >= 0 && v <= 1e6)) return fail(h, NTC_ERR_ARG, "bracket_z must be in [0, 1e6]");
        h->bracket_z = v;
    } else if (k == "heavy_rows") {
        if (!(v >= 64 && v <= kLightMax)) return fail(h, NTC_ERR_ARG, "heavy_rows must be in [64, 4096]");
        h->heavy_threshold = (int)v;
    } else if (k == "chunk") {
        if (!(v >= 256 && v <= (1 << 24))) return fail(h, NTC_ERR_ARG, "chunk must be in [256, 2^24]");
        h->chunk = (int)v;
    } else {
        return fail(h, NTC_ERR_ARG, "unknown parameter " + k);
    }
    return NTC_OK;
}

ntc_status ntc_set_stream(ntc_handle* h, void* stream) {
    if (!h) return NTC_ERR_ARG;
    h->err.clear();
    h->stream = static_cast<cudaStream_t>(stream);
    return NTC_OK;
}

ntc_status ntc_set_observed(ntc_handle* h, int64_t nnz, const int32_t* idx, const float* vals) {
    if (h) h->err.clear();
    return set_observed_impl(h, nnz, idx, vals, false);
}

ntc_status ntc_set_observed_dev(ntc_handle* h, int64_t nnz, const int32_t* idx, const float* vals) {
    if (h) h->err.clear();
    return set_observed_impl(h, nnz, idx, vals, true);
}

ntc_status ntc_epoch(ntc_handle* h, const int* mode_order, double c, uint64_t seed) {
    ntc_status st = check_ready(h);
    if (st != NTC_OK) return st;
    h->err.clear();
    if (!(c > 0.0 && c <= 1.0)) return fail(h, NTC_ERR_ARG, "c must be in (0, 1]");
    int ord[kMaxOrder];
    bool seen[kMaxOrder] = {};
    for (int i = 0; i < h->order; ++i) {
        ord[i] = mode_order ? mode_order[i] : i;
        if (ord[i] < 0 || ord[i] >= h->order || seen[ord[i]])
            return fail(h, NTC_ERR_ARG, "mode_order must be a permutation of 0..order-1");
        seen[ord[i]] = true;
    }
    for (int i = 0; i < h->order; ++i)
        if ((st = build_plan(h, i, c)) != NTC_OK) return st;
    if ((st = reset_stats(h)) != NTC_OK) return st;
    const int64_t T = (int64_t)std::ceil(1.0 / c - 1e-12);   // AO iterations per epoch
    for (int64_t t = 0; t < T; ++t) {
        for (int i = 0; i < h->order; ++i)
            if ((st = run_snmc(h, ord[i], c, seed, h->ao_iter)) != NTC_OK) return st;
        h->ao_iter += 1;
    }
    return NTC_OK;
}

ntc_status ntc_snmc(ntc_handle* h, int mode, double c, uint64_t seed) {
    ntc_status st = check_ready(h);
    if (st != NTC_OK) return st;
    h->err.clear();
    if (mode < 0 || mode >= h->order) return fail(h, NTC_ERR_ARG, "mode out of range");
    if (!(c > 0.0 && c <= 1.0)) return fail(h, NTC_ERR_ARG, "c must be in (0, 1]");
    if ((st = reset_stats(h)) != NTC_OK) return st;
    return run_snmc(h, mode, c, seed, h->ao_iter);
}

ntc_status ntc_predict_dev(ntc_handle* h, int64_t n, const int32_t* idx, float* out) {
    if (!h || n < 0 || (n > 0 && (!idx || !out))) return NTC_ERR_ARG;
    h->err.clear();
    if (n == 0) return NTC_OK;
    k_predict<<<grid_for(n), 256, 0, h->stream>>>(factor_set(h), idx, n, out);
    NTC_CUDA(h, cudaGetLastError());
    return NTC_OK;
}

static bool indices_ok(const ntc_handle* h, int64_t n, const int32_t* idx) {
    for (int64_t e = 0; e < n; ++e)
        for (int i = 0; i < h->order; ++i) {
            const int32_t v = idx[e * h->order + i];
            if (v < 0 || v >= h->dims[i]) return false;
        }
    return true;
}

ntc_status ntc_predict(ntc_handle* h, int64_t n, const int32_t* idx, float* out) {
    if (!h || n < 0 || (n > 0 && (!idx || !out))) return NTC_ERR_ARG;
    h->err.clear();
    if (n == 0) return NTC_OK;
    if (!indices_ok(h, n, idx)) return fail(h, NTC_ERR_INDEX, "a query index is out of range");
    DevMem di, dout;
    NTC_CUDA(h, di.ensure(sizeof(int32_t) * n * h->order));
    NTC_CUDA(h, dout.ensure(sizeof(float) * n));
    NTC_CUDA(h, cudaMemcpyAsync(di.p, idx, sizeof(int32_t) * n * h->order, cudaMemcpyHostToDevice, h->stream));
    k_predict<<<grid_for(n), 256, 0, h->stream>>>(factor_set(h), di.as<int32_t>(), n, dout.as<float>());
    NTC_CUDA(h, cudaGetLastError());
    NTC_CUDA(h, cudaMemcpyAsync(out, dout.p, sizeof(float) * n, cudaMemcpyDeviceToHost, h->stream));
    NTC_CUDA(h, cudaStreamSynchronize(h->stream));
    return check_faults(h);
}

ntc_status ntc_rmse(ntc_handle* h, int64_t n, const int32_t* idx, const float* vals, double* out) {
    if (!h || !out || n < 0 || (n > 0 && (!idx || !vals))) return NTC_ERR_ARG;
    h->err.clear();
    if (n == 0) {
        *out = 0.0;
        return NTC_OK;
    }
    if (!indices_ok(h, n, idx)) return fail(h, NTC_ERR_INDEX, "a query index is out of range");
    DevMem di, dv, part, tot;
    NTC_CUDA(h, di.ensure(sizeof(int32_t) * n * h->order));
    NTC_CUDA(h, dv.ensure(sizeof(float) * n));
    NTC_CUDA(h, part.ensure(sizeof(double) * 1024));
    NTC_CUDA(h, tot.ensure(sizeof(double)));
    NTC_CUDA(h, cudaMemcpyAsync(di.p, idx, sizeof(int32_t) * n * h->order, cudaMemcpyHostToDevice, h->stream));
    NTC_CUDA(h, cudaMemcpyAsync(dv.p, vals, sizeof(float) * n, cudaMemcpyHostToDevice, h->stream));
    const int gb = grid_for(n, 256, 1024);
    k_sq_resid<<<gb, kThreads, 0, h->stream>>>(factor_set(h), di.as<int32_t>(), dv.as<float>(), n, part.as<double>());
    k_sum_partials<<<1, kThreads, 0, h->stream>>>(part.as<double>(), gb, tot.as<double>());
    NTC_CUDA(h, cudaGetLastError());
    double s = 0.0;
    NTC_CUDA(h, cudaMemcpyAsync(&s, tot.p, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    NTC_CUDA(h, cudaStreamSynchronize(h->stream));
    *out = std::sqrt(s / (double)n);
    return check_faults(h);
}

ntc_status ntc_cost(ntc_handle* h, double* out) {
    ntc_status st = check_ready(h);
    if (st != NTC_OK) return st;
    if (!out) return fail(h, NTC_ERR_ARG, "out is null");
    h->err.clear();
    DevMem part, tot;
    NTC_CUDA(h, part.ensure(sizeof(double) * 1024));
    NTC_CUDA(h, tot.ensure(sizeof(double) * (kMaxOrder + 1)));
    double fit = 0.0, reg = 0.0;
    const int gb = grid_for(h->nnz, 256, 1024);
    k_sq_resid<<<gb, kThreads, 0, h->stream>>>(factor_set(h), h->coo_idx.as<int32_t>(), h->coo_val.as<float>(),
                                               h->nnz, part.as<double>());
    k_sum_partials<<<1, kThreads, 0, h->stream>>>(part.as<double>(), gb, tot.as<double>());
    for (int i = 0; i < h->order; ++i) {
        const int64_t n = h->dims[i] * h->rp;   // padding columns are zero
        const int g2 = grid_for(n, 256, 1024);
        k_sq_sum<<<g2, kThreads, 0, h->stream>>>(h->U[i].as<float>(), n, part.as<double>());
        k_sum_partials<<<1, kThreads, 0, h->stream>>>(part.as<double>(), g2, tot.as<double>() + 1 + i);
    }
    NTC_CUDA(h, cudaGetLastError());
    double t[kMaxOrder + 1];
    NTC_CUDA(h, cudaMemcpyAsync(t, tot.p, sizeof(double) * (h->order + 1), cudaMemcpyDeviceToHost, h->stream));
    NTC_CUDA(h, cudaStreamSynchronize(h->stream));
    fit = t[0];
    for (int i = 0; i < h->order; ++i) reg += t[1 + i];
    *out = 0.5 * fit + 0.5 * h->lambda * reg;
    return check_faults(h);
}

ntc_status ntc_get_factor(ntc_handle* h, int mode, float* out) {
    if (!h || !out || mode < 0 || mode >= h->order) return NTC_ERR_ARG;
    h->err.clear();
    return download_factor(h, mode, out);
}

ntc_status ntc_set_factor(ntc_handle* h, int mode, const float* in) {
    if (!h || !in || mode < 0 || mode >= h->order) return NTC_ERR_ARG;
    h->err.clear();
    const int64_t n = h->dims[mode] * (int64_t)h->rank;
    for (int64_t j = 0; j < n; ++j)
        if (!(in[j] >= 0.0f) || std::isinf(in[j])) return fail(h, NTC_ERR_ARG, "factor entries must be finite and >= 0");
    ntc_status st = upload_factor(h, mode, in);
    if (st != NTC_OK) return st;
    h->factor_set[mode] = true;
    return NTC_OK;
}

ntc_status ntc_get_state(ntc_handle* h, uint64_t* ao_iter) {
    if (!h || !ao_iter) return NTC_ERR_ARG;
    *ao_iter = h->ao_iter;
    return NTC_OK;
}

ntc_status ntc_set_state(ntc_handle* h, uint64_t ao_iter) {
    if (!h) return NTC_ERR_ARG;
    h->ao_iter = ao_iter;
    return NTC_OK;
}

ntc_status ntc_sync(ntc_handle* h) {
    if (!h) return NTC_ERR_ARG;
    h->err.clear();
    NTC_CUDA(h, cudaStreamSynchronize(h->stream));
    return check_faults(h);
}

ntc_status ntc_get_stats(ntc_handle* h, ntc_stats* out) {
    if (!h || !out) return NTC_ERR_ARG;
    *out = h->stats;
    if (h->stat.p) {
        unsigned long long st[2] = {0, 0};
        NTC_CUDA(h, cudaMemcpyAsync(st, h->stat.p, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
        NTC_CUDA(h, cudaStreamSynchronize(h->stream));
        out->fallback_rows = (int64_t)st[0];
        out->wait_timeouts = (int64_t)st[1];
    }
    return NTC_OK;
}

ntc_status ntc_get_bucket(ntc_handle* h, int mode, int64_t* row_ptr, int64_t* perm) {
    ntc_status st = check_ready(h);
    if (st != NTC_OK) return st;
    if (mode < 0 || mode >= h->order) return fail(h, NTC_ERR_ARG, "mode out of range");
    if (row_ptr)
        memcpy(row_ptr, h->row_ptr_h[mode].data(), sizeof(int64_t) * (size_t)(h->dims[mode] + 1));
    if (perm) {
        if (!h->perm[mode].p) return fail(h, NTC_ERR_STATE, "set keep_perm before ntc_set_observed");
        std::vector<uint32_t> p((size_t)h->nnz);
        NTC_CUDA(h, cudaMemcpyAsync(p.data(), h->perm[mode].p, sizeof(uint32_t) * h->nnz, cudaMemcpyDeviceToHost,
                                    h->stream));
        NTC_CUDA(h, cudaStreamSynchronize(h->stream));
        for (int64_t q = 0; q < h->nnz; ++q) perm[q] = p[(size_t)q];
    }
    return NTC_OK;
}

ntc_status ntc_sample_mask(ntc_handle* h, int mode, double c, uint64_t seed, uint64_t ao_iter, int inner,
                           uint8_t* mask) {
    ntc_status st = check_ready(h);
    if (st != NTC_OK) return st;
    h->err.clear();
    if (mode < 0 || mode >= h->order || !mask || inner < 0) return fail(h, NTC_ERR_ARG, "bad sampler arguments");
    if (!(c > 0.0 && c <= 1.0)) return fail(h, NTC_ERR_ARG, "c must be in (0, 1]");
    if ((st = build_plan(h, mode, c)) != NTC_OK) return st;
    if ((st = reset_stats(h)) != NTC_OK) return st;
    NTC_CUDA(h, h->mask.ensure((size_t)std::max<int64_t>(h->nnz, 1)));
    NTC_CUDA(h, cudaMemsetAsync(h->mask.p, 0, (size_t)std::max<int64_t>(h->nnz, 1), h->stream));
    ModeArgs a = mode_args(h, mode, inner, seed, ao_iter);
    a.mask_out = h->mask.as<uint8_t>();
    set_perm(h, a, h->plan[mode], c, ao_iter, inner);
    Launcher L = make_launcher(h);
    NTC_CUDA(h, launch_mode(h->rp, ew_of(h->order), h->storage_bf16 != 0, a, h->plan[mode], L, true));
    h->upd += 1;
    NTC_CUDA(h, cudaMemcpyAsync(mask, h->mask.p, (size_t)h->nnz, cudaMemcpyDeviceToHost, h->stream));
    NTC_CUDA(h, cudaStreamSynchronize(h->stream));
    return NTC_OK;
}

ntc_status ntc_get_profile(ntc_handle* h, int kind, double* ms, int64_t* launches, int64_t* alg_bytes) {
    if (!h || kind < 0 || kind >= NTC_K_COUNT) return NTC_ERR_ARG;
    h->err.clear();
    if (!h->pending.empty()) {
        NTC_CUDA(h, cudaStreamSynchronize(h->stream));
        for (auto& q : h->pending) {
            float t = 0.f;
            NTC_CUDA(h, cudaEventElapsedTime(&t, q.a, q.b));
            h->prof_ms[q.kind] += t;
            h->prof_launches[q.kind] += 1;
            h->prof_bytes[q.kind] += q.bytes;
            cudaEventDestroy(q.a);
            cudaEventDestroy(q.b);
        }
        h->pending.clear();
    }
    if (ms) *ms = h->prof_ms[kind];
    if (launches) *launches = h->prof_launches[kind];
    if (alg_bytes) *alg_bytes = h->prof_bytes[kind];
    h->prof_ms[kind] = 0.0;
    h->prof_launches[kind] = 0;
    h->prof_bytes[kind] = 0;
    return NTC_OK;
}

ntc_status ntc_rmse_noalloc(ntc_handle* h, int64_t n, const int32_t* idx_dev, const float* vals_dev, double* out) {
    if (!h || !out || n < 0 || (n > 0 && (!idx_dev || !vals_dev))) return NTC_ERR_ARG;
    h->err.clear();
    if (n > kNoAllocMaxQueries)
        return fail(h, NTC_ERR_ARG, "ntc_rmse_noalloc: n = " + std::to_string(n) + " exceeds the limit of " +
                                        std::to_string(kNoAllocMaxQueries) + " queries per call");
    if (n == 0) {
        *out = 0.0;
        return NTC_OK;
    }
    int dev = -1;
    NTC_CUDA(h, cudaGetDevice(&dev));
    if (dev != h->device) return fail(h, NTC_ERR_STATE, "ntc_rmse_noalloc: the handle's device is not current");
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(h, NTC_ERR_ARG, "ntc_rmse_noalloc: device id too large");
    double* scratch = nullptr;
    NTC_CUDA(h, noalloc_scratch(dev, &scratch));
    const int nb = (int)((n + kNoAllocPerBlock - 1) / kNoAllocPerBlock);
    // every partial slot 0..nb-1 is written before it is read and the sum
    // slot by the second kernel; only the out-of-range flag starts at zero
    unsigned long long* bad = reinterpret_cast<unsigned long long*>(scratch + kNoAllocMaxBlocks + 1);
    NTC_CUDA(h, cudaMemsetAsync(bad, 0, sizeof(unsigned long long), h->stream));
    k_sq_resid<<<nb, kThreads, 0, h->stream>>>(factor_set(h), idx_dev, vals_dev, n, scratch, bad);
    k_sum_partials<<<1, kThreads, 0, h->stream>>>(scratch, nb, scratch + kNoAllocMaxBlocks);
    NTC_CUDA(h, cudaGetLastError());
    double res[2] = {0.0, 0.0};   // the sum, then the flag's bits
    NTC_CUDA(h, cudaMemcpyAsync(res, scratch + kNoAllocMaxBlocks, sizeof(res), cudaMemcpyDeviceToHost, h->stream));
    NTC_CUDA(h, cudaStreamSynchronize(h->stream));
    unsigned long long flag = 0;
    memcpy(&flag, &res[1], sizeof(flag));
    if (flag != 0) return fail(h, NTC_ERR_INDEX, "ntc_rmse_noalloc: a query index is out of range");
    *out = std::sqrt(res[0] / (double)n);
    return NTC_OK;
}

const char* ntc_last_error(const ntc_handle* h) { return h ? h->err.c_str() : "null handle"; }

void ntc_destroy(ntc_handle* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    delete h;
}

}  // extern "C"
