// serve.cu -- the continuous-batching completion server of include/ntc_serve.h.
//
// Each admitted job owns an ntc_handle (its bucketed observations, factors
// and scratch stay on the device) and a non-blocking CUDA stream.  A tick
// collects finished epochs, starts the admission of queued jobs under the HBM
// budget (upload and bucketing run on a worker thread, so ticks and queries
// go on meanwhile), and enqueues one epoch plus a device RMSE reduction for
// every idle job; the epochs of different jobs then run concurrently on the
// GPU.  After each epoch the job's stream copies its factors into one of two
// snapshot buffers; prediction queries read the snapshot of the last collected
// epoch (the epoch in flight writes the other one), so they never wait for a
// job's epoch, and all jobs' queries of a call go to one multi-job launch on a
// high-priority stream.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <deque>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "../../include/ntc_serve.h"
#include "ntc_host.h"

namespace {

using ntc::DevMem;

struct Job {
    int64_t id = 0;
    ntc_job_desc d = {};
    ntc_job_info info = {};
    ntc_handle* h = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done_ev = nullptr;   // end of the last enqueued epoch + RMSE
    bool busy = false;
    DevMem tidx, tval, scratch;
    DevMem snap[2];                  // factors after epoch e in snap[e % 2]
    double* host_sum = nullptr;      // pinned: squared residual sum of the last RMSE
    unsigned long long* host_faults = nullptr;   // pinned: tensor-core Gram waits that gave up
    long long test_stall = 0;        // test hook passed to the job's handle ("test_gram_stall")
    std::vector<float> factors[ntc::kMaxOrder];   // host copy once done
    // admission on a worker thread: 0 idle, 1 running, 2 succeeded, 3 failed
    bool admitting = false;
    std::thread admit_thread;
    std::atomic<int> admit_state{0};
    ntc_status admit_status = NTC_OK;
    std::string admit_err;
    // device memory of a finished job is freed on a reaper thread (cudaFree
    // synchronizes the device); its bytes stay in the budget until then
    std::thread reap_thread;
    std::atomic<int> reap_state{0};   // 0 none, 1 freeing, 2 freed
};

bool desc_ok(const ntc_job_desc* d, std::string* why) {
    if (!d) return *why = "null job description", false;
    if (d->order < 2 || d->order > ntc::kMaxOrder) return *why = "order must be in [2, 8]", false;
    for (int i = 0; i < d->order; ++i)
        if (d->dims[i] < 1 || d->dims[i] > INT32_MAX) return *why = "dims must be in [1, 2^31)", false;
    if (d->rank < 1 || d->rank > 64) return *why = "rank must be in [1, 64]", false;
    if (!(d->lambda >= 0.0) || !std::isfinite(d->lambda)) return *why = "lambda must be finite and >= 0", false;
    if (!(d->c > 0.0 && d->c <= 1.0)) return *why = "c must be in (0, 1]", false;
    if (d->nnz < 1 || !d->idx || !d->vals) return *why = "a job needs observations", false;
    if (d->n_test < 1 || !d->test_idx || !d->test_vals) return *why = "a job needs held-out observations", false;
    if (!(d->target_rmse >= 0.0)) return *why = "target_rmse must be >= 0", false;
    if (d->max_epochs < 1) return *why = "max_epochs must be >= 1", false;
    if (!std::isfinite(d->arrival)) return *why = "arrival must be finite", false;
    return true;
}

// Device bytes of a job, following the allocations of ntc_create,
// ntc_set_observed and the per-mode plans and scratch of ntc_epoch.
int64_t model_bytes(const ntc_job_desc* d) {
    const int N = d->order;
    const int64_t nnz = d->nnz;
    const int rp = ntc::pad_rank(d->rank);
    const int T = rp / 8;
    const int64_t pw = (int64_t)T * (T + 1) / 2 * 64 + rp;   // floats per reduced-sum row
    const int64_t ent = (N <= 4 ? 4 : 8) * 4;                 // bytes per bucket entry
    int64_t sum_dims = 0, max_dim = 0;
    for (int i = 0; i < N; ++i) {
        sum_dims += d->dims[i];
        max_dim = std::max<int64_t>(max_dim, d->dims[i]);
    }
    int64_t b = 0;
    b += nnz * (4 * N + 4);                                   // COO kept for the cost
    b += N * nnz * ent;                                       // one bucket per mode
    b += sum_dims * 8 + N * 8;                                // row_ptr
    b += sum_dims * 8;                                        // row maps
    b += sum_dims * rp * (4 + (d->storage_bf16 ? 2 : 0));    // masters (+ BF16 copies)
    b += sum_dims * 8;                                        // light-row plans
    b += 2 * nnz * 4;                                         // visit lists (two sampling sets)
    b += 2 * (nnz + (1 << 20));                               // candidates and chosen lists (two sets)
    const int64_t items = nnz / 16384 + 2 * max_dim + 1;      // chunks + split rows (bound)
    b += items * pw * 4 * 2;                                  // partials and group sums
    b += max_dim * pw * 4;                                    // per-row reduced sums
    b += d->n_test * (4 * N + 4) + ntc::kRmseScratch * 8;    // held-out set
    b += 2 * sum_dims * rp * 4;                               // two factor snapshots for queries
    b += nnz * (4 * N + 4) + nnz * 16 + (nnz / 256 + 1) * 8;  // admission: COO copy + sort buffers
    b += nnz * ent;                                           // admission: entries before the bucket gather
    b += 8 << 20;                                             // small buffers and allocation rounding
    return b;
}

}  // namespace

struct ntc_server {
    double budget = 0.0;
    int max_running = 1;
    std::vector<std::unique_ptr<Job>> jobs;
    std::deque<int64_t> queue;   // queued job ids in (arrival, id) order
    std::chrono::steady_clock::time_point t0;
    std::string err;
    ntc_server_stats st = {};
    cudaStream_t qstream = nullptr;   // prediction queries
    DevMem q_slot, q_idx, q_out, q_table;
    int device = 0;
    int max_enqueue = 1 << 30;        // epochs enqueued per tick
    long long test_stall = 0;         // "test_gram_stall" for jobs submitted from now on
    size_t rr = 0;                    // round-robin start of the enqueue scan

    double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
    ntc_status fail(ntc_status s, const std::string& m) {
        err = m;
        return s;
    }
};

namespace {

ntc_status cuda_fail(ntc_server* s, cudaError_t e, const char* what) {
    return s->fail(e == cudaErrorMemoryAllocation ? NTC_ERR_OOM : NTC_ERR_CUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}

// Frees the job's device state (and its stream); touches only the job.
void free_device(Job& j) {
    if (j.stream) cudaStreamSynchronize(j.stream);
    if (j.h) ntc_destroy(j.h);
    j.h = nullptr;
    j.tidx.release();
    j.tval.release();
    j.scratch.release();
    j.snap[0].release();
    j.snap[1].release();
    if (j.host_sum) cudaFreeHost(j.host_sum);
    j.host_sum = nullptr;
    if (j.host_faults) cudaFreeHost(j.host_faults);
    j.host_faults = nullptr;
    if (j.done_ev) cudaEventDestroy(j.done_ev);
    j.done_ev = nullptr;
    if (j.stream) cudaStreamDestroy(j.stream);
    j.stream = nullptr;
}

// The job stops running; its device memory is freed on a reaper thread and
// its bytes leave the budget when a tick sees that finished.
void release_job(ntc_server* s, Job& j) {
    j.busy = false;
    if (j.info.state == NTC_JOB_RUNNING || j.admitting) s->st.running -= 1;
    j.admitting = false;
    j.reap_state.store(1);
    Job* jp = &j;
    const int dev = s->device;
    j.reap_thread = std::thread([jp, dev] {
        cudaSetDevice(dev);
        free_device(*jp);
        jp->reap_state.store(2, std::memory_order_release);
    });
}

void collect_reaped(ntc_server* s, bool wait) {
    for (auto& jp : s->jobs) {
        Job& j = *jp;
        if (j.reap_state.load(std::memory_order_acquire) == 0) continue;
        if (j.reap_state.load(std::memory_order_acquire) == 1 && !wait) continue;
        if (j.reap_thread.joinable()) {
            j.reap_thread.join();
            s->st.bytes_in_use -= j.info.bytes;
        }
    }
}

// Keeps the factors on the host, frees the device state, marks the job done.
ntc_status finish_job(ntc_server* s, Job& j, bool reached) {
    for (int m = 0; m < j.d.order; ++m) {
        j.factors[m].resize((size_t)j.d.dims[m] * j.d.rank);
        ntc_status r = ntc_get_factor(j.h, m, j.factors[m].data());
        if (r != NTC_OK) return s->fail(r, std::string("job factor download: ") + ntc_last_error(j.h));
    }
    release_job(s, j);
    j.info.state = NTC_JOB_DONE;
    j.info.reached = reached ? 1 : 0;
    j.info.t_done = s->now();
    s->st.done += 1;
    return NTC_OK;
}

void fail_job(ntc_server* s, Job& j, const std::string& why) {
    release_job(s, j);
    j.info.state = NTC_JOB_FAILED;
    j.info.t_done = s->now();
    s->st.failed += 1;
    s->err = "job " + std::to_string(j.id) + ": " + why;
}

// Device state of a job: handle, stream, observations, held-out set, initial
// RMSE and the snapshot of the initial factors.  Runs on the admission worker
// thread: it touches only the job.
ntc_status admit_job(Job& j, int device) {
    const ntc_job_desc& d = j.d;
    auto cuda_err = [&](cudaError_t e, const char* what) {
        j.admit_err = std::string(what) + ": " + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? NTC_ERR_OOM : NTC_ERR_CUDA;
    };
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&j.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j.done_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&j.host_sum, sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&j.host_faults, sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_err(e, "job stream");
    *j.host_faults = 0;
    ntc_status r = ntc_create(d.order, d.dims, d.rank, d.lambda, &j.h);
    if (r != NTC_OK) return j.admit_err = "ntc_create failed", r;
    auto chk = [&](ntc_status q) -> bool {
        if (q == NTC_OK) return true;
        r = q;
        j.admit_err = ntc_last_error(j.h);
        return false;
    };
    if (!chk(ntc_set_stream(j.h, j.stream)) || !chk(ntc_set_param(j.h, "storage_bf16", d.storage_bf16 ? 1.0 : 0.0)) ||
        !chk(ntc_set_param(j.h, "init_seed", (double)d.init_seed)) ||
        !chk(ntc_set_param(j.h, "cache_staging", 0.0)) ||
        !chk(ntc_set_param(j.h, "test_gram_stall", (double)j.test_stall)) ||
        !chk(ntc_set_observed(j.h, d.nnz, d.idx, d.vals)) || !chk(ntc::prepare_epoch(j.h, d.c)))
        return r;
    for (int64_t q = 0; q < d.n_test * d.order; ++q) {
        const int32_t v = d.test_idx[q];
        if (v < 0 || v >= d.dims[q % d.order]) return j.admit_err = "a held-out index is out of range", NTC_ERR_INDEX;
    }
    const size_t snap_bytes = sizeof(float) * (size_t)ntc::snapshot_floats(j.h);
    e = j.tidx.ensure(sizeof(int32_t) * (size_t)(d.n_test * d.order));
    if (e == cudaSuccess) e = j.tval.ensure(sizeof(float) * (size_t)d.n_test);
    if (e == cudaSuccess) e = j.scratch.ensure(sizeof(double) * ntc::kRmseScratch);
    if (e == cudaSuccess) e = j.snap[0].ensure(snap_bytes);
    if (e == cudaSuccess) e = j.snap[1].ensure(snap_bytes);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(j.tidx.p, d.test_idx, sizeof(int32_t) * (size_t)(d.n_test * d.order),
                            cudaMemcpyHostToDevice, j.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(j.tval.p, d.test_vals, sizeof(float) * (size_t)d.n_test, cudaMemcpyHostToDevice, j.stream);
    if (e == cudaSuccess) e = ntc::snapshot_factors(j.h, j.snap[0].as<float>());
    if (e == cudaSuccess)
        e = ntc::rmse_enqueue(j.h, j.tidx.as<int32_t>(), j.tval.as<float>(), d.n_test, j.scratch.as<double>(),
                              j.host_sum);
    if (e == cudaSuccess) e = cudaStreamSynchronize(j.stream);
    if (e != cudaSuccess) return cuda_err(e, "job admission");
    j.info.rmse0 = j.info.rmse = std::sqrt(*j.host_sum / (double)d.n_test);
    return NTC_OK;
}

ntc_status enqueue_epoch(ntc_server* s, Job& j) {
    ntc_status r = ntc_epoch(j.h, nullptr, j.d.c, j.d.seed + (uint64_t)j.info.epochs);
    if (r != NTC_OK) return s->fail(r, ntc_last_error(j.h));
    // factors after this epoch (number epochs + 1) go to the snapshot that
    // queries do not read until the epoch is collected
    cudaError_t e = ntc::snapshot_factors(j.h, j.snap[(j.info.epochs + 1) % 2].as<float>());
    if (e == cudaSuccess)
        e = ntc::rmse_enqueue(j.h, j.tidx.as<int32_t>(), j.tval.as<float>(), j.d.n_test, j.scratch.as<double>(),
                              j.host_sum);
    if (e == cudaSuccess) e = ntc::fault_count_enqueue(j.h, j.host_faults);
    if (e == cudaSuccess) e = cudaEventRecord(j.done_ev, j.stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "epoch enqueue");
    j.busy = true;
    return NTC_OK;
}

Job* find_job(const ntc_server* s, int64_t id) {
    if (!s || id < 0 || id >= (int64_t)s->jobs.size()) return nullptr;
    return s->jobs[(size_t)id].get();
}

}  // namespace

extern "C" {

ntc_status ntc_job_bytes(const ntc_job_desc* desc, int64_t* out) {
    std::string why;
    if (!out || !desc_ok(desc, &why)) return NTC_ERR_ARG;
    *out = model_bytes(desc);
    return NTC_OK;
}

ntc_status ntc_server_create(double hbm_budget, int max_running, ntc_server** out) {
    if (!out) return NTC_ERR_ARG;
    *out = nullptr;
    if (!(hbm_budget > 0.0) || !std::isfinite(hbm_budget) || max_running < 1) return NTC_ERR_ARG;
    auto s = std::make_unique<ntc_server>();
    s->budget = hbm_budget;
    s->max_running = max_running;
    s->t0 = std::chrono::steady_clock::now();
    if (cudaGetDevice(&s->device) != cudaSuccess) return NTC_ERR_CUDA;
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return NTC_ERR_CUDA;
    if (cudaStreamCreateWithPriority(&s->qstream, cudaStreamNonBlocking, greatest) != cudaSuccess)
        return NTC_ERR_CUDA;
    *out = s.release();
    return NTC_OK;
}

ntc_status ntc_server_set_param(ntc_server* s, const char* key, double value) {
    if (!s || !key) return NTC_ERR_ARG;
    const std::string k(key);
    if (k == "max_enqueue_per_step") {
        if (!(value >= 1.0 && value <= 1e9)) return s->fail(NTC_ERR_ARG, "max_enqueue_per_step must be >= 1");
        s->max_enqueue = (int)value;
        return NTC_OK;
    }
    if (k == "test_gram_stall") {   // test hook for jobs submitted from now on
        if (!(value >= 0.0 && value <= 1e9)) return s->fail(NTC_ERR_ARG, "test_gram_stall must be in [0, 1e9]");
        s->test_stall = (long long)value;
        return NTC_OK;
    }
    return s->fail(NTC_ERR_ARG, "unknown server parameter: " + k);
}

ntc_status ntc_server_submit(ntc_server* s, const ntc_job_desc* desc, int64_t* job_id) {
    if (!s || !job_id) return NTC_ERR_ARG;
    std::string why;
    if (!desc_ok(desc, &why)) return s->fail(NTC_ERR_ARG, why);
    const int64_t bytes = model_bytes(desc);
    if ((double)bytes > s->budget) return s->fail(NTC_ERR_ARG, "job needs more than the whole budget");
    auto j = std::make_unique<Job>();
    j->id = (int64_t)s->jobs.size();
    j->d = *desc;
    j->info.state = NTC_JOB_QUEUED;
    j->info.rmse = j->info.rmse0 = -1.0;
    j->info.t_arrival = desc->arrival;
    j->info.t_admit = j->info.t_done = -1.0;
    j->info.bytes = bytes;
    j->test_stall = s->test_stall;
    // arrival order, ties by id
    auto pos = std::upper_bound(s->queue.begin(), s->queue.end(), desc->arrival,
                                [&](double t, int64_t id) { return t < s->jobs[(size_t)id]->d.arrival; });
    s->queue.insert(pos, j->id);
    *job_id = j->id;
    s->jobs.push_back(std::move(j));
    s->st.submitted += 1;
    s->st.queued += 1;
    return NTC_OK;
}

ntc_status ntc_server_step(ntc_server* s, int64_t* running, int64_t* queued) {
    if (!s) return NTC_ERR_ARG;
    if (cudaSetDevice(s->device) != cudaSuccess) return s->fail(NTC_ERR_CUDA, "cudaSetDevice");
    // 0. memory of finished jobs that is free again, admissions that finished
    collect_reaped(s, false);
    for (auto& jp : s->jobs) {
        Job& j = *jp;
        if (!j.admitting || j.admit_state.load(std::memory_order_acquire) < 2) continue;
        j.admit_thread.join();
        if (j.admit_state.load() == 3) {
            fail_job(s, j, j.admit_err);
            continue;
        }
        j.admitting = false;
        j.info.state = NTC_JOB_RUNNING;
        if (!(j.info.rmse > j.d.target_rmse)) {   // already at the target
            ntc_status r2 = finish_job(s, j, true);
            if (r2 != NTC_OK) return r2;
        }
    }
    // 1. finished epochs
    for (auto& jp : s->jobs) {
        Job& j = *jp;
        if (j.info.state != NTC_JOB_RUNNING || !j.busy) continue;
        const cudaError_t q = cudaEventQuery(j.done_ev);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) {
            fail_job(s, j, std::string("epoch: ") + cudaGetErrorString(q));
            return NTC_ERR_CUDA;
        }
        j.busy = false;
        if (*j.host_faults > 0) {   // a bounded wait gave up: this epoch's factors are not valid
            fail_job(s, j, "tensor-core Gram: " + std::to_string(*j.host_faults) +
                               " block(s) gave up a bounded wait; the job's factors are not valid");
            continue;
        }
        j.info.epochs += 1;
        j.info.rmse = std::sqrt(*j.host_sum / (double)j.d.n_test);
        s->st.epochs += 1;
        s->st.entries += j.d.nnz;
        if (!(j.info.rmse > j.d.target_rmse) || j.info.epochs >= j.d.max_epochs) {
            const bool reached = !(j.info.rmse > j.d.target_rmse);
            ntc_status r = finish_job(s, j, reached);
            if (r != NTC_OK) return r;
        }
    }
    // 2. admission: head of the queue first, while it has arrived and fits
    const double t = s->now();
    while (!s->queue.empty()) {
        Job& j = *s->jobs[(size_t)s->queue.front()];
        if (j.d.arrival > t || s->st.running >= s->max_running) break;
        if ((double)(s->st.bytes_in_use + j.info.bytes) > s->budget) break;
        s->queue.pop_front();
        s->st.queued -= 1;
        // the memory is the job's from now on; upload and bucketing run aside
        j.admitting = true;
        j.info.t_admit = s->now();
        s->st.running += 1;
        s->st.bytes_in_use += j.info.bytes;
        s->st.peak_bytes = std::max(s->st.peak_bytes, s->st.bytes_in_use);
        s->st.peak_running = std::max(s->st.peak_running, s->st.running);
        j.admit_state.store(1);
        Job* jp = &j;
        const int dev = s->device;
        j.admit_thread = std::thread([jp, dev] {
            jp->admit_status = admit_job(*jp, dev);
            jp->admit_state.store(jp->admit_status == NTC_OK ? 2 : 3, std::memory_order_release);
        });
    }
    // 3. next epoch of idle running jobs, at most max_enqueue per tick, the
    // scan starting where the last tick stopped
    int enq = 0;
    const size_t nj = s->jobs.size();
    for (size_t k = 0; k < nj && enq < s->max_enqueue; ++k) {
        Job& j = *s->jobs[(s->rr + k) % nj];
        if (j.info.state != NTC_JOB_RUNNING || j.busy) continue;
        ntc_status r = enqueue_epoch(s, j);
        if (r != NTC_OK) {
            const std::string why = s->err;
            fail_job(s, j, why);
            return r;
        }
        ++enq;
        s->rr = (s->rr + k + 1) % nj;
    }
    if (running) *running = s->st.running;
    if (queued) *queued = s->st.queued;
    return NTC_OK;
}

ntc_status ntc_server_sync(ntc_server* s) {
    if (!s) return NTC_ERR_ARG;
    for (auto& jp : s->jobs)   // admissions in progress: wait for their threads (a tick takes them over)
        while (jp->admitting && jp->admit_state.load(std::memory_order_acquire) == 1) std::this_thread::yield();
    for (auto& jp : s->jobs)
        if (jp->info.state == NTC_JOB_RUNNING && jp->stream) {
            const cudaError_t e = cudaStreamSynchronize(jp->stream);
            if (e != cudaSuccess) return cuda_fail(s, e, "job stream");
        }
    return NTC_OK;
}

double ntc_server_now(const ntc_server* s) { return s ? s->now() : -1.0; }

ntc_status ntc_server_job_info(const ntc_server* s, int64_t job_id, ntc_job_info* out) {
    const Job* j = find_job(s, job_id);
    if (!j || !out) return NTC_ERR_ARG;
    *out = j->info;
    return NTC_OK;
}

ntc_status ntc_server_predict(ntc_server* s, int64_t n, const int64_t* job_ids, const int32_t* idx, float* out) {
    if (!s || n < 0 || (n > 0 && (!job_ids || !idx || !out))) return NTC_ERR_ARG;
    if (n == 0) return NTC_OK;
    // the running jobs named by the queries, each once, in first-use order
    std::vector<int32_t> slot((size_t)n);
    std::vector<ntc_handle*> hs;
    std::vector<const float*> snaps;
    std::vector<int64_t> slot_of(s->jobs.size(), -1);
    for (int64_t q = 0; q < n; ++q) {
        Job* j = find_job(s, job_ids[q]);
        if (!j) return s->fail(NTC_ERR_ARG, "unknown job id");
        if (j->info.state != NTC_JOB_RUNNING) return s->fail(NTC_ERR_STATE, "query to a job that is not running");
        for (int i = 0; i < j->d.order; ++i) {
            const int32_t v = idx[q * ntc::kMaxOrder + i];
            if (v < 0 || v >= j->d.dims[i]) return s->fail(NTC_ERR_INDEX, "a query index is out of range");
        }
        int64_t& sl = slot_of[(size_t)j->id];
        if (sl < 0) {
            sl = (int64_t)hs.size();
            hs.push_back(j->h);
            // factors after the last collected epoch; the epoch in flight
            // writes the other snapshot
            snaps.push_back(j->snap[j->info.epochs % 2].as<float>());
        }
        slot[(size_t)q] = (int32_t)sl;
    }
    cudaError_t e = s->q_slot.ensure(sizeof(int32_t) * (size_t)n);
    if (e == cudaSuccess) e = s->q_idx.ensure(sizeof(int32_t) * (size_t)n * ntc::kMaxOrder);
    if (e == cudaSuccess) e = s->q_out.ensure(sizeof(float) * (size_t)n);
    if (e == cudaSuccess) e = s->q_table.ensure(ntc::factor_table_bytes() * hs.size());
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->q_slot.p, slot.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s->qstream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->q_idx.p, idx, sizeof(int32_t) * (size_t)n * ntc::kMaxOrder, cudaMemcpyHostToDevice,
                            s->qstream);
    if (e == cudaSuccess)
        e = ntc::predict_multi(hs.data(), snaps.data(), (int)hs.size(), s->q_slot.as<int32_t>(),
                               s->q_idx.as<int32_t>(), n, s->q_out.as<float>(), s->q_table.p, s->qstream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, s->q_out.p, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, s->qstream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->qstream);
    if (e != cudaSuccess) return cuda_fail(s, e, "predict");
    s->st.predict_calls += 1;
    s->st.predict_queries += n;
    s->st.predict_launches += 1;
    return NTC_OK;
}

ntc_status ntc_server_get_factor(ntc_server* s, int64_t job_id, int mode, float* out) {
    Job* j = find_job(s, job_id);
    if (!j || !out || mode < 0 || mode >= (j ? j->d.order : 0)) return NTC_ERR_ARG;
    if (j->info.state == NTC_JOB_RUNNING) {
        // the snapshot queries read: factors after the last collected epoch
        const ntc_handle* h = j->h;
        const int64_t I = h->dims[mode];
        const int R = h->rank, RP = h->rp;
        int64_t off = 0;
        for (int i = 0; i < mode; ++i) off += h->dims[i] * RP;
        std::vector<float> tmp((size_t)(I * RP));
        cudaError_t e = cudaMemcpyAsync(tmp.data(), j->snap[j->info.epochs % 2].as<float>() + off,
                                        sizeof(float) * tmp.size(), cudaMemcpyDeviceToHost, s->qstream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->qstream);
        if (e != cudaSuccess) return cuda_fail(s, e, "factor snapshot");
        const std::vector<int32_t>& inv = h->inv_h[mode];   // caller row -> stored row
        for (int64_t r = 0; r < I; ++r)
            std::copy(tmp.begin() + (size_t)inv[(size_t)r] * RP, tmp.begin() + (size_t)inv[(size_t)r] * RP + R,
                      out + r * R);
        return NTC_OK;
    }
    if (j->info.state != NTC_JOB_DONE) return s->fail(NTC_ERR_STATE, "the job has no factors yet");
    std::copy(j->factors[mode].begin(), j->factors[mode].end(), out);
    return NTC_OK;
}

ntc_status ntc_server_stats_get(const ntc_server* s, ntc_server_stats* out) {
    if (!s || !out) return NTC_ERR_ARG;
    *out = s->st;
    return NTC_OK;
}

const char* ntc_server_last_error(const ntc_server* s) { return s ? s->err.c_str() : "null server"; }

void ntc_server_destroy(ntc_server* s) {
    if (!s) return;
    for (auto& jp : s->jobs)
        if (jp->admit_thread.joinable()) jp->admit_thread.join();
    collect_reaped(s, true);
    for (auto& jp : s->jobs) free_device(*jp);
    cudaSetDevice(s->device);
    if (s->qstream) cudaStreamDestroy(s->qstream);
    delete s;
}

}  // extern "C"
