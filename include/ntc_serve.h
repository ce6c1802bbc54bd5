/* ntc_serve.h -- continuous-batching completion server on one GPU.
 *
 * Many completion jobs (each a nonnegative CPD fit of Algorithm 2, run by the
 * per-mode accelerated stochastic update of Algorithm 1, Sec. II-III) share one
 * GPU.  Jobs arrive over time; the server admits them in arrival order while
 * their modelled device memory fits an HBM budget, keeps every admitted job's
 * observations (bucketed per mode), factors and scratch resident, and on each
 * call of ntc_server_step advances every admitted job by one epoch (ceil(1/c)
 * AO iterations, Sec. IV) on the job's own CUDA stream, so that the kernels of
 * different jobs overlap on the device.  After each epoch the job's held-out
 * RMSE is reduced on the device and read back asynchronously; a job is done
 * when that RMSE reaches its target or its epoch limit, and its memory is then
 * returned to the budget (its factors are kept in host memory).  Entry
 * prediction queries against the current factors of many jobs are answered by
 * one multi-job kernel launch per call.
 *
 * The paper has no serving component; the job, budget and query interfaces
 * are this library's.  Each job's arithmetic is exactly that of a single
 * ntc_handle fed the same inputs: epoch e of a job uses seed desc.seed + e, so
 * a job's factors do not depend on what else runs beside it.
 *
 * Threads: a server must be used from one host thread at a time.
 * Errors: calls return ntc_status; ntc_server_last_error gives the message.
 */
#ifndef NTC_SERVE_H
#define NTC_SERVE_H

#include <stdint.h>

#include "ntc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ntc_server ntc_server;

/* One completion job.  All pointers are host memory owned by the caller; they
 * must stay valid until the job has been admitted (ntc_job_info.state becomes
 * NTC_JOB_RUNNING or later): admission copies them to the device. */
typedef struct {
    int order;                 /* tensor order N, 2..8                                */
    int64_t dims[8];           /* I_1..I_N (entries past `order` ignored)             */
    int rank;                  /* R, 1..64                                            */
    double lambda;             /* regularisation, >= 0 (Sec. II, eq. 3)               */
    double c;                  /* minibatch fraction per row, 0 < c <= 1 (Sec. II-B)  */
    int storage_bf16;          /* 1: BF16 factor storage with FP32 masters            */
    uint64_t seed;             /* sampling seed of epoch 0; epoch e uses seed + e     */
    uint64_t init_seed;        /* seed of the initial factors                         */
    int64_t nnz;               /* training observations                              */
    const int32_t* idx;        /* [nnz][order] zero-based indices                     */
    const float* vals;         /* [nnz]                                              */
    int64_t n_test;            /* held-out observations (>= 1)                        */
    const int32_t* test_idx;   /* [n_test][order]                                    */
    const float* test_vals;    /* [n_test]                                           */
    double target_rmse;        /* done when the held-out RMSE is <= this              */
    int max_epochs;            /* done (target missed) after this many epochs, >= 1   */
    double arrival;            /* server-clock seconds before which it is not admitted */
} ntc_job_desc;

enum { NTC_JOB_QUEUED = 0, NTC_JOB_RUNNING = 1, NTC_JOB_DONE = 2, NTC_JOB_FAILED = 3 };

typedef struct {
    int state;                 /* NTC_JOB_*                                           */
    int reached;               /* 1 if the target RMSE was reached                    */
    int epochs;                /* epochs completed                                   */
    double rmse;               /* held-out RMSE after the last completed epoch        */
    double rmse0;              /* held-out RMSE of the initial factors                */
    double t_arrival, t_admit, t_done;   /* server-clock seconds (-1 if not yet)     */
    int64_t bytes;             /* modelled device bytes held while running           */
} ntc_job_info;

typedef struct {
    int64_t submitted, queued, running, done, failed;
    int64_t bytes_in_use;      /* modelled bytes of running jobs                     */
    int64_t peak_bytes;        /* largest bytes_in_use seen                           */
    int64_t peak_running;      /* largest number of jobs running at once              */
    int64_t epochs;            /* epochs completed over all jobs                      */
    int64_t entries;           /* sum over completed epochs of the job's nnz          */
    int64_t predict_calls, predict_queries, predict_launches;
} ntc_server_stats;

/* Modelled device bytes of a job while it runs: observations (COO and one
 * bucket per mode), factors (FP32 masters, BF16 copies, Y), per-mode plans,
 * sampling and reduction scratch, the held-out set, and the transient sort
 * buffers of admission.  NTC_ERR_ARG if the description is invalid. */
ntc_status ntc_job_bytes(const ntc_job_desc* desc, int64_t* out);

/* hbm_budget: bytes the running jobs' modelled memory may use together (> 0);
 * max_running: at most this many jobs run at once (>= 1). */
ntc_status ntc_server_create(double hbm_budget, int max_running, ntc_server** out);

/* "max_enqueue_per_step": at most this many epochs are enqueued by one tick
 * (default unlimited), the scan resuming where the previous tick stopped, so
 * that a tick stays short and queries issued between ticks are served soon.
 * "test_gram_stall": test hook, the handle parameter of that name for jobs
 * submitted from now on (default 0, off).
 * A job whose epoch reports a tensor-core Gram block that gave up a bounded
 * wait (ntc_stats.wait_timeouts) ends in NTC_JOB_FAILED.
 * NTC_ERR_ARG for an unknown key or a value out of range. */
ntc_status ntc_server_set_param(ntc_server* s, const char* key, double value);

/* Queues a job; *job_id is its id (0, 1, ... in submission order).
 * NTC_ERR_ARG for an invalid description or a job larger than the budget. */
ntc_status ntc_server_submit(ntc_server* s, const ntc_job_desc* desc, int64_t* job_id);

/* One scheduler tick: take over jobs whose admission finished, collect
 * finished epochs (read their RMSE, mark jobs done and free them), start the
 * admission of queued jobs whose arrival time has passed while the budget and
 * max_running allow (in arrival order, the head of the queue first; the job's
 * memory counts from here, its upload and bucketing run on a worker thread and
 * the job is RUNNING from the first tick after they finish), and enqueue the
 * next epoch of every running job that is idle.  Does not wait for the GPU.
 * *running (admitted jobs, admitting included) / *queued (may be NULL) get the
 * counts after the tick. */
ntc_status ntc_server_step(ntc_server* s, int64_t* running, int64_t* queued);

/* Blocks until every running job has finished its enqueued epoch (a tick
 * afterwards collects them). */
ntc_status ntc_server_sync(ntc_server* s);

/* Server clock: seconds since ntc_server_create. */
double ntc_server_now(const ntc_server* s);

ntc_status ntc_server_job_info(const ntc_server* s, int64_t job_id, ntc_job_info* out);

/* n queries: job_ids[q] names a running job and idx[q * 8 + i] (i < that job's
 * order) its zero-based index; out[q] gets the CP model value (eq. 1) from
 * the job's factors after its last collected epoch (a snapshot, so a query
 * never waits for an epoch in flight).  One kernel launch on a high-priority
 * stream serves all jobs of the call.
 * NTC_ERR_STATE if a job is not running, NTC_ERR_INDEX for an index out of
 * range.  Synchronous (out is host memory). */
ntc_status ntc_server_predict(ntc_server* s, int64_t n, const int64_t* job_ids, const int32_t* idx, float* out);

/* Factor `mode` of a job, [dims[mode]][rank] row-major FP32, the same factors
 * queries see: while running, those after the last epoch a tick collected (the
 * query snapshot; an epoch in flight is not waited for); once done, the final
 * factors (host copy).  NTC_ERR_STATE while queued or admitting. */
ntc_status ntc_server_get_factor(ntc_server* s, int64_t job_id, int mode, float* out);

ntc_status ntc_server_stats_get(const ntc_server* s, ntc_server_stats* out);
const char* ntc_server_last_error(const ntc_server* s);
void ntc_server_destroy(ntc_server* s);

#ifdef __cplusplus
}
#endif

#endif /* NTC_SERVE_H */
