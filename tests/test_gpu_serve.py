"""Continuous-batching completion server on the GPU: every job's factors are
the same alone and in the mix (and equal those of a plain handle fed the same
inputs), admission keeps the modelled memory under the budget and honours
arrival times, the multi-job prediction launch matches the CP model of each
job's factors, a planted job reaches its target RMSE, and the memory model
bounds what a running job really holds."""
import time

import numpy as np
import pytest

from paper_2109_09534_gb300 import ntc, synth

from gpu_helpers import require_gpu

pytestmark = pytest.mark.gpu

SEED0 = 100


def small_jobs():
    specs = [synth.JobSpec(0.0, [300, 200, 150], 8, 60_000, 0, 11),
             synth.JobSpec(0.0, [250, 180, 120], 16, 50_000, 1, 12),
             synth.JobSpec(0.0, [120, 100, 80, 40], 8, 70_000, 0, 13),
             synth.JobSpec(0.0, [400, 150, 100], 32, 80_000, 1, 14)]
    return [(s, synth.serving_job(s, test_frac=0.02)) for s in specs]


def submit(server, k, spec, p, target=0.0, max_epochs=3, arrival=0.0):
    return server.submit(p.dims, p.rank, p.lam, p.c, p.idx_train, p.val_train, p.idx_test, p.val_test,
                         target, max_epochs, arrival=arrival, seed=SEED0 + k, init_seed=7,
                         storage_bf16=spec.storage_bf16)


def drain(server, ids, timeout=300.0):
    t0 = time.time()
    while True:
        server.step()
        if all(server.job_info(j)["state"] >= ntc.JOB_DONE for j in ids):
            return
        assert time.time() - t0 < timeout, "server did not finish"
        time.sleep(0.0005)


def factors_of(server, jid, p):
    return [server.get_factor(jid, m, p.dims[m], p.rank) for m in range(len(p.dims))]


def test_each_job_alone_equals_the_mix():
    torch = require_gpu()
    jobs = small_jobs()
    mixed = ntc.Server(64e9, 8)
    mixed.set_param("max_enqueue_per_step", 1)       # epochs of different jobs interleave tick by tick
    ids = [submit(mixed, k, s, p) for k, (s, p) in enumerate(jobs)]
    drain(mixed, ids)
    st = mixed.stats()
    assert st["done"] == len(jobs) and st["failed"] == 0
    assert st["peak_running"] == len(jobs)           # they really ran together
    assert st["epochs"] == 3 * len(jobs)
    for k, (s, p) in enumerate(jobs):
        info = mixed.job_info(ids[k])
        assert info["epochs"] == 3 and info["reached"] == 0 and info["rmse"] < info["rmse0"]
        alone = ntc.Server(64e9, 1)
        jid = submit(alone, k, s, p)
        drain(alone, [jid])
        # a plain handle fed the same inputs and seeds
        g = ntc.NTC(p.dims, p.rank, p.lam, stream=torch.cuda.current_stream().cuda_stream,
                    storage_bf16=s.storage_bf16, init_seed=7)
        g.set_observed(p.idx_train, p.val_train)
        for e in range(3):
            g.epoch(p.c, seed=SEED0 + k + e)
        for m, (a, b) in enumerate(zip(factors_of(alone, jid, p), factors_of(mixed, ids[k], p))):
            np.testing.assert_array_equal(a, b, err_msg=f"job {k} mode {m}")
            np.testing.assert_array_equal(a, g.get_factor(m), err_msg=f"job {k} mode {m} vs handle")
        assert alone.job_info(jid)["rmse"] == info["rmse"]
        g.close()
        alone.close()
    mixed.close()


def test_admission_keeps_the_budget_and_the_arrival_order():
    require_gpu()
    jobs = small_jobs()[:3]
    need = [ntc.job_bytes(ntc.job_desc(p.dims, p.rank, p.lam, p.c, p.idx_train, p.val_train, p.idx_test,
                                       p.val_test, 0.0, 2)) for _, p in jobs]
    budget = 1.2 * max(need)                         # room for one job at a time
    srv = ntc.Server(budget, 8)
    ids = [submit(srv, k, s, p, max_epochs=2) for k, (s, p) in enumerate(jobs)]
    drain(srv, ids)
    st = srv.stats()
    assert st["peak_running"] == 1 and st["peak_bytes"] <= budget and st["done"] == 3
    infos = [srv.job_info(j) for j in ids]
    for a, b in zip(infos, infos[1:]):
        assert b["t_admit"] >= a["t_done"]           # the next job waited for memory
    srv.close()


def test_a_job_is_not_admitted_before_it_arrives():
    require_gpu()
    s, p = small_jobs()[0]
    srv = ntc.Server(64e9, 8)
    with pytest.raises(ntc.NTCError) as e:
        srv.set_param("no_such_parameter", 1)
    assert e.value.status == ntc.NTC_ERR_ARG
    with pytest.raises(ntc.NTCError):
        srv.set_param("max_enqueue_per_step", 0)
    t_arr = srv.now() + 0.4
    jid = submit(srv, 0, s, p, max_epochs=1, arrival=t_arr)
    srv.step()
    assert srv.job_info(jid)["state"] == ntc.JOB_QUEUED
    drain(srv, [jid])
    info = srv.job_info(jid)
    assert info["t_admit"] >= t_arr and info["state"] == ntc.JOB_DONE
    srv.close()


def test_multi_job_prediction_matches_each_jobs_model():
    require_gpu()
    jobs = small_jobs()
    srv = ntc.Server(64e9, 8)
    ids = [submit(srv, k, s, p, max_epochs=1000) for k, (s, p) in enumerate(jobs)]
    for _ in range(50):
        srv.step()
        time.sleep(0.002)
    srv.sync()
    srv.step()
    assert all(srv.job_info(j)["state"] == ntc.JOB_RUNNING for j in ids)
    assert all(srv.job_info(j)["epochs"] >= 1 for j in ids)
    rng = np.random.default_rng(0)
    q_job, q_idx, want = [], [], []
    for k, (s, p) in enumerate(jobs):
        U = [f.astype(np.float64) for f in factors_of(srv, ids[k], p)]
        n = 500
        ix = np.stack([rng.integers(0, d, n) for d in p.dims], axis=1).astype(np.int32)
        model = np.ones((n, p.rank))
        for m in range(len(p.dims)):
            model *= U[m][ix[:, m]]
        q_job += [ids[k]] * n
        q_idx.append(np.pad(ix, ((0, 0), (0, 8 - ix.shape[1]))))
        want.append(model.sum(axis=1))
    perm = rng.permutation(len(q_job))               # jobs interleaved within the launch
    q_job = np.array(q_job)[perm]
    q_idx = np.concatenate(q_idx)[perm]
    want = np.concatenate(want)[perm]
    got = srv.predict(q_job, q_idx)
    assert np.max(np.abs(got - want) / np.maximum(np.abs(want), 1e-3)) <= 1e-5
    st = srv.stats()
    assert st["predict_launches"] == 1 and st["predict_queries"] == len(q_job)
    with pytest.raises(ntc.NTCError) as e:
        srv.predict([ids[0]], np.array([[jobs[0][1].dims[0] + 5, 0, 0]], np.int32))
    assert e.value.status == ntc.NTC_ERR_INDEX
    srv.close()


def test_planted_job_reaches_its_target():
    require_gpu()
    spec = synth.JobSpec(0.0, [100, 100, 100], 4, 200_000, 0, 21)
    p = synth.serving_job(spec, test_frac=0.02)
    srv = ntc.Server(64e9, 4)
    target = 1.5 * p.sigma
    jid = submit(srv, 0, spec, p, target=target, max_epochs=200)
    drain(srv, [jid])
    info = srv.job_info(jid)
    assert info["reached"] == 1 and info["rmse"] <= target < info["rmse0"]
    assert info["epochs"] < 200 and info["t_done"] > info["t_admit"] >= 0.0
    # done: the factors live on the host, queries are refused
    U0 = srv.get_factor(jid, 0, 100, 4)
    assert np.all(np.isfinite(U0)) and np.all(U0 >= 0)
    with pytest.raises(ntc.NTCError) as e:
        srv.predict([jid], np.zeros((1, 3), np.int32))
    assert e.value.status == ntc.NTC_ERR_STATE
    srv.close()


def test_memory_model_bounds_a_running_job():
    torch = require_gpu()
    spec = synth.JobSpec(0.0, [3000, 2000, 1000], 32, 2_000_000, 1, 31)
    p = synth.serving_job(spec, test_frac=0.01)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    srv = ntc.Server(64e9, 4)
    jid = submit(srv, 0, spec, p, max_epochs=1000)
    srv.step()
    srv.sync()
    srv.step()
    srv.sync()
    used = free0 - torch.cuda.mem_get_info()[0]
    model = srv.job_info(jid)["bytes"]
    assert srv.job_info(jid)["state"] == ntc.JOB_RUNNING
    assert used <= model, (used, model)
    assert used >= 0.25 * model, (used, model)
    srv.close()


def test_job_with_a_gram_wait_timeout_fails():
    """A served job whose epoch reports a tensor-core Gram wait that gave up
    (forced by the "test_gram_stall" hook on a rank-32 job with split rows)
    ends failed instead of taking its factors; a job submitted after the hook
    is cleared runs normally."""
    require_gpu()
    spec = synth.JobSpec(0.0, [60, 50, 40], 32, 400_000, 0, 21)   # rows of mode 0 hold ~6,600 > 4096
    p = synth.serving_job(spec, test_frac=0.02)
    srv = ntc.Server(64e9, 4)
    srv.set_param("test_gram_stall", 20000)
    bad = submit(srv, 0, spec, p, max_epochs=2)
    srv.set_param("test_gram_stall", 0)
    good = submit(srv, 1, spec, p, max_epochs=2)
    drain(srv, [bad, good])
    assert srv.job_info(bad)["state"] == ntc.JOB_FAILED
    info = srv.job_info(good)
    assert info["state"] == ntc.JOB_DONE and info["epochs"] == 2 and info["rmse"] < info["rmse0"]
    assert srv.stats()["failed"] == 1
    srv.close()


@pytest.mark.parametrize("epochs", [1, 2])
def test_served_job_in_a_mix_matches_the_oracle(epochs):
    """A small job served beside three others (epochs of different jobs
    interleaved tick by tick) against the FP64 oracle run from the same initial
    factors (drawn by the oracle's rule, rounded to float32 as the device stores
    them) with the same per-epoch seeds: within 1e-5 (Frobenius) and 1e-4 (per
    row) relative after each of its epochs."""
    require_gpu()
    import oracle

    from gpu_helpers import assert_factor_close
    jobs = small_jobs()
    srv = ntc.Server(64e9, 8)
    srv.set_param("max_enqueue_per_step", 1)
    target_k = 0   # the 3-way rank-8 FP32 job
    ids = []
    for k, (s, p) in enumerate(jobs):
        ids.append(submit(srv, k, s, p, max_epochs=epochs if k == target_k else 3))
    drain(srv, ids)
    assert srv.stats()["failed"] == 0
    s, p = jobs[target_k]
    assert s.storage_bf16 == 0
    o = oracle.Oracle(p.dims, p.rank, p.lam)
    o.set_observed(p.idx_train, p.val_train.astype(np.float64))
    o.init_factors(7)
    for m in range(len(p.dims)):
        o.set_factor(m, o.get_factor(m).astype(np.float32).astype(np.float64))
    for e in range(epochs):
        o.epoch(p.c, seed=SEED0 + target_k + e)
    got = factors_of(srv, ids[target_k], p)
    for m in range(len(p.dims)):
        assert_factor_close(got[m], o.get_factor(m), 1e-5, 1e-4, f"mode {m} after {epochs} epochs")
    srv.close()
