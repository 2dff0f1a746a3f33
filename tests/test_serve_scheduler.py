"""Host logic of the continuous-batching request loop, with a fake executor
(no GPU): admission under the memory budget, slot limits, arrival order,
failure isolation and latency bookkeeping."""
import threading
import time

import numpy as np
import pytest

from paper_1811_00631_gb300 import serve


class FakeJob:
    def __init__(self, need, dur, tag, fail=False):
        self.x = np.zeros((need, 1), dtype=np.float32)  # M encodes the memory need below
        self.y = np.zeros(1, dtype=np.uint8)
        self.k, self.divisions, self.discretizations = 1, 1, 1
        self.dur, self.tag, self.fail = dur, tag, fail


def _estimate(M, N, k, div, D, itemsize):
    return M


def _run(jobs, n_slots, budget):
    active = []
    lock = threading.Lock()
    log = []

    def executor(job, slot):
        with lock:
            active.append(job.tag)
            log.append(("start", job.tag, slot, list(active)))
        time.sleep(job.dur)
        with lock:
            active.remove(job.tag)
        if job.fail:
            raise ValueError(f"job {job.tag} failed")
        return (np.array([job.tag]), None, None, None, None, None)

    srv = serve.Server(n_slots=n_slots, memory_budget=budget, executor=executor, estimate=_estimate)
    futs = [srv.submit(j) for j in jobs]
    res = []
    for f in futs:
        try:
            res.append(f.result(timeout=20))
        except ValueError as e:
            res.append(e)
    srv.close()
    return srv, res, log


def test_slots_and_budget_bound_concurrency():
    jobs = [FakeJob(need=40, dur=0.05, tag=i) for i in range(12)]
    srv, res, log = _run(jobs, n_slots=4, budget=100)
    # at most two 40-byte jobs fit in 100 bytes even though 4 slots exist
    assert srv.peak_in_use <= 100
    assert srv.peak_running == 2
    assert max(len(a) for _, _, _, a in log) <= 2
    assert [r.ig[0] for r in res] == list(range(12))


def test_arrival_order_is_kept_and_big_jobs_are_not_starved():
    jobs = [FakeJob(need=10, dur=0.03, tag=0), FakeJob(need=90, dur=0.03, tag=1)] + \
           [FakeJob(need=10, dur=0.03, tag=i) for i in range(2, 8)]
    srv, res, log = _run(jobs, n_slots=4, budget=100)
    starts = [t for kind, t, _, _ in log if kind == "start"]
    assert starts == sorted(starts)  # head-of-line admission: start order == arrival order
    assert srv.peak_in_use <= 100


def test_failure_is_isolated_and_oversize_is_rejected():
    jobs = [FakeJob(need=10, dur=0.01, tag=0), FakeJob(need=10, dur=0.01, tag=1, fail=True),
            FakeJob(need=10, dur=0.01, tag=2)]
    srv, res, _ = _run(jobs, n_slots=2, budget=100)
    assert isinstance(res[1], ValueError)
    assert res[0].ig[0] == 0 and res[2].ig[0] == 2
    srv2 = serve.Server(n_slots=1, memory_budget=5, executor=lambda j, s: None, estimate=_estimate)
    with pytest.raises(MemoryError):
        srv2.submit(FakeJob(need=10, dur=0, tag=9)).result(timeout=5)
    srv2.close()


def test_latency_bookkeeping():
    jobs = [FakeJob(need=1, dur=0.02, tag=i) for i in range(6)]
    _, res, _ = _run(jobs, n_slots=1, budget=10)
    lat = [r.latency for r in res]
    assert all(l >= 0.02 for l in lat)
    assert lat == sorted(lat)  # one slot: later arrivals wait longer
    st = serve.latency_stats(res)
    assert st["p50_s"] <= st["p99_s"] and st["n"] == 6


def test_device_byte_estimate_grows_with_the_work():
    a = serve.job_device_bytes(500, 2000, 2, 1, 30)
    b = serve.job_device_bytes(500, 2000, 3, 1, 30)
    c = serve.job_device_bytes(1000, 2000, 3, 1, 30)
    assert a < b < c
    assert b > 30 * 500 * 500 * 8  # pair records of the k = 3 path


def test_device_byte_estimate_covers_the_higher_order_tables():
    """k = 4 holds the triple tables of a chunk of discretisations (chunks fit
    4 GB, at least one discretisation); k = 5 also the quadruple tables, which
    alone are 12 C(M,4) bytes per discretisation."""
    import math
    k4 = serve.job_device_bytes(500, 2000, 4, 1, 30)
    k5 = serve.job_device_bytes(500, 2000, 5, 1, 1)
    assert k4 > 12 * math.comb(500, 3) * 10  # at least ten discretisations of triple tables
    assert k4 < 8 << 30                      # but chunked, not all thirty at once
    assert k5 > 12 * math.comb(500, 4)       # one discretisation of quadruple tables
    assert serve.job_device_bytes(200, 2000, 2, 1, 30) > 30 * 200 * 2048  # the k = 2 one-hot operand


def test_jobs_past_their_start_deadline_are_dropped():
    """A queued job that cannot start within its deadline fails with
    TimeoutError and never runs; jobs without a deadline, or with a deadline
    they meet, run as usual."""
    ran = []

    def executor(job, slot):
        ran.append(job.tag)
        time.sleep(job.dur)
        return (np.array([job.tag]), None, None, None, None, None)

    slow = FakeJob(need=1, dur=0.3, tag=0)
    late = FakeJob(need=1, dur=0.01, tag=1)
    late.deadline_s = 0.05
    patient = FakeJob(need=1, dur=0.01, tag=2)
    patient.deadline_s = 10.0
    plain = FakeJob(need=1, dur=0.01, tag=3)
    srv = serve.Server(n_slots=1, memory_budget=10, executor=executor, estimate=_estimate)
    futs = [srv.submit(j) for j in (slow, late, patient, plain)]
    with pytest.raises(TimeoutError):
        futs[1].result(timeout=5)
    assert [f.result(timeout=5).ig[0] for f in (futs[0], futs[2], futs[3])] == [0, 2, 3]
    srv.close()
    assert srv.expired == 1 and ran == [0, 2, 3]


def test_deadline_drops_a_job_blocked_behind_the_memory_budget():
    """An idle slot wakes up for the earliest deadline: a job that waits
    behind a memory-bound head-of-line job expires while the budget is held."""
    def executor(job, slot):
        time.sleep(job.dur)
        return (np.array([job.tag]), None, None, None, None, None)

    big = FakeJob(need=8, dur=1.5, tag=0)
    waiting = FakeJob(need=8, dur=0.01, tag=1)
    waiting.deadline_s = 0.1
    srv = serve.Server(n_slots=2, memory_budget=10, executor=executor, estimate=_estimate)
    t0 = time.perf_counter()
    f_big, f_wait = srv.submit(big), srv.submit(waiting)
    with pytest.raises(TimeoutError):
        f_wait.result(timeout=5)
    assert time.perf_counter() - t0 < 1.2  # dropped before the big job released the budget
    assert f_big.result(timeout=5).ig[0] == 0
    srv.close()


def test_per_job_records(tmp_path):
    """With log_path set, every job leaves one JSON line: its shape and work,
    queue wait, run time, latency and status (ok, the error, or expired)."""
    import json

    def executor(job, slot):
        time.sleep(job.dur)
        if job.fail:
            raise ValueError("bad job")
        return (np.array([job.tag]), None, None, None, None, None)

    log = tmp_path / "jobs.jsonl"
    jobs = [FakeJob(need=2, dur=0.05, tag=0), FakeJob(need=2, dur=0.01, tag=1, fail=True),
            FakeJob(need=2, dur=0.01, tag=2)]
    jobs[2].deadline_s = 0.01
    srv = serve.Server(n_slots=1, memory_budget=10, executor=executor, estimate=_estimate, log_path=str(log))
    futs = [srv.submit(j) for j in jobs]
    for f in futs:
        try:
            f.result(timeout=5)
        except (ValueError, TimeoutError):
            pass
    srv.close()
    recs = {r["tag"]: r for r in map(json.loads, log.read_text().splitlines())}
    assert set(recs) == {0, 1, 2}
    assert recs[0]["status"] == "ok" and recs[0]["run_s"] >= 0.05 and recs[0]["M"] == 2 and recs[0]["evals"] == 2.0
    assert recs[0]["latency_s"] >= recs[0]["run_s"] and recs[0]["queue_s"] >= 0
    assert recs[1]["status"].startswith("error: ValueError")
    assert recs[2]["status"] == "expired" and recs[2]["run_s"] is None


def test_unwritable_record_does_not_stop_the_slot(tmp_path):
    """A log path that cannot be written (here a directory) only counts the
    lost records; every job still completes on the one slot."""
    def executor(job, slot):
        return (np.array([job.tag]), None, None, None, None, None)

    srv = serve.Server(n_slots=1, memory_budget=10, executor=executor, estimate=_estimate, log_path=str(tmp_path))
    futs = [srv.submit(FakeJob(need=1, dur=0, tag=i)) for i in range(3)]
    assert [f.result(timeout=5).ig[0] for f in futs] == [0, 1, 2]
    srv.close()
    assert srv.log_errors == 3


def test_retained_workspaces_are_charged_and_freed_when_needed():
    """The library keeps a slot's buffers after its job.  A slot that ran a job
    using one group of buffers and then takes a job using another holds both;
    the scheduler charges what every slot retains, frees a slot's workspace
    when the merged bytes would pass the budget, and has idle slots free
    theirs when the head job does not fit beside them."""
    def est(M, N, k, div, D, itemsize):
        return {f"group{k}": M}

    def executor(job, slot):
        time.sleep(job.dur)
        return (np.array([job.tag]), None, None, None, None, None)

    def job(need, group, tag):
        j = FakeJob(need=need, dur=0.02, tag=tag)
        j.k = group
        return j

    # merged groups that fit: both stay resident, nothing is freed
    released = []
    srv = serve.Server(n_slots=1, memory_budget=100, executor=executor, estimate=est,
                       release_workspace=released.append)
    for f in [srv.submit(job(30, 1, 0)), srv.submit(job(30, 2, 1))]:
        f.result(timeout=5)
    assert srv.in_use == 60 and released == []
    # merged groups past the budget: the slot frees its workspace first
    for f in [srv.submit(job(50, 3, 2))]:
        f.result(timeout=5)
    assert released == [0] and srv.in_use == 50 and srv.peak_in_use <= 100
    srv.close()

    # two slots: the idle slot that retains 60 bytes frees them for a 50-byte job
    for _ in range(3):
        released = []
        srv = serve.Server(n_slots=2, memory_budget=100, executor=executor, estimate=est,
                           release_workspace=released.append)
        srv.submit(job(60, 1, 0)).result(timeout=5)
        assert srv.in_use == 60
        srv.submit(job(50, 2, 1)).result(timeout=5)
        srv.close()
        assert len(released) == 1 and srv.in_use == 50 and srv.peak_in_use <= 100


def test_estimate_parts_add_up():
    parts = serve.job_device_parts(500, 2000, 3, 1, 30)
    assert {"inputs", "planes", "onehot", "k3tc"} <= set(parts)
    assert sum(parts.values()) == serve.job_device_bytes(500, 2000, 3, 1, 30)
