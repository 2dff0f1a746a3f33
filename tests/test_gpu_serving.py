"""The serving loop on the GPU: a Poisson stream of mixed jobs (k = 1..3, mixed
N, M, divisions, float32 and int8), admitted into concurrent slots; every
result equals the same job run alone, bit for bit, jobs overlap, and the jobs
small enough for the FP64 oracle match it (IG within 1e-4 + 1e-5 |IG|; the
fit's p-values equal the oracle fit of the same IG)."""
import math
import time

import numpy as np
import pytest

import oracle
from paper_1811_00631_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_00631_gb300 import build
    build.build()
    return torch


def test_mix_equals_alone_and_overlaps(cuda):
    from paper_1811_00631_gb300 import mdfs, serve
    specs = synth.serving_mix(n_jobs=24, seed=11, rate_hz=200.0, n_range=(100, 1500), m_range=(40, 300),
                              max_work=2e9)
    jobs = []
    for sp in specs:
        x, y = synth.serving_data(sp)
        jobs.append(serve.Job(x=x, y=y, k=sp["k"], divisions=sp["divisions"], discretizations=sp["discretizations"],
                              range_=0.5, pc_xi=0.25, seed=sp["seed"], alpha=0.05, tag=sp["job"]))
    with serve.Server(n_slots=4) as srv:
        t0 = time.perf_counter()
        futs = []
        for sp, job in zip(specs, jobs):
            delay = sp["arrival"] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            futs.append(srv.submit(job))
        results = [f.result(timeout=120) for f in futs]
    assert srv.peak_running >= 2
    assert srv.peak_in_use <= srv.budget
    for job, r in zip(jobs, results):
        ig, tu, di = mdfs.max_ig(job.x, job.y, job.k, job.divisions, job.discretizations, job.range_, job.pc_xi,
                                 job.seed)
        assert np.array_equal(r.ig, ig), f"job {job.tag}"
        assert np.array_equal(r.disc, di)
        if job.k > 1:
            assert np.array_equal(r.tuples, tu)
        assert r.latency > 0
    st = serve.latency_stats(results)
    assert st["p99_s"] >= st["p50_s"] > 0
    checked = 0
    for sp, job, r in zip(specs, jobs, results):
        M, N = job.x.shape
        if math.comb(M, job.k) * job.discretizations * N > 3e8:
            continue
        c = job.divisions + 1
        codes = oracle.discretize(np.asarray(job.x, dtype=np.float32), job.divisions, job.discretizations, job.range_,
                                  job.seed)
        ref = oracle.max_ig(codes, job.y, c, job.k, job.pc_xi)
        assert np.all(np.abs(r.ig - ref["ig"]) <= 1e-4 + 1e-5 * np.abs(ref["ig"])), f"job {job.tag}"
        if r.p_values is not None:
            p_ref, _, _ = oracle.ig_lim(r.ig.astype(np.float64), job.k, job.divisions, alpha=job.alpha)
            assert np.allclose(r.p_values, p_ref, rtol=1e-9, atol=1e-12), f"job {job.tag}"
        checked += 1
    assert checked >= 5


def test_full_serving_mix_sampled(cuda):
    """The serving configuration at full size, as bench.py generates it: 512
    jobs with k in 1..3, N in [100, 5000], M log-uniform in [100, 5000] (capped
    at C(M,k) D N <= 2e10), float32 and int8, 1-3 divisions, 5-30
    discretisations, arriving as a Poisson stream into 4 slots.  Every result
    equals the job run alone bit for bit; jobs whose rows the oracle computes
    quickly are checked on sampled variables against the FP64 oracle."""
    from paper_1811_00631_gb300 import mdfs, serve
    specs = synth.serving_mix(n_jobs=512, seed=17, rate_hz=1.0, n_range=(100, 5000), m_range=(100, 5000),
                              max_work=2e10)
    jobs = []
    for sp in specs:
        x, y = synth.serving_data(sp)
        jobs.append(serve.Job(x=x, y=y, k=sp["k"], divisions=sp["divisions"], discretizations=sp["discretizations"],
                              range_=0.5, pc_xi=0.25, seed=sp["seed"], alpha=0.05, tag=sp["job"]))
    rng = np.random.default_rng(5)
    gaps = rng.exponential(1.0 / 400.0, size=len(jobs))
    with serve.Server(n_slots=4) as srv:
        t0 = time.perf_counter()
        futs = []
        for job, g in zip(jobs, np.cumsum(gaps)):
            delay = g - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            futs.append(srv.submit(job))
        results = [f.result(timeout=600) for f in futs]
    assert srv.peak_running >= 2
    assert srv.peak_in_use <= srv.budget
    for job, r in zip(jobs, results):
        ig, tu, di = mdfs.max_ig(job.x, job.y, job.k, job.divisions, job.discretizations, job.range_, job.pc_xi,
                                 job.seed)
        assert np.array_equal(r.ig, ig), f"job {job.tag}"
        assert np.array_equal(r.disc, di)
        if job.k > 1:
            assert np.array_equal(r.tuples, tu)
    checked = 0
    for job, r in zip(jobs, results):
        M, N = job.x.shape
        D, c = job.discretizations, job.divisions + 1
        if M * N * D > 1e8 or math.comb(M - 1, job.k - 1) * D * N > 3e8:
            continue
        codes = oracle.discretize(np.asarray(job.x, dtype=np.float32), job.divisions, D, job.range_, job.seed)
        variables = np.array(sorted({0, int(rng.integers(1, M))}), np.int32)
        ref = oracle.max_ig(codes, job.y, c, job.k, job.pc_xi, variables=variables)
        got = r.ig[variables].astype(np.float64)
        assert np.all(np.abs(got - ref["ig"]) <= 1e-4 + 1e-5 * np.abs(ref["ig"])), f"job {job.tag}"
        checked += 1
        if checked == 40:
            break
    assert checked >= 20
