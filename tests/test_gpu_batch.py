"""Batched scans (bootstrap resamples x label permutations) against the same
jobs run one by one through mdfs_max_ig on explicitly resampled data, and one
job against the FP64 oracle."""
import numpy as np
import pytest

import argmax_rule
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


def _jobs(N, n_folds, n_perms, seed):
    idx, yperm = synth.bootstrap_jobs(N, n_folds=n_folds, n_perms=n_perms, seed=seed)
    si = np.repeat(idx, n_perms, axis=0)           # job j = fold j // n_perms, permutation j % n_perms
    yp = np.tile(yperm, (n_folds, 1))
    return si.astype(np.int32), yp.astype(np.int32)


@pytest.mark.parametrize("k,div,M,N,D", [(1, 2, 40, 300, 3), (2, 1, 70, 256, 2), (2, 2, 45, 333, 2),
                                        (3, 1, 140, 200, 2), (3, 2, 24, 150, 1), (4, 1, 40, 300, 2),
                                        (5, 1, 24, 200, 2)])
def test_batch_equals_jobs_one_by_one(cuda, k, div, M, N, D):
    torch = cuda
    from paper_1811_00631_gb300 import mdfs
    ds = synth.xor_pairs(N=N, M=M, n_pairs=3, seed=M + N)
    si, yp = _jobs(N, 3, 2, seed=k)
    x = torch.from_numpy(ds.x).cuda()
    y = torch.from_numpy(ds.y).cuda()
    ig, tu, di = mdfs.max_ig_batch(x, y, torch.from_numpy(si).cuda(), yp, k=k, divisions=div, discretizations=D,
                                   range_=0.5, pc_xi=0.25, seed=13)
    torch.cuda.synchronize()
    for j in range(len(si)):
        xj = np.ascontiguousarray(ds.x[:, si[j]])
        yj = ds.y[yp[j][si[j]]]
        w_ig, w_tu, w_di = mdfs.max_ig(xj, yj, k, div, D, 0.5, 0.25, 13)
        assert np.array_equal(ig[j].cpu().numpy(), w_ig), f"job {j}"
        assert np.array_equal(di[j].cpu().numpy(), w_di)
        if k > 1:
            assert np.array_equal(tu[j].cpu().numpy(), w_tu)


def test_batch_job_against_oracle_and_host_pointers(cuda):
    from paper_1811_00631_gb300 import mdfs
    ds = synth.xor_pairs(N=400, M=60, n_pairs=4, seed=3)
    si, yp = _jobs(400, 2, 2, seed=9)
    ig, tu, di = mdfs.max_ig_batch(ds.x, ds.y, si, yp, k=2, divisions=2, discretizations=3, range_=0.4,
                                   pc_xi=0.25, seed=5)
    j = 3
    xj = np.ascontiguousarray(ds.x[:, si[j]])
    yj = ds.y[yp[j][si[j]]]
    codes = oracle.discretize(xj, 2, 3, 0.4, 5)
    ref = oracle.max_ig(codes, yj, 3, 2, 0.25)
    err = np.abs(ig[j].astype(np.float64) - ref["ig"])
    assert np.all(err <= 1e-4 + 1e-5 * np.abs(ref["ig"]))


def test_batch_rejects_bad_indices(cuda):
    from paper_1811_00631_gb300 import mdfs
    ds = synth.xor_small()
    si = np.zeros((2, 200), np.int32)
    si[1, 7] = 200
    with pytest.raises(mdfs.MdfsError) as e:
        mdfs.max_ig_batch(ds.x, ds.y, si, None, k=2)
    assert e.value.code in (-1, -2)


@pytest.mark.parametrize("k,div,M,N", [(2, 1, 300, 500), (2, 2, 90, 400), (3, 1, 160, 300), (3, 2, 40, 200),
                                      (1, 1, 50, 200), (4, 1, 60, 300), (5, 1, 40, 300)])
def test_sharded_scan_merges_to_the_unsharded_result(cuda, k, div, M, N):
    """Three shards scanned one after another on one GPU, merged by unsigned
    maximum, decode to exactly the result of the unsharded scan."""
    from paper_1811_00631_gb300 import mdfs, shard
    ds = synth.xor_pairs(N=N, M=M, n_pairs=4, seed=M)
    want = mdfs.max_ig(ds.x, ds.y, k, div, 3, 0.5, 0.25, 21)
    keys = shard.merge([mdfs.max_ig_shard(ds.x, ds.y, k, div, 3, 0.5, 0.25, 21, s, 3) for s in range(3)])
    got = mdfs.decode_keys(keys, k)
    for a, b in zip(got, want):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("k", [3, 5])
def test_resumable_scan_equals_the_unsharded_scan(cuda, tmp_path, k):
    """The checkpointed sharded scan, first run and a resumed run that finds
    every shard on disk, decode to exactly the unsharded result."""
    from paper_1811_00631_gb300 import mdfs, shard
    ds = synth.xor_pairs(N=300, M=30 if k == 5 else 120, n_pairs=3, seed=k)
    want = mdfs.max_ig(ds.x, ds.y, k, 1, 2, 0.5, 0.25, 8)
    for _ in range(2):
        got = shard.max_ig_resumable(ds.x, ds.y, k, 1, 2, 0.5, 0.25, 8, 4, str(tmp_path))
        for a, b in zip(got, want):
            assert np.array_equal(a, b)


def test_batched_full_size_sampled(cuda):
    """The batched workload at full size, in the launch that bench.py --batched
    times: N = 1000 x M = 20000 (100 planted XOR pairs), 3 classes, 10
    discretisations, 16 bootstrap folds x 4 label permutations = 64 jobs in one
    call.  Sampled jobs and variables are compared with the FP64 oracle (IG
    within 1e-4 + 1e-5 |o|; an argmax that differs only where the oracle's
    top two lie within that tolerance), one job with the single-job scan bit for bit, and job 0 (the
    unpermuted labels) must name the planted partner of every XOR member."""
    torch = cuda
    from paper_1811_00631_gb300 import mdfs
    N, M, D, div, r, xi, seed = 1000, 20000, 10, 2, 0.5, 0.25, 1
    c = div + 1
    ds = synth.xor_pairs(N=N, M=M, n_pairs=100, seed=4)
    si, yp = _jobs(N, 16, 4, seed=5)
    xt, yt = torch.from_numpy(ds.x).cuda(), torch.from_numpy(ds.y).cuda()
    ig, tu, di = mdfs.max_ig_batch(xt, yt, torch.from_numpy(si).cuda(), torch.from_numpy(yp).cuda(), k=2,
                                   divisions=div, discretizations=D, range_=r, pc_xi=xi, seed=seed)
    torch.cuda.synchronize()
    ig, tu, di = ig.cpu().numpy(), tu.cpu().numpy(), di.cpu().numpy()
    assert ig.shape == (64, M) and tu.shape == (64, M, 1) and di.shape == (64, M)

    pairs = ds.info["pairs"]
    found = sum(int(tu[0, a, 0] == b) + int(tu[0, b, 0] == a) for a, b in pairs)
    assert found == 2 * len(pairs), f"job 0 names {found} of {2 * len(pairs)} planted partners"

    rng = np.random.default_rng(17)
    for j in (0, 29, 63):
        xj = np.ascontiguousarray(ds.x[:, si[j]])
        yj = ds.y[yp[j][si[j]]]
        codes = oracle.discretize(xj, div, D, r, seed)
        a, b = pairs[rng.integers(len(pairs))]
        variables = np.array(sorted({int(a), int(b), *rng.choice(M, 6, replace=False).tolist()}), np.int32)
        ref = oracle.max_ig(codes, yj, c, 2, xi, variables=variables)
        for row, i in enumerate(variables):
            o = ref["ig"][row]
            assert abs(float(ig[j, i]) - o) <= argmax_rule.tol(o), f"job {j} var {i}: gpu {ig[j, i]!r} oracle {o!r}"
            if di[j, i] != ref["disc"][row] or tu[j, i, 0] != ref["tuples"][row, 0]:
                m = int(tu[j, i, 0])
                assert 0 <= m < M and m != i and 0 <= di[j, i] < D
                alt = oracle.ig_one(codes, yj, c, xi, int(di[j, i]), int(i), [m])
                argmax_rule.check_alternative(o, ref["second"][row], alt, f"job {j} var {i}")

    j = 63
    w_ig, w_tu, w_di = mdfs.max_ig(torch.from_numpy(np.ascontiguousarray(ds.x[:, si[j]])).cuda(),
                                   torch.from_numpy(ds.y[yp[j][si[j]]]).cuda(), 2, div, D, r, xi, seed)
    torch.cuda.synchronize()
    assert np.array_equal(ig[j], w_ig.cpu().numpy())
    assert np.array_equal(tu[j], w_tu.cpu().numpy())
    assert np.array_equal(di[j], w_di.cpu().numpy())


@pytest.mark.parametrize("div,M,N,chunk_bytes", [(1, 50, 300, None), (2, 33, 257, None), (1, 40, 200, 1)])
def test_batch_chunks_equal_jobs_one_by_one(cuda, monkeypatch, div, M, N, chunk_bytes):
    """k = 2 batches of 20 jobs: more jobs than one tensor-core launch holds, or
    (a one-byte operand budget) one job per launch.  Every job equals the
    single-job scan of its resampled data bit for bit, whatever the chunking."""
    torch = cuda
    from paper_1811_00631_gb300 import mdfs
    if chunk_bytes is not None:
        monkeypatch.setenv("MDFS_BATCH_BYTES", str(chunk_bytes))
    ds = synth.xor_pairs(N=N, M=M, n_pairs=3, seed=N)
    si, yp = _jobs(N, 5, 4, seed=div + N)
    x = torch.from_numpy(ds.x).cuda()
    y = torch.from_numpy(ds.y).cuda()
    ig, tu, di = mdfs.max_ig_batch(x, y, torch.from_numpy(si).cuda(), torch.from_numpy(yp).cuda(), k=2,
                                   divisions=div, discretizations=3, range_=0.5, pc_xi=0.25, seed=7)
    torch.cuda.synchronize()
    ig, tu, di = ig.cpu().numpy(), tu.cpu().numpy(), di.cpu().numpy()
    for j in range(len(si)):
        xj = np.ascontiguousarray(ds.x[:, si[j]])
        yj = ds.y[yp[j][si[j]]]
        w_ig, w_tu, w_di = mdfs.max_ig(xj, yj, 2, div, 3, 0.5, 0.25, 7)
        assert np.array_equal(ig[j], w_ig), f"job {j}"
        assert np.array_equal(tu[j], w_tu), f"job {j}"
        assert np.array_equal(di[j], w_di), f"job {j}"


def test_batch_names_the_single_class_job(cuda):
    """A job whose resample holds one class only is refused with its index
    before any scan runs."""
    from paper_1811_00631_gb300 import mdfs
    ds = synth.xor_pairs(N=200, M=20, n_pairs=2, seed=1)
    si = np.tile(np.arange(200, dtype=np.int32), (3, 1))
    one = int(np.flatnonzero(ds.y == 1)[0])
    si[2, :] = one
    with pytest.raises(mdfs.MdfsError) as e:
        mdfs.max_ig_batch(ds.x, ds.y, si, None, k=2)
    assert "job 2" in str(e.value)
