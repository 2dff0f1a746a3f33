"""Batched scans (bootstrap resamples x label permutations) against the same
jobs run one by one through mdfs_max_ig on explicitly resampled data, and one
job against the FP64 oracle."""
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
