"""The bounded device-side waits of the tensor-core triple kernel.

Every mbarrier wait of the kernel gives up after a time limit, records an
error, drains the copies and MMAs in flight, frees its tensor memory and lets
the kernel exit, so that the call returns MDFS_ETIMEOUT and the context stays
usable.  A test hook (mdfs_testing_k3_wait_fault) shortens the limit to 20 ms
and has the TMA producer of one CTA never fill one pipeline stage: the wait of
that stage's consumers runs out.  The next call on the same stream must be
complete and match the oracle.
"""
import time

import numpy as np
import pytest

import argmax_rule
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_00631_gb300 import build
    build.build()
    return torch


def test_k3_wait_runs_out_then_the_next_call_is_correct(cuda):
    torch = cuda
    from paper_1811_00631_gb300 import mdfs
    rng = np.random.default_rng(12)
    M, N, D = 60, 500, 2
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((x[2] > 0) ^ (x[30] > 0) ^ (x[59] > 0) ^ (rng.random(N) < 0.1)).astype(np.uint8)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    mdfs.testing_k3_wait_fault(withhold_kb=1, wait_ns=20_000_000)
    t0 = time.perf_counter()
    with pytest.raises(mdfs.MdfsError) as e:
        mdfs.max_ig(xt, yt, 3, 1, D, 0.5, 0.25, 5)
    assert e.value.code == -6 and "timed out" in str(e.value)
    assert time.perf_counter() - t0 < 10.0
    # the hook is one-shot: the same scan again, on the same stream
    ig, tu, di = (t.cpu().numpy() for t in mdfs.max_ig(xt, yt, 3, 1, D, 0.5, 0.25, 5))
    codes = oracle.discretize(x, 1, D, 0.5, 5)
    ref = oracle.max_ig(codes, y, 2, 3, 0.25)
    for i in range(M):
        o = ref["ig"][i]
        assert abs(float(ig[i]) - o) <= argmax_rule.tol(o)
        if di[i] != ref["disc"][i] or tuple(tu[i]) != tuple(ref["tuples"][i]):
            alt = oracle.ig_one(codes, y, 2, 0.25, int(di[i]), i, [int(v) for v in tu[i]])
            argmax_rule.check_alternative(o, ref["second"][i], alt, f"var {i}")


def test_hook_arguments(cuda):
    from paper_1811_00631_gb300 import mdfs
    with pytest.raises(mdfs.MdfsError):
        mdfs.testing_k3_wait_fault(-2, 0)
    with pytest.raises(mdfs.MdfsError):
        mdfs.testing_k3_wait_fault(0, -1)
    mdfs.testing_k3_wait_fault()  # disarm
