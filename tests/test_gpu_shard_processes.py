"""The sharded scan across processes (the multi-GPU split of the tuple space):
two processes on the one GPU each scan their share of the tuple tiles with
mdfs_max_ig_shard, merge the packed keys with one all-reduce (MAX) over gloo,
and decode them; the result must equal mdfs_max_ig bit for bit, for k = 2
(tensor-core pair kernel) and k = 3 (tensor-core triple kernel), and at the
bench step's size (2000 x 500, 30 discretisations).

The two processes' kernels never wait on one another: each rank scans and
then meets the other only in the host-side all-reduce."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_00631_gb300 import build
    build.build()
    return torch


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, case, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from paper_1811_00631_gb300 import mdfs, shard, synth
    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}")
    try:
        torch.cuda.set_device(0)
        ds = synth.madelon_like() if case["full"] else synth.madelon_like(N=1300, M=260, seed=9)
        x, y = torch.from_numpy(ds.x).cuda(), torch.from_numpy(ds.y).cuda()
        for k in (2, 3):
            keys = mdfs.max_ig_shard(x, y, k, case["div"] if k == 2 else 1, case["D"], 0.5, 0.25, 11,
                                     shard=rank, n_shards=world)
            merged = shard.allreduce_max(keys)
            if rank == 0:
                np.save(os.path.join(out_dir, f"keys_k{k}.npy"), merged)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", [{"full": False, "div": 2, "D": 3}, {"full": True, "div": 1, "D": 30}],
                         ids=["small_c3", "bench_size"])
def test_two_processes_merge_to_the_unsharded_scan(cuda, case, tmp_path):
    torch = cuda
    import torch.multiprocessing as mp

    from paper_1811_00631_gb300 import mdfs, synth
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, case, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    ds = synth.madelon_like() if case["full"] else synth.madelon_like(N=1300, M=260, seed=9)
    x, y = torch.from_numpy(ds.x).cuda(), torch.from_numpy(ds.y).cuda()
    for k in (2, 3):
        want = [t.cpu().numpy() for t in mdfs.max_ig(x, y, k, case["div"] if k == 2 else 1, case["D"], 0.5, 0.25, 11)]
        got = mdfs.decode_keys(np.load(tmp_path / f"keys_k{k}.npy"), k)
        for a, b, name in zip(want, got, ("ig", "tuples", "disc")):
            assert np.array_equal(a, b), f"k = {k}: {name} differs"
