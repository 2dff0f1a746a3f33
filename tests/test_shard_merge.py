"""Host logic of the sharded scan: the key format and the MAX merge across
ranks (torch.distributed, gloo, world size 2, on CPU)."""
import os
import socket
import time

import numpy as np
import pytest

from paper_1811_00631_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _candidates(seed, M=37, n=4000):
    """Random candidate (variable, IG, index) triples with exact ties."""
    rng = np.random.default_rng(seed)
    var = rng.integers(0, M, n)
    ig = np.round(rng.normal(0, 3, n), 1).astype(np.float32)  # many exact ties, both signs
    idx = rng.integers(0, 2**31, n).astype(np.uint64)
    return var, ig, idx


def _reference(var, ig, idx, M):
    """Max IG per variable, ties to the lowest index (plain loops)."""
    best = [None] * M
    for v, g, i in zip(var, ig, idx):
        if best[v] is None or g > best[v][0] or (g == best[v][0] and i < best[v][1]):
            best[v] = (g, i)
    return best


def _keys_of(var, ig, idx, M):
    keys = np.zeros(M, np.uint64)
    packed = shard.pack(ig, idx)
    for v, k in zip(var, packed):
        keys[v] = max(keys[v], k)
    return keys


def test_key_order_is_ig_then_lowest_index():
    ig = np.array([-5.5, -0.0, 0.0, 1e-30, 2.0, 2.0, np.float32(3e38)], np.float32)
    idx = np.array([1, 2, 3, 4, 9, 5, 0], np.uint64)
    keys = shard.pack(ig, idx)
    order = np.argsort(keys)
    assert list(order[-2:]) == [5, 6]               # 2.0 with index 5 beats 2.0 with index 9
    assert keys[5] > keys[4] and keys[0] < keys[1] < keys[3]
    g, i = shard.unpack(keys)
    assert np.array_equal(g, ig) and np.array_equal(i.astype(np.uint64), idx)
    # flipping bit 63 maps unsigned order onto signed order
    assert np.array_equal(np.argsort(shard.to_signed_order(keys), kind="stable"), np.argsort(keys, kind="stable"))
    assert np.array_equal(shard.from_signed_order(shard.to_signed_order(keys)), keys)


def test_merge_of_shards_equals_global_max():
    M = 37
    var, ig, idx = _candidates(1, M)
    parts = np.array_split(np.arange(len(var)), 5)
    keys = shard.merge([_keys_of(var[p], ig[p], idx[p], M) for p in parts])
    ref = _reference(var, ig, idx, M)
    g, i = shard.unpack(keys)
    for v in range(M):
        assert (g[v], i[v]) == (ref[v][0], ref[v][1])


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    M = 37
    var, ig, idx = _candidates(2, M)
    mine = np.arange(len(var))[rank::world]  # disjoint shares of the tuple space
    mine_keys = _keys_of(var[mine], ig[mine], idx[mine], M)
    merged = shard.allreduce_max(mine_keys)
    np.save(out_path + f".{rank}.npy", merged)
    # the in-place tensor form the benchmark uses with NCCL on CUDA tensors
    import torch
    t = torch.from_numpy(mine_keys.view(np.int64).copy())
    shard.allreduce_max_device(t)
    np.save(out_path + f".t{rank}.npy", t.numpy().view(np.uint64))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_allreduce_merge(tmp_path):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    out = str(tmp_path / "keys")
    mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
    k0 = np.load(out + ".0.npy")
    k1 = np.load(out + ".1.npy")
    assert np.array_equal(k0, k1)
    for r in (0, 1):
        assert np.array_equal(np.load(out + f".t{r}.npy"), k0)
    M = 37
    var, ig, idx = _candidates(2, M)
    ref = _reference(var, ig, idx, M)
    g, i = shard.unpack(k0)
    for v in range(M):
        assert (g[v], i[v]) == (ref[v][0], ref[v][1])


def test_resumable_scan_skips_finished_shards_and_refuses_other_scans(tmp_path):
    """An interrupted checkpointed scan resumes with the missing shards only,
    and its merge equals the merge of a run without interruption."""
    rng = np.random.default_rng(3)
    n_shards, M = 5, 40
    per_shard = [shard.pack(rng.standard_normal(M).astype(np.float32), rng.integers(0, 2**31, M)) for _ in range(n_shards)]
    want = shard.merge(per_shard)
    calls = []

    def flaky(s):
        calls.append(s)
        if s == 3 and calls.count(3) == 1:
            raise RuntimeError("interrupted")
        return per_shard[s]

    params = {"k": 2, "seed": 1}
    with pytest.raises(RuntimeError):
        shard.run_resumable(flaky, n_shards, str(tmp_path), params)
    assert calls == [0, 1, 2, 3]
    got = shard.run_resumable(flaky, n_shards, str(tmp_path), params)
    assert calls == [0, 1, 2, 3, 3, 4]  # only the unfinished shards ran again
    assert np.array_equal(got, want)
    again = shard.run_resumable(lambda s: pytest.fail("nothing left to scan"), n_shards, str(tmp_path), params)
    assert np.array_equal(again, want)
    with pytest.raises(ValueError):
        shard.run_resumable(flaky, n_shards, str(tmp_path), {"k": 3, "seed": 1})


def _recovery_rank(rank, world, port, ckpt, out_path, fail_rank):
    """One host rank of a sharded scan; ``fail_rank`` dies after its first shard."""
    from datetime import timedelta

    import torch.distributed as dist
    store = dist.TCPStore("127.0.0.1", port, world, is_master=(rank == 0), timeout=timedelta(seconds=30))
    per_shard = _recovery_shards()
    done = []

    def scan(s):
        if rank == fail_rank and done:
            os._exit(0)  # the process ends in the middle of its share, without a word to the others
        done.append(s)
        time.sleep(0.05)
        return per_shard[s]

    # a dead rank is given up on after 2 s; without a failure the wait is long,
    # so a slow but live rank is never taken for dead on a loaded machine
    keys, failed = shard.run_ranks_with_recovery(scan, len(per_shard), ckpt, {"k": 2, "seed": 9}, rank, world, store,
                                                 timeout_s=2.0 if fail_rank >= 0 else 60.0)
    np.save(out_path + f".{rank}.npy", keys)
    with open(out_path + f".{rank}.failed", "w") as f:
        f.write(",".join(map(str, failed)))
    store.set(f"exit/{rank}", "1")
    if rank == 0:  # the store lives in rank 0: keep it up until the live ranks are through
        deadline = time.monotonic() + 20
        while time.monotonic() < deadline and not all(
                store.check([f"exit/{r}"]) for r in range(world) if r != fail_rank):
            time.sleep(0.05)


def _recovery_shards():
    rng = np.random.default_rng(17)
    return [shard.pack(rng.standard_normal(30).astype(np.float32), rng.integers(0, 2**31, 30)) for _ in range(6)]


@pytest.mark.parametrize("fail_rank", [None, 1])
def test_sharded_scan_survives_a_failed_rank(tmp_path, fail_rank):
    """Two host ranks share six shards.  With no failure both return the
    merged keys and name no failed rank.  When rank 1 dies after its first
    shard, rank 0 stops waiting for it after the bounded wait, names it, scans
    its unfinished shards from the shared checkpoint directory, and still
    returns the keys of the whole scan."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    out = str(tmp_path / "res")
    mp.spawn(_recovery_rank, args=(2, port, str(tmp_path / "ckpt"), out, fail_rank if fail_rank is not None else -1),
             nprocs=2, join=True)
    want = shard.merge(_recovery_shards())
    live = [0, 1] if fail_rank is None else [0]
    for r in live:
        assert np.array_equal(np.load(out + f".{r}.npy"), want)
        with open(out + f".{r}.failed") as f:
            assert f.read() == ("" if fail_rank is None else str(fail_rank))
    if fail_rank is not None:
        assert not os.path.exists(out + f".{fail_rank}.npy")
