"""Merging the packed max keys of a scan sharded over processes or GPUs.

The scan's per-variable result is a 64-bit key: the order-preserving bits of
the float IG in the high word and the complement of the tie-break index
(discretisation and partner set) in the low word, so that the element-wise
unsigned maximum over shards is the result of the unsharded scan.  torch has
no unsigned 64-bit all-reduce, so keys travel as int64 with bit 63 flipped,
which maps unsigned order onto signed order.
"""
from __future__ import annotations

import numpy as np

_FLIP = np.uint64(1) << np.uint64(63)


def to_signed_order(keys_u64: np.ndarray) -> np.ndarray:
    """uint64 keys -> int64 values with the same order under signed comparison."""
    return (np.asarray(keys_u64, dtype=np.uint64) ^ _FLIP).view(np.int64)


def from_signed_order(vals_i64: np.ndarray) -> np.ndarray:
    return (np.asarray(vals_i64, dtype=np.int64).view(np.uint64) ^ _FLIP)


def merge(keys_per_shard) -> np.ndarray:
    """Element-wise unsigned maximum of the shards' keys (host)."""
    out = None
    for k in keys_per_shard:
        k = np.asarray(k, dtype=np.uint64)
        out = k.copy() if out is None else np.maximum(out, k)
    return out


def allreduce_max(keys_u64: np.ndarray, group=None) -> np.ndarray:
    """All-reduce MAX of uint64 keys across a torch.distributed group (any backend)."""
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(to_signed_order(keys_u64).copy())
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return from_signed_order(t.numpy())


def allreduce_max_device(keys_t, group=None):
    """In-place all-reduce MAX of uint64 keys held as raw bits in a CUDA int64
    tensor (any backend that reduces CUDA tensors, e.g. NCCL): bit 63 is
    flipped before and after so that signed order is unsigned order."""
    import torch
    import torch.distributed as dist
    flip = torch.iinfo(torch.int64).min  # -2^63: only bit 63 set
    keys_t.bitwise_xor_(flip)
    dist.all_reduce(keys_t, op=dist.ReduceOp.MAX, group=group)
    keys_t.bitwise_xor_(flip)
    return keys_t


# --- key format (mirrors the device packing; used to build test candidates) ---
def pack(ig: np.ndarray, index: np.ndarray) -> np.ndarray:
    """Keys of float32 IG values and uint32 tie-break indices."""
    b = np.asarray(ig, dtype=np.float32).view(np.uint32).astype(np.uint64)
    neg = (b & np.uint64(0x80000000)) != 0
    ordered = np.where(neg, (~b) & np.uint64(0xFFFFFFFF), b | np.uint64(0x80000000))
    return (ordered << np.uint64(32)) | ((~np.asarray(index, dtype=np.uint64)) & np.uint64(0xFFFFFFFF))


def unpack(keys: np.ndarray):
    """(IG float32, index uint32) of keys (keys of 0 give NaN, index 2^32-1)."""
    keys = np.asarray(keys, dtype=np.uint64)
    ordered = keys >> np.uint64(32)
    pos = (ordered & np.uint64(0x80000000)) != 0
    bits = np.where(pos, ordered & np.uint64(0x7FFFFFFF), (~ordered) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    ig = bits.view(np.float32).copy()
    ig[keys == 0] = np.nan
    index = ((~keys) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    return ig, index


# --- checkpointed (resumable) sharded scan ------------------------------------
def _fingerprint(params: dict) -> str:
    import hashlib
    import json
    return hashlib.sha256(json.dumps(params, sort_keys=True).encode()).hexdigest()


def _open_checkpoint(checkpoint_dir: str, n_shards: int, params: dict) -> str:
    """Creates or checks the checkpoint directory of one scan; returns its fingerprint."""
    import json
    import os
    os.makedirs(checkpoint_dir, exist_ok=True)
    fp = _fingerprint(dict(params, n_shards=n_shards))
    meta = os.path.join(checkpoint_dir, "scan.json")
    if not os.path.exists(meta):
        tmp = meta + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump({"fingerprint": fp, "params": params, "n_shards": n_shards}, f)
        os.replace(tmp, meta)
    with open(meta) as f:
        old = json.load(f)
    if old.get("fingerprint") != fp:
        raise ValueError(f"{checkpoint_dir} holds shards of a different scan")
    return fp


def _shard_keys(s: int, scan_shard, checkpoint_dir: str) -> np.ndarray:
    """Keys of shard s: read from its checkpoint file, or scanned and saved
    (temporary name, then rename: a file that exists is complete)."""
    import os
    path = os.path.join(checkpoint_dir, f"shard_{s}.npy")
    if os.path.exists(path):
        return np.load(path)
    k = np.asarray(scan_shard(s), dtype=np.uint64)
    tmp = path + f".tmp{os.getpid()}.npy"
    np.save(tmp, k)
    os.replace(tmp, path)
    return k


def run_resumable(scan_shard, n_shards: int, checkpoint_dir: str, params: dict) -> np.ndarray:
    """Merged keys of a scan split into `n_shards` shards, resumable.

    ``scan_shard(s)`` returns the uint64 keys of shard s (e.g. a closure over
    ``mdfs.max_ig_shard``).  Each finished shard's keys are written to
    ``checkpoint_dir/shard_<s>.npy`` (written to a temporary name, then
    renamed, so a file that exists is complete) next to a fingerprint of
    ``params`` (the scan's arguments and a digest of its data); a rerun with
    the same fingerprint scans only the shards without a file, and one with a
    different fingerprint refuses to mix results.  Because the merge is an
    element-wise maximum, the order in which shards finish does not matter.
    """
    _open_checkpoint(checkpoint_dir, n_shards, params)
    return merge([_shard_keys(s, scan_shard, checkpoint_dir) for s in range(n_shards)])


def run_ranks_with_recovery(scan_shard, n_shards: int, checkpoint_dir: str, params: dict, rank: int, world: int,
                            store, timeout_s: float = 30.0, poll_s: float = 0.05):
    """A scan sharded over ``world`` host processes that survives a failed rank.

    Rank r scans shards r, r + world, ... through the checkpoint directory
    (shared by all ranks), then posts a done flag in the c10d ``store`` (e.g. a
    ``torch.distributed.TCPStore``).  It then waits at most ``timeout_s`` for
    the other ranks' flags.  A rank whose flag has not appeared by then is
    taken as failed, and the waiting rank scans whatever shards have no
    checkpoint file itself.  No step waits on a peer without a bound, and the
    merge needs no collective, so a dead rank cannot hang the others.  Shards
    are deterministic, so a shard scanned twice (a slow rank taken for dead)
    gives the same keys.  Returns (merged keys, sorted ranks taken as failed);
    the keys equal those of the unsharded scan.
    """
    import time
    fp = _open_checkpoint(checkpoint_dir, n_shards, params)
    for s in range(rank, n_shards, world):
        _shard_keys(s, scan_shard, checkpoint_dir)
    flag = f"mdfs/{fp[:16]}/done/"
    store.set(flag + str(rank), "1")
    pending = [r for r in range(world) if r != rank]
    deadline = time.monotonic() + timeout_s
    while pending:
        pending = [r for r in pending if not store.check([flag + str(r)])]
        if not pending or time.monotonic() >= deadline:
            break
        time.sleep(poll_s)
    keys = merge([_shard_keys(s, scan_shard, checkpoint_dir) for s in range(n_shards)])
    return keys, sorted(pending)


def max_ig_resumable(x, y, k: int, divisions: int, discretizations: int, range_: float, pc_xi: float, seed: int,
                     n_shards: int, checkpoint_dir: str):
    """``mdfs.max_ig`` computed shard by shard with the shards' keys kept in
    ``checkpoint_dir`` (see ``run_resumable``); returns (ig, tuples, disc) as
    numpy arrays, identical to the unsharded scan."""
    import hashlib
    from . import mdfs
    xh = x.detach().cpu().numpy() if hasattr(x, "detach") else np.asarray(x)
    yh = y.detach().cpu().numpy() if hasattr(y, "detach") else np.asarray(y)
    digest = hashlib.sha256(np.ascontiguousarray(xh).tobytes() + np.ascontiguousarray(yh).tobytes()).hexdigest()
    params = dict(k=k, divisions=divisions, discretizations=discretizations, range=range_, pc_xi=pc_xi, seed=seed,
                  shape=list(xh.shape), dtype=str(xh.dtype), data=digest)
    keys = run_resumable(lambda s: mdfs.max_ig_shard(x, y, k, divisions, discretizations, range_, pc_xi, seed, s,
                                                     n_shards), n_shards, checkpoint_dir, params)
    return mdfs.decode_keys(keys, k)
