"""Seeded synthetic inputs for the MDFS information-gain scan.

This module only draws random numbers (numpy PCG64): it holds none of the
method's arithmetic, and both the CUDA path and the CPU oracle are fed from it.
Every array is variable-major: ``x`` has shape (M, N), i.e. ``x[v, s]`` is
sample ``s`` of variable ``v`` (the layout the C ABI takes), and ``y`` is a
uint8 vector of N decisions in {0, 1}.

Workloads (shapes and structure follow the Madelon description in section
"Madelon example" of arXiv 1811.00631, which is not available here):

* ``xor_small``       N=200, M=50, y = [sign x0 * sign x1 > 0] XOR 10% flips.
* ``madelon_like``    N=2000, M=500: 5 base variables whose sign pattern sets
  y by parity, 15 random linear combinations of them plus small noise, 480
  pure N(0,1) variables, columns shuffled.
* ``xor_pairs``       N=1000, M=20000: 100 XOR pairs with 10% label noise, the
  rest N(0,1).
* ``bootstrap_jobs``  resampling indices and y permutations for batched jobs.
* ``serving_mix``     a Poisson stream of mixed jobs.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Dataset:
    x: np.ndarray          # (M, N) float32 or int8, variable-major
    y: np.ndarray          # (N,) uint8 in {0, 1}
    informative: np.ndarray  # indices of variables built to carry signal
    info: dict


def xor_small(N: int = 200, M: int = 50, flip: float = 0.1, seed: int = 1) -> Dataset:
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = ((np.sign(x[0]) * np.sign(x[1])) > 0).astype(np.uint8)
    flips = rng.random(N) < flip
    y ^= flips.astype(np.uint8)
    return Dataset(x=x, y=y, informative=np.array([0, 1]), info=dict(kind="xor_small", seed=seed))


def madelon_like(N: int = 2000, M: int = 500, n_base: int = 5, n_comb: int = 15, seed: int = 2) -> Dataset:
    """Parity-structured data with Madelon's shapes (N=2000, M=500)."""
    assert M >= n_base + n_comb
    rng = np.random.Generator(np.random.PCG64(seed))
    vert = rng.choice(np.array([-1.0, 1.0]), size=(N, n_base))
    base = vert + rng.standard_normal((N, n_base))
    y = (np.sum(vert > 0, axis=1) % 2).astype(np.uint8)
    mix = rng.standard_normal((n_base, n_comb))
    comb = base @ mix + 0.1 * rng.standard_normal((N, n_comb))
    noise = rng.standard_normal((N, M - n_base - n_comb))
    cols = np.concatenate([base, comb, noise], axis=1)  # (N, M)
    perm = rng.permutation(M)  # column j of the output is original column perm[j]
    x = np.ascontiguousarray(cols[:, perm].T).astype(np.float32)
    inv = np.argsort(perm)
    return Dataset(x=x, y=y, informative=np.sort(inv[: n_base + n_comb]),
                   info=dict(kind="madelon_like", seed=seed, base=np.sort(inv[:n_base]),
                             comb=np.sort(inv[n_base:n_base + n_comb]), perm=perm))


def xor_pairs(N: int = 1000, M: int = 20000, n_pairs: int = 100, flip: float = 0.1, seed: int = 4) -> Dataset:
    """Each of n_pairs variable pairs encodes y by the parity of its two signs (10% flips)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.standard_normal((M, N)).astype(np.float32)
    y = (rng.random(N) < 0.5).astype(np.uint8)
    members = rng.permutation(M)[: 2 * n_pairs].reshape(n_pairs, 2)
    for a, b in members:
        agree = (y == 1) ^ (rng.random(N) < flip)  # sign(x_a) * sign(x_b) > 0  <=>  agree
        sa = np.sign(x[a])
        sa[sa == 0] = 1.0
        x[b] = (np.abs(x[b]) * np.where(agree, sa, -sa)).astype(np.float32)
    return Dataset(x=x, y=y, informative=np.sort(members.ravel()),
                   info=dict(kind="xor_pairs", seed=seed, pairs=members))


def to_int8(x: np.ndarray, scale: float = 24.0) -> np.ndarray:
    """Quantise a float array to int8 (ties and empty classes become possible)."""
    return np.clip(np.rint(x * scale), -127, 127).astype(np.int8)


def bootstrap_jobs(N: int, n_folds: int = 16, n_perms: int = 4, seed: int = 5):
    """Per job: a resampling index vector (N draws with replacement) and a y permutation.

    Job j = fold * n_perms + p uses ``idx[fold]`` and ``yperm[p]``; permutation 0
    is the identity (the un-permuted decision).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = rng.integers(0, N, size=(n_folds, N)).astype(np.int32)
    yperm = np.stack([np.arange(N)] + [rng.permutation(N) for _ in range(n_perms - 1)]).astype(np.int32)
    return idx, yperm


def serving_mix(n_jobs: int = 512, seed: int = 7, rate_hz: float = 50.0, n_range=(100, 5000),
                m_range=(100, 5000), max_work: float = 2e11):
    """Job descriptors for a Poisson request stream of mixed MDFS scans."""
    rng = np.random.Generator(np.random.PCG64(seed))
    arrivals = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_jobs))
    jobs = []
    for j in range(n_jobs):
        k = int(rng.integers(1, 4))
        N = int(rng.integers(n_range[0], n_range[1] + 1))
        M = int(np.exp(rng.uniform(np.log(m_range[0]), np.log(m_range[1]))))
        div = int(rng.integers(1, 4))
        D = int(rng.integers(5, 31))
        dtype = "i8" if rng.random() < 0.5 else "f32"
        # keep one job within the work cap: C(M, k) * D * N sample visits
        while M > k + 1 and _comb(M, k) * D * N > max_work:
            M = int(M * 0.9)
        jobs.append(dict(job=j, arrival=float(arrivals[j]), k=k, N=N, M=M, divisions=div,
                         discretizations=D, dtype=dtype, seed=int(rng.integers(1, 2**31)),
                         data_seed=int(rng.integers(1, 2**31))))
    return jobs


def serving_data(job: dict):
    rng = np.random.Generator(np.random.PCG64(job["data_seed"]))
    N, M = job["N"], job["M"]
    x = rng.standard_normal((M, N)).astype(np.float32)
    # plant one XOR pair so that every job carries some signal
    y = ((np.sign(x[0]) * np.sign(x[min(1, M - 1)])) > 0).astype(np.uint8)
    y ^= (rng.random(N) < 0.1).astype(np.uint8)
    if y.min() == y.max():
        y[0] ^= 1
    if job["dtype"] == "i8":
        return to_int8(x), y
    return x, y


def _comb(n: int, k: int) -> float:
    from math import comb
    return float(comb(n, k))
