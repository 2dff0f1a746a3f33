"""Argument checks of every C entry point: each bad argument below is refused
with MDFS_EINVAL (-1) and a message naming it, on the host, before any CUDA
call, so these run on a machine without a GPU.  Buffers are tiny host arrays:
the library must not read them once an argument is refused."""
import ctypes
import math

import numpy as np
import pytest

from paper_1811_00631_gb300 import mdfs

EINVAL = -1


@pytest.fixture(scope="module")
def lib():
    from paper_1811_00631_gb300 import build
    build.build()
    return mdfs.load()


_BUF = np.zeros(64, dtype=np.float64)  # stands in for every array argument
P = ctypes.c_void_p(_BUF.ctypes.data)
Y = np.zeros(64, dtype=np.uint8)


def _data(N=10, M=4, dtype=mdfs.MDFS_F32, x=True, y=True):
    return ctypes.byref(mdfs._Data(dtype, _BUF.ctypes.data if x else None, Y.ctypes.data if y else None, N, M))


def max_ig(data=None, k=2, div=1, D=1, r=0.5, xi=0.25, ig=P):
    return lambda lib: lib.mdfs_max_ig(data or _data(), k, div, D, r, xi, 1, ig, P, P, None)


def max_ig_multi(ks=(2, 3), n_k=None, ig_null=None, ig_all_null=False, k_null=False, div=1, data=None):
    n = len(ks) if n_k is None else n_k
    karr = (ctypes.c_int * max(len(ks), 1))(*ks)
    ptrs = (ctypes.c_void_p * max(len(ks), 1))(*[None if j == ig_null else P.value for j in range(len(ks))])
    return lambda lib: lib.mdfs_max_ig_multi(data or _data(), n, None if k_null else karr, div, 1, 0.5, 0.25, 1,
                                             None if ig_all_null else ptrs, None, None, None)


CASES = [
    ("max_ig_multi: n_k = 0", max_ig_multi(n_k=0), "n_k = 0"),
    ("max_ig_multi: n_k = 6", max_ig_multi(ks=(1, 2, 3, 4, 5, 1)), "n_k = 6"),
    ("max_ig_multi: ks NULL", max_ig_multi(k_null=True), "ks / ig NULL"),
    ("max_ig_multi: ig NULL", max_ig_multi(ig_all_null=True), "ks / ig NULL"),
    ("max_ig_multi: k = 0", max_ig_multi(ks=(2, 0)), "ks[1] = 0"),
    ("max_ig_multi: k = 6", max_ig_multi(ks=(6,)), "ks[0] = 6"),
    ("max_ig_multi: k twice", max_ig_multi(ks=(3, 2, 3)), "k = 3 appears twice"),
    ("max_ig_multi: ig[1] NULL", max_ig_multi(ks=(1, 3), ig_null=1), "ig[1] is NULL"),
    ("max_ig_multi: k = 4 keys overflow", max_ig_multi(ks=(2, 4), div=2, data=_data(M=2000)), "2^32"),
    ("max_ig: k = 0", max_ig(k=0), "k = 0"),
    ("max_ig: k = 6", max_ig(k=6), "k = 6"),
    ("max_ig: M < k", max_ig(data=_data(M=2), k=3), "smaller than k"),
    ("max_ig: divisions = 0", max_ig(div=0), "divisions"),
    ("max_ig: divisions = 4", max_ig(div=4), "divisions"),
    ("max_ig: N < classes", max_ig(data=_data(N=3), div=3), "smaller than the number of classes"),
    ("max_ig: no discretisation", max_ig(D=0), "discretizations"),
    ("max_ig: 1025 discretisations", max_ig(D=1025), "discretizations"),
    ("max_ig: range < 0", max_ig(r=-0.1), "range"),
    ("max_ig: range > 1", max_ig(r=1.5), "range"),
    ("max_ig: range NaN", max_ig(r=math.nan), "range"),
    ("max_ig: pc_xi = 0", max_ig(xi=0.0), "pc_xi"),
    ("max_ig: pc_xi = 1", max_ig(xi=1.0), "pc_xi"),
    ("max_ig: ig NULL", max_ig(ig=None), "ig is NULL"),
    ("max_ig: bad dtype", max_ig(data=_data(dtype=7)), "dtype"),
    ("max_ig: x NULL", max_ig(data=_data(x=False)), "x is NULL"),
    ("max_ig: y NULL", max_ig(data=_data(y=False)), "y is NULL"),
    ("max_ig: N = 1", max_ig(data=_data(N=1)), "N = 1"),
    ("max_ig: N above the limit", max_ig(data=_data(N=32769)), "N = 32769"),
    ("max_ig: M = 0", max_ig(data=_data(M=0)), "M = 0"),
    ("max_ig: M = 65536", max_ig(data=_data(M=65536)), "M = 65536"),
    ("max_ig: k = 5, three classes, keys overflow", max_ig(data=_data(M=200), k=5, div=2, D=67), "2^32"),
    ("max_ig: k = 3 keys overflow", max_ig(data=_data(M=65535), k=3, D=2), "2^32"),
    ("max_ig: k = 4 keys overflow", max_ig(data=_data(M=2000), k=4, D=1), "2^32"),
    ("discretize: divisions = 0",
     lambda lib: lib.mdfs_discretize(_data(), 0, 1, 0.5, 1, P, None), "divisions"),
    ("discretize: no discretisation",
     lambda lib: lib.mdfs_discretize(_data(), 1, 0, 0.5, 1, P, None), "discretizations"),
    ("discretize: range > 1",
     lambda lib: lib.mdfs_discretize(_data(), 1, 1, 2.0, 1, P, None), "range"),
    ("discretize: codes NULL",
     lambda lib: lib.mdfs_discretize(_data(), 1, 1, 0.5, 1, None, None), "codes is NULL"),
    ("batch: no job",
     lambda lib: lib.mdfs_max_ig_batch(_data(), 0, P, P, 2, 1, 1, 0.5, 0.25, 1, P, P, P, None), "n_jobs"),
    ("shard: index below 0",
     lambda lib: lib.mdfs_max_ig_shard(_data(), 2, 1, 1, 0.5, 0.25, 1, -1, 2, P, None), "shard"),
    ("shard: index past the count",
     lambda lib: lib.mdfs_max_ig_shard(_data(), 2, 1, 1, 0.5, 0.25, 1, 2, 2, P, None), "shard"),
    ("shard: keys NULL",
     lambda lib: lib.mdfs_max_ig_shard(_data(), 2, 1, 1, 0.5, 0.25, 1, 0, 1, None, None), "keys is NULL"),
    ("keys_decode: keys NULL", lambda lib: lib.mdfs_keys_decode(None, 4, 2, P, P, P, None), "NULL"),
    ("keys_decode: k = 6", lambda lib: lib.mdfs_keys_decode(P, 4, 6, P, P, P, None), "out of range"),
    ("keys_decode: M = 0", lambda lib: lib.mdfs_keys_decode(P, 0, 2, P, P, P, None), "out of range"),
    ("ig_lim: ig NULL", lambda lib: lib.mdfs_ig_lim(None, 4, 1, 1, 1, None, 0.05, P, P, P, None), "NULL"),
    ("ig_lim: M = 0", lambda lib: lib.mdfs_ig_lim(P, 0, 1, 1, 1, None, 0.05, P, P, P, None), "M = 0"),
    ("ig_lim: k = 0", lambda lib: lib.mdfs_ig_lim(P, 4, 0, 1, 1, None, 0.05, P, P, P, None), "k = 0"),
    ("ig_lim: divisions = 0", lambda lib: lib.mdfs_ig_lim(P, 4, 1, 0, 1, None, 0.05, P, P, P, None), "divisions"),
    ("ig_lim: alpha = 0", lambda lib: lib.mdfs_ig_lim(P, 4, 1, 1, 1, None, 0.0, P, P, P, None), "alpha"),
    ("ig_lim: alpha = 1", lambda lib: lib.mdfs_ig_lim(P, 4, 1, 1, 1, None, 1.0, P, P, P, None), "alpha"),
    ("contrast: negative count", lambda lib: lib.mdfs_contrast(_data(), -1, 1, P, P, None), "n_contrast"),
    ("contrast: too many variables", lambda lib: lib.mdfs_contrast(_data(), 65535, 1, P, P, None), "n_contrast"),
    ("contrast: x_ext NULL", lambda lib: lib.mdfs_contrast(_data(), 3, 1, None, P, None), "x_ext is NULL"),
    ("p_adjust: p NULL", lambda lib: lib.mdfs_p_adjust(None, 4, 2, P, None), "NULL"),
    ("p_adjust: m = 0", lambda lib: lib.mdfs_p_adjust(P, 0, 2, P, None), "m = 0"),
    ("p_adjust: unknown method", lambda lib: lib.mdfs_p_adjust(P, 4, 9, P, None), "unknown method"),
    ("select: no contrast",
     lambda lib: lib.mdfs_select(_data(), 0, 2, 1, 1, 0.5, 0.25, 1, 2, 0.05, P, P, P, P, P, P, P, P, P, None),
     "n_contrast"),
    ("select: level = 0",
     lambda lib: lib.mdfs_select(_data(), 4, 2, 1, 1, 0.5, 0.25, 1, 2, 0.0, P, P, P, P, P, P, P, P, P, None),
     "level"),
    ("select: unknown method",
     lambda lib: lib.mdfs_select(_data(), 4, 2, 1, 1, 0.5, 0.25, 1, 9, 0.05, P, P, P, P, P, P, P, P, P, None),
     "p_adjust_method"),
    ("select: outputs NULL",
     lambda lib: lib.mdfs_select(_data(), 4, 2, 1, 1, 0.5, 0.25, 1, 2, 0.05, None, P, P, P, P, P, P, P, P, None),
     "NULL"),
    ("interesting: threshold not finite",
     lambda lib: lib.mdfs_interesting_tuples(_data(), 2, 1, 1, 0.5, 0.25, 1, math.inf, 16, P, P, P, P, P, None),
     "threshold"),
    ("interesting: capacity 0",
     lambda lib: lib.mdfs_interesting_tuples(_data(), 2, 1, 1, 0.5, 0.25, 1, 1.0, 0, P, P, P, P, P, None),
     "capacity"),
    ("interesting: outputs NULL",
     lambda lib: lib.mdfs_interesting_tuples(_data(), 2, 1, 1, 0.5, 0.25, 1, 1.0, 16, None, P, P, P, P, None),
     "NULL"),
    ("noalloc: k = 3",
     lambda lib: lib.mdfs_max_ig_noalloc(_data(), 3, 1, 1, 0.5, 0.25, 1, P, P, P, None), "k must be 1 or 2"),
    ("noalloc: divisions = 4",
     lambda lib: lib.mdfs_max_ig_noalloc(_data(), 2, 4, 1, 0.5, 0.25, 1, P, P, P, None), "divisions"),
    ("testing counts: k = 1",
     lambda lib: lib.mdfs_testing_counts(_data(), 1, 1, 1, 0.5, 1, P, None), "k = 1"),
    ("testing counts: divisions = 4",
     lambda lib: lib.mdfs_testing_counts(_data(), 2, 4, 1, 0.5, 1, P, None), "divisions"),
    ("testing counts: counts NULL",
     lambda lib: lib.mdfs_testing_counts(_data(), 2, 1, 1, 0.5, 1, None, None), "counts is NULL"),
    ("testing wait fault: stage below -1", lambda lib: lib.mdfs_testing_k3_wait_fault(-2, 0), "withhold_kb"),
    ("testing wait fault: limit above 10 s",
     lambda lib: lib.mdfs_testing_k3_wait_fault(0, 20_000_000_000), "wait_ns"),
    ("testing wait fault: negative limit", lambda lib: lib.mdfs_testing_k3_wait_fault(0, -1), "wait_ns"),
]


@pytest.mark.parametrize("name,call,words", CASES, ids=[c[0] for c in CASES])
def test_bad_argument_is_refused_on_the_host(lib, name, call, words):
    rc = call(lib)
    msg = lib.mdfs_last_error().decode()
    assert rc == EINVAL, f"{name}: rc {rc}, message {msg!r}"
    assert words in msg, f"{name}: message {msg!r}"
    assert lib.mdfs_last_launch_count() == 0
