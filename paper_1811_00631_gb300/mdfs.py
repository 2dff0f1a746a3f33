"""Thin ctypes binding of the MDFS C ABI (``include/mdfs.h``).

Argument marshalling only: every step of the scan runs in the CUDA library
``libmdfs_gb300.so``.  Inputs may be CUDA tensors (device pointers are passed
through, outputs are allocated on the same device and the current torch stream
is used) or host arrays (numpy arrays or CPU tensors; outputs are numpy arrays
and the library copies inputs to the device inside the call).  There is no CPU
fallback: if the library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmdfs_gb300.so")

MDFS_F32 = 0
MDFS_I8 = 1

_ERRORS = {
    -1: "MDFS_EINVAL",
    -2: "MDFS_EDEGENERATE",
    -3: "MDFS_ENONFINITE",
    -4: "MDFS_ENOMEM",
    -5: "MDFS_ECUDA",
    -6: "MDFS_ETIMEOUT",
    -7: "MDFS_ETRUNCATED",
}

EXPORTED = ("mdfs_discretize", "mdfs_max_ig", "mdfs_max_ig_multi", "mdfs_ig_lim", "mdfs_last_error", "mdfs_release",
            "mdfs_abi_version", "mdfs_last_launch_count", "mdfs_profile", "mdfs_profile_report",
            "mdfs_max_ig_noalloc", "mdfs_max_ig_batch", "mdfs_max_ig_shard", "mdfs_keys_decode",
            "mdfs_contrast", "mdfs_p_adjust", "mdfs_select", "mdfs_interesting_tuples",
            "mdfs_release_stream", "mdfs_bench_mma_f8", "mdfs_bench_smem_lookup", "mdfs_testing_counts", "mdfs_testing_k3_wait_fault",
            "mdfs_testing_exact", "mdfs_testing_k3_claim_order")

# p-value adjustment methods (MDFS_ADJUST_* of include/mdfs.h)
P_ADJUST = {"none": 0, "bonferroni": 1, "holm": 2, "hochberg": 3, "BH": 4, "BY": 5}


class MdfsError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{_ERRORS.get(code, code)}: {message}")
        self.code = code


class _Data(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("N", ctypes.c_int), ("M", ctypes.c_int)]


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Loads the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"MDFS CUDA library not built ({path} missing); run python -m paper_1811_00631_gb300.build")
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        lib.mdfs_discretize.argtypes = [ctypes.POINTER(_Data), ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_uint64, P, P]
        lib.mdfs_discretize.restype = ctypes.c_int
        lib.mdfs_max_ig.argtypes = [ctypes.POINTER(_Data), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_uint64, P, P, P, P]
        lib.mdfs_max_ig.restype = ctypes.c_int
        lib.mdfs_max_ig_multi.argtypes = [ctypes.POINTER(_Data), ctypes.c_int, P, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_uint64, P, P, P, P]
        lib.mdfs_max_ig_multi.restype = ctypes.c_int
        lib.mdfs_max_ig_noalloc.argtypes = [ctypes.POINTER(_Data), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_uint64, P, P, P, P]
        lib.mdfs_max_ig_noalloc.restype = ctypes.c_int
        lib.mdfs_max_ig_batch.argtypes = [ctypes.POINTER(_Data), ctypes.c_int, P, P, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_uint64, P, P, P, P]
        lib.mdfs_max_ig_batch.restype = ctypes.c_int
        lib.mdfs_max_ig_shard.argtypes = [ctypes.POINTER(_Data), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                          P, P]
        lib.mdfs_max_ig_shard.restype = ctypes.c_int
        lib.mdfs_keys_decode.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, P, P]
        lib.mdfs_keys_decode.restype = ctypes.c_int
        lib.mdfs_ig_lim.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P,
                                    ctypes.c_double, P, P, P, P]
        lib.mdfs_ig_lim.restype = ctypes.c_int
        lib.mdfs_contrast.argtypes = [ctypes.POINTER(_Data), ctypes.c_int, ctypes.c_uint64, P, P, P]
        lib.mdfs_contrast.restype = ctypes.c_int
        lib.mdfs_p_adjust.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P]
        lib.mdfs_p_adjust.restype = ctypes.c_int
        lib.mdfs_select.argtypes = [ctypes.POINTER(_Data), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_uint64, ctypes.c_int, ctypes.c_double,
                                    P, P, P, P, P, P, P, P, P, P]
        lib.mdfs_select.restype = ctypes.c_int
        lib.mdfs_interesting_tuples.argtypes = [ctypes.POINTER(_Data), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_double, ctypes.c_double, ctypes.c_uint64, ctypes.c_double,
                                                ctypes.c_int, P, P, P, P, P, P]
        lib.mdfs_interesting_tuples.restype = ctypes.c_int
        lib.mdfs_last_error.argtypes = []
        lib.mdfs_last_error.restype = ctypes.c_char_p
        lib.mdfs_release.argtypes = []
        lib.mdfs_release.restype = ctypes.c_int
        lib.mdfs_release_stream.argtypes = [P]
        lib.mdfs_release_stream.restype = ctypes.c_int
        lib.mdfs_abi_version.argtypes = []
        lib.mdfs_abi_version.restype = ctypes.c_int
        lib.mdfs_last_launch_count.argtypes = []
        lib.mdfs_last_launch_count.restype = ctypes.c_int
        lib.mdfs_profile.argtypes = [ctypes.c_int]
        lib.mdfs_profile.restype = ctypes.c_int
        lib.mdfs_profile_report.argtypes = [ctypes.c_char_p, ctypes.c_int]
        lib.mdfs_profile_report.restype = ctypes.c_int
        # hardware microbenchmarks (include/mdfs_bench.h)
        lib.mdfs_bench_mma_f8.argtypes = [ctypes.c_int, P, P]
        lib.mdfs_bench_mma_f8.restype = ctypes.c_int
        lib.mdfs_bench_smem_lookup.argtypes = [ctypes.c_int, ctypes.c_int, P, P]
        lib.mdfs_bench_smem_lookup.restype = ctypes.c_int
        # test-only entry points (include/mdfs_testing.h)
        lib.mdfs_testing_counts.argtypes = [ctypes.POINTER(_Data), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_uint64, P, P]
        lib.mdfs_testing_counts.restype = ctypes.c_int
        lib.mdfs_testing_k3_wait_fault.argtypes = [ctypes.c_int, ctypes.c_longlong]
        lib.mdfs_testing_k3_wait_fault.restype = ctypes.c_int
        lib.mdfs_testing_k3_claim_order.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_int]
        lib.mdfs_testing_k3_claim_order.restype = ctypes.c_int
        lib.mdfs_testing_exact.argtypes = []
        lib.mdfs_testing_exact.restype = ctypes.c_int
        _lib = lib
        return lib


def _check(rc: int):
    if rc != 0:
        msg = load().mdfs_last_error().decode(errors="replace")
        raise MdfsError(rc, msg)


def _is_cuda(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


def _stream_of(a):
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream(a.device).cuda_stream)


def _host(a, dtype):
    if hasattr(a, "detach"):  # CPU torch tensor
        a = a.detach().numpy()
    return np.ascontiguousarray(a, dtype=dtype)


def _x_info(x):
    """(pointer, dtype code, keep-alive) of the variable-major (M, N) array."""
    if _is_cuda(x):
        import torch
        x = x.contiguous()
        if x.dtype == torch.float32:
            return x.data_ptr(), MDFS_F32, x
        if x.dtype == torch.int8:
            return x.data_ptr(), MDFS_I8, x
        raise TypeError("x must be float32 or int8")
    arr = x.detach().numpy() if hasattr(x, "detach") else np.asarray(x)
    if arr.dtype == np.int8:
        arr = np.ascontiguousarray(arr)
        return arr.ctypes.data, MDFS_I8, arr
    arr = np.ascontiguousarray(arr, dtype=np.float32)
    return arr.ctypes.data, MDFS_F32, arr


def _data(x, y):
    xp, dt, xk = _x_info(x)
    M, N = int(x.shape[0]), int(x.shape[1])
    yk = None
    yp = None
    if y is not None:
        if _is_cuda(y):
            import torch
            yk = y.contiguous().to(torch.uint8)
            yp = yk.data_ptr()
        else:
            yk = _host(y, np.uint8)
            yp = yk.ctypes.data
        if int(y.shape[0]) != N:
            raise ValueError("y must have N entries")
    return _Data(dt, xp, yp, N, M), (xk, yk)


def _check_out(arrs, shapes, dtypes, like):
    """Preallocated outputs must match the kind of ``like`` (CUDA tensors on its
    device, else numpy arrays), be C-contiguous and have the exact dtype and
    shape the library writes; anything else is refused before the call, since
    the library trusts the sizes it is given."""
    for a, shape, dt in zip(arrs, shapes, dtypes):
        if _is_cuda(like):
            import torch
            tdt = {np.float32: torch.float32, np.int32: torch.int32}[dt]
            ok = (_is_cuda(a) and a.device == like.device and a.dtype == tdt and a.is_contiguous()
                  and tuple(a.shape) == shape)
        else:
            ok = (isinstance(a, np.ndarray) and a.dtype == dt and a.flags.c_contiguous and a.shape == shape
                  and a.flags.writeable)
        if not ok:
            raise ValueError(f"out: expected a contiguous {np.dtype(dt).name} array of shape {shape} "
                             f"{'on ' + str(like.device) if _is_cuda(like) else 'in host memory'}")


def discretize(x, divisions: int = 1, discretizations: int = 1, range_: float = 0.0, seed: int = 0):
    """Codes u8[D][M][N] (section "Algorithm and implementation" of arXiv 1811.00631)."""
    lib = load()
    data, keep = _data(x, None)
    D, M, N = discretizations, data.M, data.N
    if _is_cuda(x):
        import torch
        out = torch.empty((D, M, N), dtype=torch.uint8, device=x.device)
        rc = lib.mdfs_discretize(ctypes.byref(data), divisions, D, float(range_), int(seed) & (2**64 - 1),
                                 ctypes.c_void_p(out.data_ptr()), _stream_of(x))
    else:
        out = np.empty((D, M, N), dtype=np.uint8)
        rc = lib.mdfs_discretize(ctypes.byref(data), divisions, D, float(range_), int(seed) & (2**64 - 1),
                                 ctypes.c_void_p(out.ctypes.data), None)
    _check(rc)
    del keep
    return out


def max_ig(x, y, k: int = 2, divisions: int = 1, discretizations: int = 1, range_: float = 0.0,
           pc_xi: float = 0.25, seed: int = 0, out=None):
    """IG^k_max per variable (Eq. 1 of arXiv 1811.00631) with its argmax tuple and discretisation.

    Returns (ig f32[M], tuples i32[M, k-1], disc i32[M]) on the device of x
    (torch tensors) or on the host (numpy arrays).  ``out`` may pass
    preallocated (ig, tuples, disc) of the matching kind.
    """
    lib = load()
    data, keep = _data(x, y)
    M = data.M
    kk = max(k - 1, 1)
    if _is_cuda(x):
        import torch
        if out is None:
            ig = torch.empty(M, dtype=torch.float32, device=x.device)
            tu = torch.empty((M, kk), dtype=torch.int32, device=x.device)
            di = torch.empty(M, dtype=torch.int32, device=x.device)
        else:
            ig, tu, di = out
            _check_out(out, ((M,), (M, kk), (M,)), (np.float32, np.int32, np.int32), x)
        ptrs = (ig.data_ptr(), tu.data_ptr(), di.data_ptr())
        stream = _stream_of(x)
    else:
        if out is None:
            ig = np.empty(M, dtype=np.float32)
            tu = np.empty((M, kk), dtype=np.int32)
            di = np.empty(M, dtype=np.int32)
        else:
            ig, tu, di = out
            _check_out(out, ((M,), (M, kk), (M,)), (np.float32, np.int32, np.int32), x)
        ptrs = (ig.ctypes.data, tu.ctypes.data, di.ctypes.data)
        stream = None
    rc = lib.mdfs_max_ig(ctypes.byref(data), k, divisions, discretizations, float(range_), float(pc_xi),
                         int(seed) & (2**64 - 1), ctypes.c_void_p(ptrs[0]),
                         ctypes.c_void_p(ptrs[1]) if k > 1 else None, ctypes.c_void_p(ptrs[2]), stream)
    _check(rc)
    del keep
    return ig, tu[:, : k - 1], di


def max_ig_multi(x, y, ks=(2, 3), divisions: int = 1, discretizations: int = 1, range_: float = 0.0,
                 pc_xi: float = 0.25, seed: int = 0, out=None):
    """mdfs_max_ig_multi: IG^k_max for every k in ``ks`` (distinct, 1..5) of the same
    data and discretisations in one call; entry k equals max_ig with that k.

    Returns {k: (ig f32[M], tuples i32[M, k-1], disc i32[M])} on the device of x
    (torch tensors) or on the host (numpy arrays).  ``out`` may pass a dict of
    preallocated triples of the matching kind.
    """
    lib = load()
    data, keep = _data(x, y)
    M = data.M
    ks = [int(k) for k in ks]
    res, ptrs = {}, []
    for k in ks:
        kk = max(k - 1, 1)
        if out is not None and k in out:
            _check_out(out[k], ((M,), (M, kk), (M,)), (np.float32, np.int32, np.int32), x)
            trip = out[k]
        elif _is_cuda(x):
            import torch
            trip = (torch.empty(M, dtype=torch.float32, device=x.device),
                    torch.empty((M, kk), dtype=torch.int32, device=x.device),
                    torch.empty(M, dtype=torch.int32, device=x.device))
        else:
            trip = (np.empty(M, dtype=np.float32), np.empty((M, kk), dtype=np.int32), np.empty(M, dtype=np.int32))
        res[k] = trip
        ptrs.append(tuple(t.data_ptr() if _is_cuda(x) else t.ctypes.data for t in trip))
    n = len(ks)
    karr = (ctypes.c_int * n)(*ks)
    igp = (ctypes.c_void_p * n)(*[p[0] for p in ptrs])
    tup = (ctypes.c_void_p * n)(*[p[1] if k > 1 else None for p, k in zip(ptrs, ks)])
    dip = (ctypes.c_void_p * n)(*[p[2] for p in ptrs])
    rc = lib.mdfs_max_ig_multi(ctypes.byref(data), n, karr, divisions, discretizations, float(range_), float(pc_xi),
                               int(seed) & (2**64 - 1), igp, tup, dip, _stream_of(x) if _is_cuda(x) else None)
    _check(rc)
    del keep
    return {k: (ig, tu[:, : k - 1], di) for k, (ig, tu, di) in res.items()}


def max_ig_batch(x, y, sample_idx=None, y_perm=None, n_jobs=None, k: int = 2, divisions: int = 1,
                 discretizations: int = 1, range_: float = 0.0, pc_xi: float = 0.25, seed: int = 0):
    """mdfs_max_ig_batch: independent scans of resampled / label-permuted copies of (x, y).

    Job j scans x[:, idx_j] with labels y[perm_j[idx_j]] (idx_j = sample_idx[j],
    perm_j = y_perm[j]; None = identity).  Returns (ig [J, M], tuples [J, M, k-1],
    disc [J, M]) on the device of x (CUDA tensors) or as numpy arrays.
    """
    lib = load()
    data, keep = _data(x, y)
    M, N = data.M, data.N
    J = n_jobs if n_jobs is not None else (len(sample_idx) if sample_idx is not None else len(y_perm))
    kk = max(k - 1, 1)

    def index_ptr(a):
        # the library reads J x N indices from each map
        if a is None:
            return None, None
        if _is_cuda(a):
            import torch
            t = a.contiguous().to(torch.int32)
            if t.numel() < J * N:
                raise ValueError(f"index map holds {t.numel()} entries; {J} jobs x N = {N} need {J * N}")
            return ctypes.c_void_p(t.data_ptr()), t
        h = _host(a, np.int32)
        if h.size < J * N:
            raise ValueError(f"index map holds {h.size} entries; {J} jobs x N = {N} need {J * N}")
        return ctypes.c_void_p(h.ctypes.data), h
    ip, ik = index_ptr(sample_idx)
    pp, pk = index_ptr(y_perm)
    if _is_cuda(x):
        import torch
        ig = torch.empty((J, M), dtype=torch.float32, device=x.device)
        tu = torch.empty((J, M, kk), dtype=torch.int32, device=x.device)
        di = torch.empty((J, M), dtype=torch.int32, device=x.device)
        ptrs = (ig.data_ptr(), tu.data_ptr(), di.data_ptr())
        stream = _stream_of(x)
    else:
        ig = np.empty((J, M), np.float32)
        tu = np.empty((J, M, kk), np.int32)
        di = np.empty((J, M), np.int32)
        ptrs = (ig.ctypes.data, tu.ctypes.data, di.ctypes.data)
        stream = None
    rc = lib.mdfs_max_ig_batch(ctypes.byref(data), J, ip, pp, k, divisions, discretizations, float(range_),
                               float(pc_xi), int(seed) & (2**64 - 1), ctypes.c_void_p(ptrs[0]),
                               ctypes.c_void_p(ptrs[1]) if k > 1 else None, ctypes.c_void_p(ptrs[2]), stream)
    _check(rc)
    del keep, ik, pk
    return ig, tu[:, :, : k - 1], di


def max_ig_shard(x, y, k: int = 2, divisions: int = 1, discretizations: int = 1, range_: float = 0.0,
                 pc_xi: float = 0.25, seed: int = 0, shard: int = 0, n_shards: int = 1, keys_out=None):
    """Packed max keys [M] of shard `shard` of `n_shards` of the scan: a uint64
    numpy array, or, with keys_out (a CUDA int64 tensor of M entries on the
    device of x), the raw uint64 bits written into that tensor on the
    current stream."""
    lib = load()
    data, keep = _data(x, y)
    stream = _stream_of(x) if _is_cuda(x) else None
    if keys_out is not None:
        import torch
        if not (_is_cuda(keys_out) and keys_out.dtype == torch.int64 and keys_out.is_contiguous()
                and tuple(keys_out.shape) == (data.M,)):
            raise ValueError(f"keys_out: expected a contiguous CUDA int64 tensor of shape ({data.M},)")
        ptr = keys_out.data_ptr()
        keys = keys_out
    else:
        keys = np.zeros(data.M, dtype=np.uint64)
        ptr = keys.ctypes.data
    rc = lib.mdfs_max_ig_shard(ctypes.byref(data), k, divisions, discretizations, float(range_), float(pc_xi),
                               int(seed) & (2**64 - 1), shard, n_shards, ctypes.c_void_p(ptr), stream)
    _check(rc)
    del keep
    return keys


def decode_keys(keys, k: int, out=None):
    """(ig, tuples, disc) of merged keys, as max_ig returns them: numpy arrays
    for numpy keys; for keys in a CUDA int64 tensor (raw uint64 bits), CUDA
    tensors on its device (or the preallocated `out` of max_ig's kind)."""
    lib = load()
    kk = max(k - 1, 1)
    if _is_cuda(keys):
        import torch
        M = int(keys.shape[0])
        if out is None:
            ig = torch.empty(M, dtype=torch.float32, device=keys.device)
            tu = torch.empty((M, kk), dtype=torch.int32, device=keys.device)
            di = torch.empty(M, dtype=torch.int32, device=keys.device)
        else:
            ig, tu, di = out
            _check_out(out, ((M,), (M, kk), (M,)), (np.float32, np.int32, np.int32), keys)
        rc = lib.mdfs_keys_decode(ctypes.c_void_p(keys.data_ptr()), M, k, ctypes.c_void_p(ig.data_ptr()),
                                  ctypes.c_void_p(tu.data_ptr()) if k > 1 else None, ctypes.c_void_p(di.data_ptr()),
                                  _stream_of(keys))
        _check(rc)
        return ig, tu[:, : k - 1], di
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    M = len(keys)
    ig = np.empty(M, np.float32)
    tu = np.empty((M, kk), np.int32)
    di = np.empty(M, np.int32)
    rc = lib.mdfs_keys_decode(ctypes.c_void_p(keys.ctypes.data), M, k, ctypes.c_void_p(ig.ctypes.data),
                              ctypes.c_void_p(tu.ctypes.data) if k > 1 else None, ctypes.c_void_p(di.ctypes.data),
                              None)
    _check(rc)
    return ig, tu[:, : k - 1], di


def max_ig_noalloc(x, y, k: int = 2, divisions: int = 1, discretizations: int = 1, range_: float = 0.0,
                   pc_xi: float = 0.25, seed: int = 0, out=None):
    """mdfs_max_ig_noalloc: k = 1 or 2 with all scratch in the library's fixed device array.

    x, y and the outputs must be CUDA tensors; outputs are allocated here (by
    torch) unless ``out`` passes (ig, tuples, disc).  Returns them like max_ig.
    """
    import torch
    lib = load()
    if not (_is_cuda(x) and _is_cuda(y)):
        raise TypeError("max_ig_noalloc needs CUDA tensors")
    data, keep = _data(x, y)
    M = data.M
    if out is None:
        ig = torch.empty(M, dtype=torch.float32, device=x.device)
        tu = torch.empty((M, 1), dtype=torch.int32, device=x.device)
        di = torch.empty(M, dtype=torch.int32, device=x.device)
    else:
        ig, tu, di = out
        _check_out(out, ((M,), (M, 1), (M,)), (np.float32, np.int32, np.int32), x)
    rc = lib.mdfs_max_ig_noalloc(ctypes.byref(data), k, divisions, discretizations, float(range_), float(pc_xi),
                                 int(seed) & (2**64 - 1), ctypes.c_void_p(ig.data_ptr()),
                                 ctypes.c_void_p(tu.data_ptr()) if k > 1 else None, ctypes.c_void_p(di.data_ptr()),
                                 _stream_of(x))
    _check(rc)
    del keep
    return ig, tu[:, : k - 1], di


def max_ig_raw(data_ptr_x, dtype: int, data_ptr_y, N: int, M: int, k: int, divisions: int, discretizations: int,
               range_: float, pc_xi: float, seed: int, ig_ptr, tuples_ptr, disc_ptr, stream_ptr):
    """Direct pass-through of raw pointers (host or device) to mdfs_max_ig."""
    lib = load()
    data = _Data(dtype, data_ptr_x, data_ptr_y, N, M)
    rc = lib.mdfs_max_ig(ctypes.byref(data), k, divisions, discretizations, float(range_), float(pc_xi),
                         int(seed) & (2**64 - 1), ctypes.c_void_p(ig_ptr),
                         ctypes.c_void_p(tuples_ptr) if tuples_ptr else None,
                         ctypes.c_void_p(disc_ptr) if disc_ptr else None,
                         ctypes.c_void_p(stream_ptr) if stream_ptr else None)
    _check(rc)


def ig_lim(ig, k: int, divisions: int, discretizations: int = 1, irrelevant_mask=None, alpha: float = 0.05):
    """chi^2 / extreme-value fit (section "Theory"): (p_values f64[M], IG_lim, T_hat)."""
    lib = load()
    M = int(ig.shape[0])
    lim = ctypes.c_double()
    neff = ctypes.c_double()
    if _is_cuda(ig):
        import torch
        igc = ig.contiguous().float()
        p = torch.empty(M, dtype=torch.float64, device=ig.device)
        mk = None
        if irrelevant_mask is not None:
            mk = torch.as_tensor(irrelevant_mask, device=ig.device).to(torch.uint8).contiguous()
            if mk.numel() != M:
                raise ValueError(f"irrelevant_mask holds {mk.numel()} entries, ig {M}")
        rc = lib.mdfs_ig_lim(ctypes.c_void_p(igc.data_ptr()), M, k, divisions, discretizations,
                             ctypes.c_void_p(mk.data_ptr()) if mk is not None else None, float(alpha),
                             ctypes.c_void_p(p.data_ptr()), ctypes.byref(lim), ctypes.byref(neff), _stream_of(ig))
    else:
        igc = _host(ig, np.float32)
        p = np.empty(M, dtype=np.float64)
        mk = _host(irrelevant_mask, np.uint8) if irrelevant_mask is not None else None
        if mk is not None and mk.size != M:
            raise ValueError(f"irrelevant_mask holds {mk.size} entries, ig {M}")
        rc = lib.mdfs_ig_lim(ctypes.c_void_p(igc.ctypes.data), M, k, divisions, discretizations,
                             ctypes.c_void_p(mk.ctypes.data) if mk is not None else None, float(alpha),
                             ctypes.c_void_p(p.ctypes.data), ctypes.byref(lim), ctypes.byref(neff), None)
    _check(rc)
    return p, lim.value, neff.value


def contrast(x, n_contrast: int, seed: int = 0):
    """Contrast variables (section "Canonical package usage"): returns
    (x_ext [(M + n_contrast), N] of x's dtype, src i32[n_contrast]) on the
    device of x (torch) or the host (numpy).  Row M + j is variable src[j] with
    its samples shuffled by a counter-based permutation (include/mdfs.h)."""
    lib = load()
    data, keep = _data(x, None)
    M, N = data.M, data.N
    if _is_cuda(x):
        import torch
        xe = torch.empty((M + n_contrast, N), dtype=x.dtype, device=x.device)
        src = torch.empty(max(n_contrast, 1), dtype=torch.int32, device=x.device)
        rc = lib.mdfs_contrast(ctypes.byref(data), int(n_contrast), int(seed) & (2**64 - 1),
                               ctypes.c_void_p(xe.data_ptr()), ctypes.c_void_p(src.data_ptr()), _stream_of(x))
    else:
        xe = np.empty((M + n_contrast, N), dtype=np.int8 if data.dtype == MDFS_I8 else np.float32)
        src = np.empty(max(n_contrast, 1), dtype=np.int32)
        rc = lib.mdfs_contrast(ctypes.byref(data), int(n_contrast), int(seed) & (2**64 - 1),
                               ctypes.c_void_p(xe.ctypes.data), ctypes.c_void_p(src.ctypes.data), None)
    _check(rc)
    del keep
    return xe, src[:n_contrast]


def p_adjust(p, method: str = "holm"):
    """Multiple-testing adjustment of p-values (Holm, Hochberg, Bonferroni, BH,
    BY, none) on the device; returns an array of the same kind as p."""
    lib = load()
    m = int(p.shape[0])
    if _is_cuda(p):
        import torch
        pc = p.contiguous().double()
        out = torch.empty(m, dtype=torch.float64, device=p.device)
        rc = lib.mdfs_p_adjust(ctypes.c_void_p(pc.data_ptr()), m, P_ADJUST[method], ctypes.c_void_p(out.data_ptr()),
                               _stream_of(p))
    else:
        pc = _host(p, np.float64)
        out = np.empty(m, dtype=np.float64)
        rc = lib.mdfs_p_adjust(ctypes.c_void_p(pc.ctypes.data), m, P_ADJUST[method], ctypes.c_void_p(out.ctypes.data),
                               None)
    _check(rc)
    return out


def select(x, y, n_contrast: int = None, k: int = 1, divisions: int = 1, discretizations: int = 1,
           range_: float = 0.0, pc_xi: float = 0.25, seed: int = 0, p_adjust_method: str = "holm",
           level: float = 0.05):
    """The canonical selection pipeline (section "Canonical package usage"):
    contrast variables, IG^k_max over the extended set, the chi^2 /
    extreme-value fit on the contrasts, adjusted p-values and the relevant set,
    all on the device.  n_contrast defaults to max(M, 30).  Returns a dict of
    arrays for the M original variables (torch on x's device, or numpy):
    ig, tuples, disc, p_value, adjusted_p_value, relevant (bool), plus ig_lim,
    n_eff and contrast_src."""
    lib = load()
    data, keep = _data(x, y)
    M = data.M
    nc = max(M, 30) if n_contrast is None else int(n_contrast)
    kk = max(k - 1, 1)
    lim = ctypes.c_double()
    neff = ctypes.c_double()
    if _is_cuda(x):
        import torch
        dev = x.device
        ig = torch.empty(M, dtype=torch.float32, device=dev)
        tu = torch.empty((M, kk), dtype=torch.int32, device=dev)
        di = torch.empty(M, dtype=torch.int32, device=dev)
        pv = torch.empty(M, dtype=torch.float64, device=dev)
        adj = torch.empty(M, dtype=torch.float64, device=dev)
        rel = torch.empty(M, dtype=torch.uint8, device=dev)
        src = torch.empty(nc, dtype=torch.int32, device=dev)
        ptr = lambda a: ctypes.c_void_p(a.data_ptr())
        stream = _stream_of(x)
    else:
        ig = np.empty(M, dtype=np.float32)
        tu = np.empty((M, kk), dtype=np.int32)
        di = np.empty(M, dtype=np.int32)
        pv = np.empty(M, dtype=np.float64)
        adj = np.empty(M, dtype=np.float64)
        rel = np.empty(M, dtype=np.uint8)
        src = np.empty(nc, dtype=np.int32)
        ptr = lambda a: ctypes.c_void_p(a.ctypes.data)
        stream = None
    rc = lib.mdfs_select(ctypes.byref(data), nc, k, divisions, discretizations, float(range_), float(pc_xi),
                         int(seed) & (2**64 - 1), P_ADJUST[p_adjust_method], float(level), ptr(ig),
                         ptr(tu) if k > 1 else None, ptr(di), ptr(pv), ptr(adj), ptr(rel), ctypes.byref(lim),
                         ctypes.byref(neff), ptr(src), stream)
    _check(rc)
    del keep
    return {"ig": ig, "tuples": tu[:, : k - 1], "disc": di, "p_value": pv, "adjusted_p_value": adj,
            "relevant": rel != 0, "ig_lim": lim.value, "n_eff": neff.value, "contrast_src": src}


def interesting_tuples(x, y, k: int = 2, divisions: int = 1, discretizations: int = 1, range_: float = 0.0,
                       pc_xi: float = 0.25, seed: int = 0, threshold: float = 0.0, capacity: int = 1 << 20):
    """Every (variable, partner tuple) whose IG, maximised over discretisations,
    reaches ``threshold`` (ComputeInterestingTuples, section "Examples").

    Returns (var i32[n], tuples i32[n, k-1], ig f32[n], disc i32[n]) sorted by
    (var, tuple), on the device of x (torch) or the host (numpy).  Raises
    MdfsError MDFS_ETRUNCATED when more than ``capacity`` records qualify."""
    lib = load()
    data, keep = _data(x, y)
    kk = max(k - 1, 1)
    count = ctypes.c_int64(0)
    if _is_cuda(x):
        import torch
        dev = x.device
        var = torch.empty(capacity, dtype=torch.int32, device=dev)
        tu = torch.empty((capacity, kk), dtype=torch.int32, device=dev)
        ig = torch.empty(capacity, dtype=torch.float32, device=dev)
        di = torch.empty(capacity, dtype=torch.int32, device=dev)
        ptr = lambda a: ctypes.c_void_p(a.data_ptr())
        stream = _stream_of(x)
    else:
        var = np.empty(capacity, dtype=np.int32)
        tu = np.empty((capacity, kk), dtype=np.int32)
        ig = np.empty(capacity, dtype=np.float32)
        di = np.empty(capacity, dtype=np.int32)
        ptr = lambda a: ctypes.c_void_p(a.ctypes.data)
        stream = None
    rc = lib.mdfs_interesting_tuples(ctypes.byref(data), k, divisions, discretizations, float(range_), float(pc_xi),
                                     int(seed) & (2**64 - 1), float(threshold), int(capacity), ptr(var),
                                     ptr(tu) if k > 1 else None, ptr(ig), ptr(di), ctypes.byref(count), stream)
    _check(rc)
    del keep
    n = count.value
    return var[:n], tu[:n, : k - 1], ig[:n], di[:n]


def last_launch_count() -> int:
    return load().mdfs_last_launch_count()


def profile(enable: bool) -> None:
    """Switches per-kernel CUDA-event timing of every library launch on or off."""
    _check(load().mdfs_profile(1 if enable else 0))


def profile_report() -> dict:
    """{kernel name: {"count": launches, "ms": total milliseconds}} since the last report."""
    buf = ctypes.create_string_buffer(1 << 16)
    _check(load().mdfs_profile_report(buf, len(buf)))
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms = line.split()
        out[name] = {"count": int(cnt), "ms": float(ms)}
    return out


def release() -> None:
    _check(load().mdfs_release())


def release_stream(stream) -> None:
    """Frees the library's workspace of one torch CUDA stream (no call in flight on it)."""
    _check(load().mdfs_release_stream(ctypes.c_void_p(stream.cuda_stream)))


def abi_version() -> int:
    return load().mdfs_abi_version()


# ---- hardware microbenchmarks (include/mdfs_bench.h) --------------------------
def bench_mma_f8(iters: int = 40000) -> dict:
    """Dense E4M3 tensor-core throughput of the current device (tcgen05.mma
    128 x 256 x 32 on shared-memory operands, one CTA per SM)."""
    tf, sec = ctypes.c_double(), ctypes.c_double()
    _check(load().mdfs_bench_mma_f8(int(iters), ctypes.byref(tf), ctypes.byref(sec)))
    return {"tflops": tf.value, "seconds": sec.value, "iters": int(iters)}


def bench_smem_lookup(iters: int = 4000, window: int = 0) -> dict:
    """Random 4-byte shared-memory loads per second (window 0: the whole 64 KB
    table; else that many consecutive entries at a warp-wide offset)."""
    rate, sec = ctypes.c_double(), ctypes.c_double()
    _check(load().mdfs_bench_smem_lookup(int(iters), int(window), ctypes.byref(rate), ctypes.byref(sec)))
    return {"lookups_per_s": rate.value, "seconds": sec.value, "iters": int(iters), "window": int(window)}


# ---- test-only entry points (include/mdfs_testing.h) -------------------------
def testing_counts(x, y, k: int, divisions: int = 1, discretizations: int = 1, range_: float = 0.0, seed: int = 0):
    """The voxel class counts of the tensor-core k = 2 / k = 3 kernels, as an
    int32 CUDA tensor [D, C(M, k), c^k] of n0 | n1 << 16 (x, y CUDA tensors)."""
    import math

    import torch
    lib = load()
    if not (_is_cuda(x) and _is_cuda(y)):
        raise ValueError("testing_counts takes CUDA tensors")
    data, keep = _data(x, y)
    c = divisions + 1
    # -1 marks entries the kernel did not write
    out = torch.full((discretizations, math.comb(data.M, k), c ** k), -1, dtype=torch.int32, device=x.device)
    rc = lib.mdfs_testing_counts(ctypes.byref(data), k, divisions, discretizations, float(range_),
                                 int(seed) & (2**64 - 1), ctypes.c_void_p(out.data_ptr()), _stream_of(x))
    _check(rc)
    del keep
    return out


def testing_k3_wait_fault(withhold_kb: int = -1, wait_ns: int = 0) -> None:
    """Arms (or, with the defaults, disarms) the one-shot bounded-wait hook of
    the next k = 3 tensor-core scan."""
    _check(load().mdfs_testing_k3_wait_fault(int(withhold_kb), int(wait_ns)))


def testing_exact() -> None:
    """Arms the one-shot hook under which the next tensor-core scan (k = 2 or
    k = 3) evaluates every tuple exactly (no entropy lower-bound skipping)."""
    _check(load().mdfs_testing_exact())
