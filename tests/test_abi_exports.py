"""The C ABI library loads on a machine without a GPU and exports every entry
point declared in include/*.h (no compute calls are made here)."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(mdfs_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1811_00631_gb300 import build, mdfs
    build.build()
    return mdfs.load()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("mdfs_discretize", "mdfs_max_ig", "mdfs_ig_lim", "mdfs_last_error", "mdfs_release"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in _declared():
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_abi_version_and_error_string(lib):
    assert lib.mdfs_abi_version() == 1
    # the message is thread-local: a thread that has made no call sees ""
    import threading
    seen = []
    t = threading.Thread(target=lambda: seen.append(lib.mdfs_last_error()))
    t.start()
    t.join()
    assert seen == [b""]


def test_binding_names_match_header():
    from paper_1811_00631_gb300 import mdfs
    assert set(mdfs.EXPORTED) <= set(_declared())


def test_argument_errors_need_no_gpu(lib):
    """Host-side argument checks fail before any CUDA call."""
    import ctypes
    from paper_1811_00631_gb300 import mdfs
    import numpy as np
    x = np.zeros((4, 10), dtype=np.float32)
    y = np.zeros(10, dtype=np.uint8)
    d = mdfs._Data(0, x.ctypes.data, y.ctypes.data, 10, 4)
    ig = np.zeros(4, dtype=np.float32)
    rc = lib.mdfs_max_ig(ctypes.byref(d), 6, 1, 1, 0.0, 0.25, 1, ctypes.c_void_p(ig.ctypes.data), None, None, None)
    assert rc == -1 and b"k = 6" in lib.mdfs_last_error()
    rc = lib.mdfs_max_ig(ctypes.byref(d), 2, 1, 1, 0.0, 1.5, 1, ctypes.c_void_p(ig.ctypes.data), None, None, None)
    assert rc == -1 and b"pc_xi" in lib.mdfs_last_error()
    rc = lib.mdfs_max_ig(ctypes.byref(d), 2, 9, 1, 0.0, 0.5, 1, ctypes.c_void_p(ig.ctypes.data), None, None, None)
    assert rc == -1 and b"divisions" in lib.mdfs_last_error()
    rc = lib.mdfs_max_ig(ctypes.byref(d), 2, 1, 1025, 0.0, 0.5, 1, ctypes.c_void_p(ig.ctypes.data), None, None, None)
    assert rc == -1 and b"discretizations" in lib.mdfs_last_error()
    # N beyond the discretiser's limit (32768) and below 2; M = 0
    for n, m in [(32769, 4), (1, 4), (10, 0)]:
        dd = mdfs._Data(0, x.ctypes.data, y.ctypes.data, n, m)
        rc = lib.mdfs_max_ig(ctypes.byref(dd), 2, 1, 1, 0.0, 0.5, 1, ctypes.c_void_p(ig.ctypes.data), None, None,
                             None)
        assert rc == -1 and (b"N = " in lib.mdfs_last_error() or b"M = " in lib.mdfs_last_error())


def test_k5_limits_need_no_gpu(lib):
    """k = 5 argument limits: two to four classes per variable, C(M, 4) < 2^32,
    and for the single-word keys of a shard (and of every scan with three or
    four classes) also discretizations * C(M, 4) < 2^32."""
    import ctypes
    from paper_1811_00631_gb300 import mdfs
    import numpy as np

    def call(M, divisions, D, shard=False):
        x = np.zeros((M, 10), dtype=np.float32)
        y = (np.arange(10) % 2).astype(np.uint8)
        d = mdfs._Data(0, x.ctypes.data, y.ctypes.data, 10, M)
        out = np.zeros(M, dtype=np.uint64 if shard else np.float32)
        if shard:
            return lib.mdfs_max_ig_shard(ctypes.byref(d), 5, divisions, D, 0.0, 0.25, 1, 0, 1,
                                         ctypes.c_void_p(out.ctypes.data), None)
        return lib.mdfs_max_ig(ctypes.byref(d), 5, divisions, D, 0.0, 0.25, 1, ctypes.c_void_p(out.ctypes.data),
                               None, None, None)

    assert call(20, 4, 1) == -1 and b"divisions" in lib.mdfs_last_error()  # five classes
    assert call(200, 2, 67) == -1 and b"2^32" in lib.mdfs_last_error()  # three classes: 67 C(200, 4) > 2^32
    assert call(569, 1, 1) == -1 and b"C(M, 4)" in lib.mdfs_last_error()  # C(569, 4) > 2^32
    assert call(500, 1, 2, shard=True) == -1 and b"shard" in lib.mdfs_last_error()  # 2 C(500, 4) > 2^32
    assert call(4, 1, 1) == -1 and b"smaller than k" in lib.mdfs_last_error()


def test_profile_report_and_release_without_work(lib):
    """Tracing switches and an empty report need no GPU: nothing recorded
    gives an empty report; releasing with no workspace succeeds."""
    import ctypes
    assert lib.mdfs_profile(1) == 0
    buf = ctypes.create_string_buffer(64)
    assert lib.mdfs_profile_report(buf, 64) == 0
    assert buf.value == b""
    assert lib.mdfs_profile(0) == 0
    assert lib.mdfs_release() == 0
