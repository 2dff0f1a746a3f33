"""Host-side checks of the ctypes binding: preallocated outputs of max_ig are
refused unless they match the kind, device, dtype, shape and layout the
library writes (no GPU needed; the CUDA branch is driven with stand-ins that
carry torch's attributes)."""
import numpy as np
import pytest

from paper_1811_00631_gb300 import mdfs

torch = pytest.importorskip("torch")


class FakeCuda:
    """Stand-in for a CUDA tensor: the attributes _check_out reads."""

    def __init__(self, shape, dtype, device=0, contiguous=True):
        self.is_cuda = True
        self.shape = torch.Size(shape)
        self.dtype = dtype
        self.device = torch.device("cuda", device)
        self._contig = contiguous

    def is_contiguous(self):
        return self._contig


def _host_outs(M, kk):
    return np.empty(M, np.float32), np.empty((M, kk), np.int32), np.empty(M, np.int32)


def test_host_outputs_as_the_bench_allocates_them_pass():
    M = 500
    for k in (2, 3):
        kk = max(k - 1, 1)
        mdfs._check_out(_host_outs(M, kk), ((M,), (M, kk), (M,)), (np.float32, np.int32, np.int32),
                        np.zeros((M, 4), np.float32))


@pytest.mark.parametrize("bad", ["short", "dtype", "strided", "readonly", "not_numpy"])
def test_bad_host_outputs_are_refused(bad):
    M, kk = 40, 2
    ig, tu, di = _host_outs(M, kk)
    if bad == "short":
        ig = np.empty(M - 1, np.float32)
    elif bad == "dtype":
        tu = np.empty((M, kk), np.int64)
    elif bad == "strided":
        di = np.empty(2 * M, np.int32)[::2]
    elif bad == "readonly":
        ig.flags.writeable = False
    else:
        ig = [0.0] * M
    with pytest.raises(ValueError):
        mdfs._check_out((ig, tu, di), ((M,), (M, kk), (M,)), (np.float32, np.int32, np.int32),
                        np.zeros((M, 4), np.float32))


def test_cuda_outputs_as_the_bench_allocates_them_pass():
    M = 500
    x = FakeCuda((M, 2000), torch.float32)
    for k in (2, 3):
        kk = max(k - 1, 1)
        outs = (FakeCuda((M,), torch.float32), FakeCuda((M, kk), torch.int32), FakeCuda((M,), torch.int32))
        mdfs._check_out(outs, ((M,), (M, kk), (M,)), (np.float32, np.int32, np.int32), x)


@pytest.mark.parametrize("bad", ["host", "device", "dtype", "shape", "strided"])
def test_bad_cuda_outputs_are_refused(bad):
    M, kk = 40, 2
    x = FakeCuda((M, 100), torch.float32)
    outs = [FakeCuda((M,), torch.float32), FakeCuda((M, kk), torch.int32), FakeCuda((M,), torch.int32)]
    if bad == "host":
        outs[0] = np.empty(M, np.float32)
    elif bad == "device":
        outs[1] = FakeCuda((M, kk), torch.int32, device=1)
    elif bad == "dtype":
        outs[2] = FakeCuda((M,), torch.int64)
    elif bad == "shape":
        outs[1] = FakeCuda((M, kk + 1), torch.int32)
    else:
        outs[0] = FakeCuda((M,), torch.float32, contiguous=False)
    with pytest.raises(ValueError):
        mdfs._check_out(outs, ((M,), (M, kk), (M,)), (np.float32, np.int32, np.int32), x)


def test_short_batch_index_maps_are_refused():
    """mdfs_max_ig_batch reads n_jobs x N indices from each map: shorter maps
    are refused in the binding, before the library is called."""
    x = np.zeros((5, 20), np.float32)
    y = (np.arange(20) % 2).astype(np.uint8)
    good = np.zeros((3, 20), np.int32)
    with pytest.raises(ValueError, match="index map"):
        mdfs.max_ig_batch(x, y, good[:, :19], None, n_jobs=3)
    with pytest.raises(ValueError, match="index map"):
        mdfs.max_ig_batch(x, y, good, good[:2], n_jobs=3)
    with pytest.raises(ValueError, match="index map"):
        mdfs.max_ig_batch(x, y, good, None, n_jobs=4)


def test_fit_mask_of_the_wrong_length_is_refused():
    ig = np.ones(10, np.float32)
    with pytest.raises(ValueError, match="irrelevant_mask"):
        mdfs.ig_lim(ig, 1, 1, 1, np.ones(9, np.uint8))
