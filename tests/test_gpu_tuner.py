"""The stage tuner of the k = 2 tensor-core kernel: a process with
MDFS_TUNE_FILE set writes its choice per shape there, a later process reads
it back instead of measuring, and every choice (measured, read back, forced to
either candidate, or tuning off) gives the same result bit for bit."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# one single-job scan and one batch; prints nothing, saves the results
SCRIPT = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1811_00631_gb300 import mdfs, synth
ds = synth.xor_pairs(N=600, M=150, n_pairs=4, seed=2)
ig, tu, di = mdfs.max_ig(ds.x, ds.y, 2, 2, 4, 0.5, 0.25, 3)
idx, yperm = synth.bootstrap_jobs(600, n_folds=3, n_perms=2, seed=4)
si = np.repeat(idx, 2, axis=0).astype(np.int32)
yp = np.tile(yperm, (3, 1)).astype(np.int32)
big, btu, bdi = mdfs.max_ig_batch(ds.x, ds.y, si, yp, k=2, divisions=1, discretizations=3)
np.savez(sys.argv[2], ig=ig, tu=tu, di=di, big=big, btu=btu, bdi=bdi)
"""


@pytest.fixture(scope="module")
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_00631_gb300 import build
    build.build()


def _run(tmp_path, name, env):
    out = str(tmp_path / f"{name}.npz")
    e = dict(os.environ)
    e.pop("MDFS_TUNE_FILE", None)
    e.pop("MDFS_TUNE", None)
    e.update(env)
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT, out], env=e, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return dict(np.load(out))


def test_tune_file_written_read_back_and_results_unchanged(built, tmp_path):
    tune = tmp_path / "tune.txt"
    first = _run(tmp_path, "first", {"MDFS_TUNE_FILE": str(tune)})
    lines = tune.read_text().splitlines()
    single = [ln for ln in lines if ln.startswith("k2tc_stages M=150 N=600 c=3 D=4 -> ")]
    batch = [ln for ln in lines if ln.startswith("k2tc_batch_stages M=150 N=600 c=2 D=3 -> ")]
    assert len(single) == 1 and len(batch) == 1, lines
    assert single[0].split(" -> ")[1] in ("3", "4") and batch[0].split(" -> ")[1] in ("3", "4")
    # a second process finds both shapes in the file and measures nothing
    again = _run(tmp_path, "again", {"MDFS_TUNE_FILE": str(tune)})
    assert tune.read_text().splitlines() == lines
    runs = [again, _run(tmp_path, "off", {"MDFS_TUNE": "0"})]
    for forced in ("3", "4"):
        f = tmp_path / f"forced{forced}.txt"
        f.write_text(f"k2tc_stages M=150 N=600 c=3 D=4 -> {forced}\n"
                     f"k2tc_batch_stages M=150 N=600 c=2 D=3 -> {forced}\n")
        runs.append(_run(tmp_path, f"forced{forced}", {"MDFS_TUNE_FILE": str(f)}))
    for r in runs:
        for key in first:
            assert np.array_equal(first[key], r[key]), key
