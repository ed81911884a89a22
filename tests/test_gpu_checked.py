"""The bounds-checked build (the substitute for a memory sanitizer, which is
not available on this GPU pool): every index the step kernels compute into a
global or shared array is tested against the array's extent; one outside it
sets a status bit and the access is skipped.  tests/checked_cases.py runs every
kernel variant on small ragged lattices, once with the checked library and once
with the normal one, each in a child process: no index may leave its array, and
the two builds must give bit-identical populations (the checks change no
arithmetic)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _run(lib, out):
    env = dict(os.environ, WDLB_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_cases.py"), out], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return np.load(out)


def test_checked_build_finds_no_index_outside_its_array(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1304_7880_gb300 import build
    lib_checked = build.build(checked=True)
    lib_normal = build.build()
    a = _run(lib_checked, str(tmp_path / "checked.npz"))
    b = _run(lib_normal, str(tmp_path / "normal.npz"))
    assert sorted(a.files) == sorted(b.files) and len(a.files) >= 20
    for k in a.files:
        assert np.array_equal(a[k], b[k]), k
