"""The bounds-checking build of the library (``build(debug=True)``: every kernel
checks its store and gather indices against the field, and the pitch padding of
the wavefields is verified after each forward and adjoint call) on small cases
that reach every edge of the grid: no check may fire, and the results must equal
the release build's bit for bit (the checks change no arithmetic).  Both builds
run in child processes, so this process's library stays the release one."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def run_cases(lib, out):
    env = dict(os.environ, WAVPROP_LIB=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_bounds_cases.py"), out], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return dict(np.load(out))


def test_debug_build_reports_nothing_and_matches_release(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_01995_gb300 import build
    release = build.build()
    debug = build.build(debug=True)
    got = run_cases(debug, str(tmp_path / "debug.npz"))
    ref = run_cases(release, str(tmp_path / "release.npz"))
    errors = {k: str(v) for k, v in got.items() if k.endswith("__message")}
    assert not errors, errors
    assert sorted(got) == sorted(ref)
    assert len(ref) >= 14
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k
