"""The measurement arithmetic of bench.py, on the CPU.

- Compulsory stencil bytes per launch: 16 B per point (u^n, u^(n-1), b read,
  u^(n+1) written) plus 4 B per point where eta != 0 (s read).  On the layered
  workload the damping layer is everything outside the interior cube, so the
  damped count is (n + 2 nbl)^3 - n^3, a closed form independent of the code
  that counts it; at n = 256 this is the 691,552,256 B per launch that the
  roofline and the profiles quote.
- The gradient's compulsory bytes per point and step on the 280^3 workload
  (S = 10, 1500 steps): 68.43 B, the figure quoted beside its roofline.
- roofline.traffic is taken from a profile summary only while the kernel source
  it names has the sha recorded there.
"""
import hashlib
import os

import pytest

import bench


@pytest.mark.parametrize("n,nbl", [(24, 8), (40, 12), (32, 40)])
def test_algorithmic_bytes_match_the_closed_form(n, nbl):
    from paper_1808_01995_gb300 import synth
    model = synth.layers_3d(space_order=8, n=n, nbl=nbl, nt=4)
    side = n + 2 * nbl
    assert model.shape == (side, side, side)
    alg, npts, ndamp = bench.algorithmic_bytes_per_launch(model)
    assert npts == side ** 3
    assert ndamp == side ** 3 - n ** 3
    assert alg == 16 * side ** 3 + 4 * (side ** 3 - n ** 3)


def test_benchmark_grid_bytes_per_launch():
    side, n = 336, 256
    # the value quoted by the roofline and the profile summaries
    assert 16 * side ** 3 + 4 * (side ** 3 - n ** 3) == 691_552_256


def test_gradient_bytes_per_point_and_step():
    side, n, nt, S = 280, 200, 1500, 10
    npts, ndamp = side ** 3, side ** 3 - n ** 3
    alg = bench.gradient_alg_bytes(npts, ndamp, nt, nt // S)
    assert alg / (npts * nt) == pytest.approx(68.4348, abs=1e-4)
    # without recomputation (whole history): one forward stencil fewer, no snapshot pairs
    fh = bench.full_history_alg_bytes(npts, ndamp, nt)
    assert (alg - fh) == nt * (16 * npts + 4 * ndamp) + (nt // S) * 8 * npts


def test_traffic_is_read_only_for_the_recorded_kernel_source(tmp_path, monkeypatch):
    src_dir = tmp_path / "paper_1808_01995_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    kernel = b"// a kernel source\n"
    (src_dir / "stencil3d.cuh").write_bytes(kernel)
    sha = hashlib.sha256(kernel).hexdigest()[:16]
    prof = tmp_path / "profiles" / "stencil3d_fwd_so8_10x10x10.md"
    prof.write_text(f"# summary\n\n- stencil3d.cuh sha256[:16]: `{sha}`\n- dram bytes per launch: `123456`\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic(8, "10x10x10") == 123456.0
    assert bench.kernel_traffic(8, "11x11x11") is None          # no summary for that grid
    assert bench.kernel_traffic(16, "10x10x10") is None         # another kernel's summary
    (src_dir / "stencil3d.cuh").write_bytes(kernel + b"// edited\n")
    assert bench.kernel_traffic(8, "10x10x10") is None          # source changed since the capture
    assert os.path.exists(prof)
