"""Two time steps per stencil launch (temporal blocking) on the GPU, both ways:
mode 1 keeps u^{n+1} on chip (one kernel computes both steps), mode 2 runs the
two steps as two roles of CTAs in one cooperative launch.

Both evaluate the per-point arithmetic of the single-step stencil and of the
injection kernel in the same order, so a forward run must give the same receiver
data bit for bit with temporal blocking on and off, for
every covered order (2..8), ragged grids, odd and even step counts, graph and
non-graph loops, and sources anywhere (also in the damping layer and on tile
borders).  The FP64 oracle bounds it as well (1e-4 relative L2).
"""
import numpy as np
import pytest

import oracle as O
from paper_1808_01995_gb300 import synth
from paper_1808_01995_gb300 import wavprop as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_01995_gb300 import build
    build.build()
    c = W.Context(0)
    yield c
    c.close()


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run_both(ctx, grid, m, e, q, src, rec, mode=1):
    W.wp_set_temporal_blocking(ctx.handle, mode)
    l0 = W.wp_kernel_launches(ctx.handle)
    d_tb = W.wp_forward(ctx.handle, grid, m, e, q, src, rec)
    l1 = W.wp_kernel_launches(ctx.handle)
    W.wp_set_temporal_blocking(ctx.handle, 0)
    d_1 = W.wp_forward(ctx.handle, grid, m, e, q, src, rec)
    l2 = W.wp_kernel_launches(ctx.handle)
    return d_tb, d_1, l1 - l0, l2 - l1


@pytest.mark.parametrize("shape,k,nt,nsrc", [
    ((40, 37, 29), 8, 31, 1),     # odd nt: a last single step; graphs
    ((64, 48, 40), 4, 40, 3),     # several sources
    ((57, 33, 21), 2, 12, 2),     # no graphs (nt < 16)
    ((70, 50, 45), 6, 64, 2),
    ((120, 70, 50), 8, 48, 1),    # several tiles in x and y
    ((36, 36, 36), 8, 17, 8),     # 64 targets: the in-kernel limit
])
@pytest.mark.parametrize("mode", [1, 2])
def test_two_step_forward_is_bit_identical(ctx, shape, k, nt, nsrc, mode):
    case = synth.random_case(shape, k, nsrc=nsrc, nrec=40, nbl=5, seed=nt + k, vmin=1600, vmax=2800, nt=nt)
    dt = 0.9 * O.cfl_dt(case.spacing, k, case.vmax)
    grid = W.Grid(case.shape, case.spacing, case.origin, k, dt, nt)
    q = case.wavelet(dt, nt)
    m, e = case.m32(), case.eta32()
    d_tb, d_1, l_tb, l_1 = run_both(ctx, grid, m, e, q, case.src, case.rec, mode)
    assert np.abs(d_1).max() > 0
    assert np.array_equal(d_tb, d_1)
    assert l_tb < l_1  # one stencil launch per two steps
    og = O.Grid(case.shape, case.spacing, case.origin, k, dt, nt)
    d_ref = O.forward(og, m, e, q, case.src, case.rec)
    assert rel_l2(d_tb, d_ref) < 1e-4


@pytest.mark.parametrize("mode", [1, 2])
def test_many_sources_fall_back_to_single_steps(ctx, mode):
    # 10 sources = 80 injection targets: above the in-kernel limit, single steps run
    case = synth.random_case((30, 34, 38), 4, nsrc=10, nrec=20, nbl=4, seed=2, nt=20)
    dt = 0.9 * O.cfl_dt(case.spacing, 4, case.vmax)
    grid = W.Grid(case.shape, case.spacing, case.origin, 4, dt, 20)
    q = case.wavelet(dt, 20)
    d_tb, d_1, l_tb, l_1 = run_both(ctx, grid, case.m32(), case.eta32(), q, case.src, case.rec, mode)
    assert np.array_equal(d_tb, d_1)
    assert l_tb == l_1


@pytest.mark.parametrize("mode", [1, 2])
def test_two_step_adjoint_with_few_receivers(ctx, mode):
    case = synth.random_case((44, 39, 35), 8, nsrc=2, nrec=6, nbl=5, seed=9, nt=26)
    dt = 0.9 * O.cfl_dt(case.spacing, 8, case.vmax)
    grid = W.Grid(case.shape, case.spacing, case.origin, 8, dt, 26)
    rng = np.random.default_rng(4)
    d = rng.standard_normal((26, len(case.rec))).astype(np.float32)
    W.wp_set_temporal_blocking(ctx.handle, mode)
    a_tb = W.wp_adjoint(ctx.handle, grid, case.m32(), case.eta32(), d, case.rec, case.src)
    W.wp_set_temporal_blocking(ctx.handle, 0)
    a_1 = W.wp_adjoint(ctx.handle, grid, case.m32(), case.eta32(), d, case.rec, case.src)
    assert np.abs(a_1).max() > 0
    assert np.array_equal(a_tb, a_1)


@pytest.mark.parametrize("mode", [1, 2])
def test_two_step_on_the_bench_workload(ctx, mode):
    """336^3 SO8 (256^3 + 40-point layer), 40 steps, 16384 receivers."""
    model = synth.layers_3d(space_order=8, n=256, nt=40)
    dt = 0.9 * W.wp_cfl_dt(W.Grid(model.shape, model.spacing, model.origin, 8), model.vmax)
    grid = W.Grid(model.shape, model.spacing, model.origin, 8, dt, 40)
    q = model.wavelet(dt, 40)
    d_tb, d_1, l_tb, l_1 = run_both(ctx, grid, model.m32(), model.eta32(), q, model.src, model.rec, mode)
    assert np.abs(d_1).max() > 0
    assert np.array_equal(d_tb, d_1)
    assert l_tb < l_1
