"""Gradient by boundary-wavefield reconstruction (Sec. 3.3) on the GPU.

The forward field is rebuilt backward in time on the box Z where eta = 0 from
the stored ring of width k/2 around it.  On Z the gradient must match the FP64
oracle's adjoint-state gradient (Eq. Grad) within 1e-3 relative L2 and the
periodic-snapshot GPU gradient within the FP32 rounding of the reversal; in the
damping layer it is zero.
"""
import math

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


def zero_box(eta):
    idx = np.argwhere(eta == 0)
    lo, hi = idx.min(0), idx.max(0) + 1
    return tuple(slice(a, b) for a, b in zip(lo, hi))


def case(shape, k, nt, seed, nbl=6):
    """Random model with its sources and receivers moved off-grid into the physical
    domain (inside the box where eta = 0): a source inside the damping layer makes
    the ring's values many orders larger than the field inside the box, and the
    FP32 rounding of the reversal then swamps the small gradient there."""
    true = synth.random_case(shape, k, nsrc=2, nrec=19, nbl=nbl, seed=seed, vmin=1800, vmax=2600)
    rng = np.random.default_rng(seed + 3)
    lo = np.array(true.origin) + nbl * np.array(true.spacing)
    hi = np.array(true.origin) + (np.array(shape) - nbl - 1) * np.array(true.spacing)
    true.src = lo + rng.random((2, len(shape))) * (hi - lo)
    true.rec = lo + rng.random((19, len(shape))) * (hi - lo)
    dt = 0.85 * O.cfl_dt(true.spacing, k, true.vmax)
    og = O.Grid(true.shape, true.spacing, true.origin, k, dt, nt)
    wg = W.Grid(true.shape, true.spacing, true.origin, k, dt, nt)
    q = true.wavelet(dt, nt)
    rng = np.random.default_rng(seed + 7)
    r = (rng.standard_normal((nt, len(true.rec))) * 1e-3).astype(np.float32)
    return true, og, wg, q, r


@pytest.mark.parametrize("shape,k,nt", [((30, 33, 37), 8, 80), ((34, 29, 31), 16, 60), ((61, 57), 4, 200),
                                        ((40, 45), 2, 150),
                                        ((27, 31, 35), 2, 90),    # box x start rounded beyond the 1-point ring
                                        ((29, 26, 41), 6, 70)])
def test_reconstructed_gradient_matches_oracle_on_the_undamped_box(ctx, shape, k, nt):
    true, og, wg, q, r = case(shape, k, nt, 11)
    m, e = true.m32(), true.eta32()
    Z = zero_box(e)
    assert (e[Z] == 0).all()
    g_ref = O.gradient(og, m, e, q, true.src, r, true.rec)
    g = W.wp_gradient_reconstruct(ctx.handle, wg, m, e, q, true.src, r, true.rec)
    g_per = W.wp_gradient(ctx.handle, wg, m, e, q, true.src, r, true.rec, 9)
    err = rel_l2(g[Z], g_ref[Z])
    err_per = rel_l2(g[Z], g_per[Z])
    print(f"{shape} SO{k} nt={nt}: vs oracle {err:.2e}, vs snapshots {err_per:.2e}")
    assert err < 1e-3
    assert err_per < 1e-4
    mask = np.ones(e.shape, bool)
    mask[Z] = False
    assert (g[mask] == 0).all()


def test_reconstructed_gradient_device_arrays_and_repeatable(ctx):
    true, og, wg, q, r = case((26, 28, 30), 4, 60, 23)
    m, e = true.m32(), true.eta32()
    g_host = W.wp_gradient_reconstruct(ctx.handle, wg, m, e, q, true.src, r, true.rec)
    out = torch.full(true.shape, float("nan"), device="cuda")
    for _ in range(2):
        W.wp_gradient_reconstruct_dev(ctx.handle, wg, torch.from_numpy(m).cuda(), torch.from_numpy(e).cuda(),
                                      torch.from_numpy(q).cuda(), true.src, torch.from_numpy(r).cuda(), true.rec,
                                      out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), g_host)


def test_reconstruction_without_damping_is_the_whole_grid(ctx):
    # eta = 0 everywhere: Z is the grid, the ring is the zero Dirichlet halo
    true, og, wg, q, r = case((24, 25, 27), 8, 50, 3)
    m = true.m32()
    e = np.zeros_like(m)
    g_ref = O.gradient(og, m, e, q, true.src, r, true.rec)
    g = W.wp_gradient_reconstruct(ctx.handle, wg, m, e, q, true.src, r, true.rec)
    assert rel_l2(g, g_ref) < 1e-3


def test_reconstruction_rejects_eta_without_a_zero_box(ctx):
    true, og, wg, q, r = case((20, 22, 24), 4, 20, 5)
    m, e = true.m32(), true.eta32()
    e_all = np.full_like(e, 1e-4) * m
    with pytest.raises(W.WpError, match="nonzero everywhere"):
        W.wp_gradient_reconstruct(ctx.handle, wg, m, e_all, q, true.src, r, true.rec)
    e_hole = e.copy()
    Z = zero_box(e)
    c = tuple((s.start + s.stop) // 2 for s in Z)
    e_hole[c] = 1e-4 * m[c]
    with pytest.raises(W.WpError, match="not a box"):
        W.wp_gradient_reconstruct(ctx.handle, wg, m, e_hole, q, true.src, r, true.rec)
    g = W.wp_gradient_reconstruct(ctx.handle, wg, m, e, q, true.src, r, true.rec)
    assert np.isfinite(g).all()


def test_reconstruction_on_the_gradient_workload_crop(ctx):
    """The 3D gradient workload's central 48^3 with a 40-point layer (128^3, SO8,
    1500 steps): the reconstructed gradient on the 48^3 interior against the
    periodic-snapshot gradient and the oracle."""
    true_full, start_full = synth.blobs_3d()
    t = synth.crop(true_full, 48, nt=1500)
    s = synth.crop(start_full, 48, nt=1500)
    k, nt = 8, 1500
    dt = 0.9 * O.cfl_dt(t.spacing, k, max(t.vmax, s.vmax))
    wg = W.Grid(t.shape, t.spacing, t.origin, k, dt, nt)
    og = O.Grid(t.shape, t.spacing, t.origin, k, dt, nt)
    q = t.wavelet(dt, nt)
    d_obs = W.wp_forward(ctx.handle, wg, t.m32(), t.eta32(), q, t.src, t.rec)
    d0 = W.wp_forward(ctx.handle, wg, s.m32(), s.eta32(), q, t.src, t.rec)
    r = (d0 - d_obs).astype(np.float32)
    e = s.eta32()
    Z = zero_box(e)
    g_rec = W.wp_gradient_reconstruct(ctx.handle, wg, s.m32(), e, q, t.src, r, t.rec)
    g_per = W.wp_gradient(ctx.handle, wg, s.m32(), e, q, t.src, r, t.rec, 10)
    g_ref = O.gradient(og, s.m32(), e, q, t.src, r, t.rec, checkpoint_every=10)
    err_per = rel_l2(g_rec[Z], g_per[Z])
    err = rel_l2(g_rec[Z], g_ref[Z])
    print(f"blobs crop 128^3 nt=1500: reconstructed vs snapshots {err_per:.2e}, vs oracle {err:.2e}")
    assert err_per < 1e-4
    assert err < 1e-3
    assert math.isfinite(float(np.abs(g_rec).sum()))
