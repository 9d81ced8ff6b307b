"""GPU gradient path: the torch.autograd Function on the misfit (Eq. AS) against
the FP64 oracle's adjoint-state gradient (Eq. Grad) and against centred finite
differences of the GPU forward map; the 3D FWI gradient workload (layered model
plus Gaussian blobs, start model smoothed by a 20-point Gaussian, SO8, 1500
steps, snapshots every 10 steps) on its 48^3 crop against the oracle, and at full
size (200^3 + 40-point layer) against the oracle and by finite differences.

Tolerances: gradient 1e-3 relative L2 against the oracle; directional
derivative within 1e-2 of centred finite differences of the FP32 forward.
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


def smooth_random(shape, rng, passes=3):
    u = rng.standard_normal(shape)
    for _ in range(passes):
        for a in range(len(shape)):
            u = (np.roll(u, 1, a) + 2 * u + np.roll(u, -1, a)) / 4
    return u / np.abs(u).max()


def fwi_pair(true, start, nt, S, k):
    from paper_1808_01995_gb300.autograd import AcousticPropagator
    vmax = max(true.vmax, start.vmax)
    dt = 0.9 * O.cfl_dt(true.spacing, k, vmax)
    og = O.Grid(true.shape, true.spacing, true.origin, k, dt, nt)
    q = true.wavelet(dt, nt)
    return dt, og, q


def test_autograd_gradient_matches_oracle(ctx):
    from paper_1808_01995_gb300.autograd import AcousticPropagator, misfit
    true = synth.random_case((28, 31, 34), 8, nsrc=1, nrec=20, nbl=6, seed=5, vmin=1800, vmax=2600)
    rng = np.random.default_rng(3)
    m0 = (true.m * (1.0 + 0.04 * smooth_random(true.shape, rng))).astype(np.float32)
    nt, S = 90, 8
    dt = 0.85 * O.cfl_dt(true.spacing, 8, 1.0 / math.sqrt(float(m0.min())))
    og = O.Grid(true.shape, true.spacing, true.origin, 8, dt, nt)
    q = true.wavelet(dt, nt)
    e32 = true.eta32()
    d_obs = O.forward(og, true.m32(), e32, q, true.src, true.rec)
    d0 = O.forward(og, m0, e32, q, true.src, true.rec)
    g_ref = O.gradient(og, m0, e32, q, true.src, (d0 - d_obs).astype(np.float32), true.rec)

    prop = AcousticPropagator(true.shape, true.spacing, true.origin, 8, dt, nt, true.src, true.rec, S, ctx)
    m = torch.from_numpy(m0).cuda().requires_grad_(True)
    eta = torch.from_numpy(e32).cuda()
    wav = torch.from_numpy(q).cuda().requires_grad_(True)
    d = prop(m, eta, wav)
    assert rel_l2(d.detach().cpu().numpy(), d0) < 1e-4
    J = misfit(d, torch.from_numpy(d_obs.astype(np.float32)).cuda())
    J.backward()
    err = rel_l2(m.grad.cpu().numpy(), g_ref)
    print(f"autograd dJ/dm vs oracle: rel L2 {err:.3e}")
    assert err < 1e-3
    # dJ/dq = F^T (d - d_obs): the oracle's adjoint of its own residual
    q_ref = O.adjoint(og, m0, e32, (d0 - d_obs).astype(np.float32), true.rec, true.src)
    assert rel_l2(wav.grad.cpu().numpy(), q_ref) < 1e-3


def test_backward_twice_and_linear_in_upstream_gradient(ctx):
    from paper_1808_01995_gb300.autograd import AcousticPropagator
    model = synth.random_case((20, 22, 24), 4, nsrc=1, nrec=9, nbl=4, seed=8)
    dt = 0.9 * O.cfl_dt(model.spacing, 4, model.vmax)
    prop = AcousticPropagator(model.shape, model.spacing, model.origin, 4, dt, 40, model.src, model.rec, 6, ctx)
    m = torch.from_numpy(model.m32()).cuda().requires_grad_(True)
    d = prop(m, torch.from_numpy(model.eta32()).cuda(), torch.from_numpy(model.wavelet(dt, 40)).cuda())
    gen = torch.Generator(device="cuda").manual_seed(8)
    r = torch.randn(d.shape, device="cuda", generator=gen)
    (g1,) = torch.autograd.grad(d, m, r, retain_graph=True)
    # a second backward pass from the same state repeats the first one exactly
    (g1b,) = torch.autograd.grad(d, m, r, retain_graph=True)
    assert torch.equal(g1, g1b)
    # scaling the upstream gradient by two scales every FP32 operation of the
    # backward pass exactly (up to the rounding of denormal results)
    (g2,) = torch.autograd.grad(d, m, 2.0 * r)
    assert torch.allclose(g2, 2.0 * g1, rtol=1e-6, atol=1e-30 + 1e-7 * g1.abs().max().item())


def _fd_check(ctx, true, start_m, dt, nt, S, k, q, d_obs, direction, eps_list):
    from paper_1808_01995_gb300.autograd import AcousticPropagator, misfit
    prop = AcousticPropagator(true.shape, true.spacing, true.origin, k, dt, nt, true.src, true.rec, S, ctx)
    eta = torch.from_numpy(true.eta32()).cuda()
    wav = torch.from_numpy(q).cuda()
    dobs = torch.from_numpy(np.asarray(d_obs, np.float32)).cuda()
    m = torch.from_numpy(start_m).cuda().requires_grad_(True)
    J = misfit(prop(m, eta, wav), dobs)
    J.backward()
    dm = torch.from_numpy(direction.astype(np.float32)).cuda()
    pred = float((m.grad.double() * dm.double()).sum())
    errs = []
    with torch.no_grad():
        for eps in eps_list:
            jp = float(misfit(prop(m + eps * dm, eta, wav), dobs).double())
            jm = float(misfit(prop(m - eps * dm, eta, wav), dobs).double())
            fd = (jp - jm) / (2 * eps)
            errs.append(abs(fd - pred) / abs(pred))
    return m.grad.detach().cpu().numpy(), errs


@pytest.fixture(scope="module")
def blobs():
    true, start = synth.blobs_3d()
    return true, start


def test_blobs_crop_gradient_matches_oracle_and_fd(ctx, blobs):
    """48^3 crop (+40-point layer = 128^3), SO8, 1500 steps, snapshots every 10."""
    true_full, start_full = blobs
    tc = synth.crop(true_full, 48, nt=1500)
    sc = synth.crop(start_full, 48, nt=1500)
    sc.eta = tc.eta.copy()
    k, nt, S = 8, 1500, 10
    dt = 0.9 * O.cfl_dt(tc.spacing, k, max(tc.vmax, sc.vmax))
    og = O.Grid(tc.shape, tc.spacing, tc.origin, k, dt, nt)
    q = tc.wavelet(dt, nt)
    e32 = tc.eta32()
    m0 = sc.m32()
    d_obs = O.forward(og, tc.m32(), e32, q, tc.src, tc.rec)
    d0 = O.forward(og, m0, e32, q, tc.src, tc.rec)
    g_ref = O.gradient(og, m0, e32, q, tc.src, (d0 - d_obs).astype(np.float32), tc.rec, checkpoint_every=S)
    rng = np.random.default_rng(17)
    direction = 0.01 * m0 * smooth_random(tc.shape, rng)
    g, errs = _fd_check(ctx, tc, m0, dt, nt, S, k, q, d_obs, direction, [1.0, 0.5])
    err = rel_l2(g, g_ref)
    print(f"blobs 48^3 crop (128^3, nt=1500): gradient rel L2 vs oracle {err:.3e}; FD {errs}")
    assert err < 1e-3
    assert min(errs) < 1e-2


def test_blobs_full_size_gradient_by_finite_differences(ctx, blobs):
    """200^3 + 40-point layer (280^3), SO8, 1500 steps, snapshots every 10: the
    autograd gradient's directional derivative against centred differences of
    the FP32 forward map."""
    true, start = blobs
    k, nt, S = 8, 1500, 10
    dt = 0.9 * W.wp_cfl_dt(W.Grid(true.shape, true.spacing, true.origin, k), max(true.vmax, start.vmax))
    q = true.wavelet(dt, nt)
    # J = 1/2 ||F(m) q||^2 (d_obs = 0): a check of the GPU gradient against the
    # GPU forward map it differentiates, a property that holds at any size
    d_obs = np.zeros((nt, len(true.rec)), np.float32)
    start.eta = true.eta.copy()
    rng = np.random.default_rng(23)
    m0 = start.m32()
    direction = 0.01 * m0 * smooth_random(true.shape, rng, passes=2)
    g, errs = _fd_check(ctx, true, m0, dt, nt, S, k, q, d_obs, direction, [1.0, 0.5])
    print(f"blobs 280^3 nt=1500: directional derivative vs centred FD {errs}")
    assert np.isfinite(g).all()
    assert min(errs) < 1e-2


def test_blobs_full_size_gradient_matches_oracle(ctx, blobs):
    """The benchmark's gradient exactly: 200^3 + 40-point layer (280^3), SO8, 1500
    steps, snapshots every 10 steps, 40000 receivers, wp_fwi_gradient_dev with the
    true model's damping; misfit and gradient against the FP64 oracle over the
    whole grid, observed data from the oracle's forward of the true model (about
    two minutes and 21 GB on the host)."""
    true, start = blobs
    k, nt, S = 8, 1500, 10
    dt = 0.9 * O.cfl_dt(true.spacing, k, max(true.vmax, start.vmax))
    og = O.Grid(true.shape, true.spacing, true.origin, k, dt, nt)
    wg = W.Grid(true.shape, true.spacing, true.origin, k, dt, nt)
    q = true.wavelet(dt, nt)
    e32 = true.eta32()
    m0 = start.m32()
    d_obs = O.forward(og, true.m32(), e32, q, true.src, true.rec).astype(np.float32)
    d0 = O.forward(og, m0, e32, q, true.src, true.rec)
    J_ref = 0.5 * float(((d0 - d_obs) ** 2).sum())
    g_ref = O.gradient(og, m0, e32, q, true.src, (d0 - d_obs).astype(np.float32), true.rec,
                       checkpoint_every=40)
    g = torch.empty(true.shape, device="cuda")
    J = W.wp_fwi_gradient_dev(ctx.handle, wg, torch.from_numpy(m0).cuda(), torch.from_numpy(e32).cuda(),
                              torch.from_numpy(q).cuda(), true.src, torch.from_numpy(d_obs).cuda(), true.rec,
                              S, g)
    torch.cuda.synchronize()
    err = rel_l2(g.cpu().numpy(), g_ref)
    print(f"blobs 280^3 nt=1500: misfit {J:.6e} vs oracle {J_ref:.6e}; gradient rel L2 vs oracle {err:.3e}")
    assert abs(J - J_ref) <= 1e-3 * J_ref
    assert err < 1e-3


def test_fwi_gradient_call_matches_oracle(ctx):
    """wp_fwi_gradient (host and device arrays): misfit and gradient of one shot."""
    true = synth.random_case((22, 27, 30), 4, nsrc=1, nrec=14, nbl=5, seed=19, vmin=1800, vmax=2600)
    rng = np.random.default_rng(6)
    m0 = (true.m * (1.0 + 0.03 * smooth_random(true.shape, rng))).astype(np.float32)
    nt, S = 70, 9
    dt = 0.85 * O.cfl_dt(true.spacing, 4, 1.0 / math.sqrt(float(m0.min())))
    og = O.Grid(true.shape, true.spacing, true.origin, 4, dt, nt)
    wg = W.Grid(true.shape, true.spacing, true.origin, 4, dt, nt)
    q = true.wavelet(dt, nt)
    e32 = true.eta32()
    d_obs = O.forward(og, true.m32(), e32, q, true.src, true.rec).astype(np.float32)
    d0 = O.forward(og, m0, e32, q, true.src, true.rec)
    J_ref = 0.5 * float(((d0 - d_obs) ** 2).sum())
    g_ref = O.gradient(og, m0, e32, q, true.src, (d0 - d_obs).astype(np.float32), true.rec)
    g, J = W.wp_fwi_gradient(ctx.handle, wg, m0, e32, q, true.src, d_obs, true.rec, S)
    assert abs(J - J_ref) <= 1e-4 * J_ref
    assert rel_l2(g, g_ref) < 1e-3
    gd = torch.empty(true.shape, device="cuda")
    Jd = W.wp_fwi_gradient_dev(ctx.handle, wg, torch.from_numpy(m0).cuda(), torch.from_numpy(e32).cuda(),
                               torch.from_numpy(q).cuda(), true.src, torch.from_numpy(d_obs).cuda(), true.rec, S, gd)
    torch.cuda.synchronize()
    assert Jd == J
    assert np.array_equal(gd.cpu().numpy(), g)
