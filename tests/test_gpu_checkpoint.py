"""Gradient with binomial checkpointing (Sec. 3.3: the forward field recomputed
from a partial time history) on the GPU.

The recomputed forward states are produced by the same kernels as in the
periodic-snapshot path, so the gradient must be bit-identical to wp_gradient's
for every number of stored states (including none, the quadratic recompute from
the initial state), and within 1e-3 relative L2 of the FP64 oracle's
adjoint-state gradient (Eq. Grad).
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


def case(shape, k, nt, seed):
    true = synth.random_case(shape, k, nsrc=2, nrec=17, nbl=5, seed=seed, vmin=1800, vmax=2600)
    dt = 0.85 * O.cfl_dt(true.spacing, k, true.vmax)
    og = O.Grid(true.shape, true.spacing, true.origin, k, dt, nt)
    wg = W.Grid(true.shape, true.spacing, true.origin, k, dt, nt)
    q = true.wavelet(dt, nt)
    rng = np.random.default_rng(seed + 1)
    r = (rng.standard_normal((nt, len(true.rec))) * 1e-3).astype(np.float32)
    return true, og, wg, q, r


@pytest.mark.parametrize("shape,k,nt", [((26, 29, 33), 8, 60), ((45, 51), 4, 120)])
def test_checkpointed_gradient_equals_periodic_and_oracle(ctx, shape, k, nt):
    true, og, wg, q, r = case(shape, k, nt, 31)
    m, e = true.m32(), true.eta32()
    g_ref = O.gradient(og, m, e, q, true.src, r, true.rec)
    g_per = W.wp_gradient(ctx.handle, wg, m, e, q, true.src, r, true.rec, 7)
    assert rel_l2(g_per, g_ref) < 1e-3
    for c in (0, 1, 3, 8, nt):
        g = W.wp_gradient_checkpointed(ctx.handle, wg, m, e, q, true.src, r, true.rec, c)
        assert np.array_equal(g, g_per), c


def test_checkpointed_gradient_device_arrays(ctx):
    true, og, wg, q, r = case((24, 30, 27), 4, 50, 41)
    m, e = true.m32(), true.eta32()
    g_host = W.wp_gradient_checkpointed(ctx.handle, wg, m, e, q, true.src, r, true.rec, 4)
    out = torch.full(true.shape, float("nan"), device="cuda")
    W.wp_gradient_checkpointed_dev(ctx.handle, wg, torch.from_numpy(m).cuda(), torch.from_numpy(e).cuda(),
                                   torch.from_numpy(q).cuda(), true.src, torch.from_numpy(r).cuda(), true.rec, 4, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), g_host)


def test_checkpointed_gradient_rejects_bad_input(ctx):
    true, og, wg, q, r = case((20, 21, 22), 4, 10, 5)
    m, e = true.m32(), true.eta32()
    with pytest.raises(W.WpError):
        W.wp_gradient_checkpointed(ctx.handle, wg, m, e, q, true.src, r, true.rec, -1)
    r_bad = r.copy()
    r_bad[3, 2] = np.nan
    with pytest.raises(W.WpError):
        W.wp_gradient_checkpointed(ctx.handle, wg, m, e, q, true.src, r_bad, true.rec, 2)
    # the context stays usable
    g = W.wp_gradient_checkpointed(ctx.handle, wg, m, e, q, true.src, r, true.rec, 2)
    assert np.isfinite(g).all()


def test_checkpointed_gradient_large_model_matches_periodic(ctx):
    """The 3D gradient workload's central 48^3 with a 24-point layer (96^3, SO8,
    400 steps) with 12 stored states against 40 periodic snapshots: identical
    gradients."""
    true, start = synth.blobs_3d()
    t = synth.crop(true, 48, nbl=24, nt=400)
    s = synth.crop(start, 48, nbl=24, nt=400)
    k, nt = 8, 400
    dt = 0.9 * O.cfl_dt(t.spacing, k, max(t.vmax, s.vmax))
    wg = W.Grid(t.shape, t.spacing, t.origin, k, dt, nt)
    q = t.wavelet(dt, nt)
    d_obs = W.wp_forward(ctx.handle, wg, t.m32(), t.eta32(), q, t.src, t.rec)
    d0 = W.wp_forward(ctx.handle, wg, s.m32(), s.eta32(), q, t.src, t.rec)
    r = (d0 - d_obs).astype(np.float32)
    g_per = W.wp_gradient(ctx.handle, wg, s.m32(), s.eta32(), q, t.src, r, t.rec, 10)
    g_ck = W.wp_gradient_checkpointed(ctx.handle, wg, s.m32(), s.eta32(), q, t.src, r, t.rec, 12)
    assert np.abs(g_per).max() > 0
    assert np.array_equal(g_ck, g_per)
    assert math.isfinite(float(np.abs(g_ck).sum()))


@pytest.mark.parametrize("shape,k,nt", [((26, 29, 33), 8, 60), ((45, 51), 4, 120)])
def test_full_history_gradient_equals_snapshot_gradient(ctx, shape, k, nt):
    """snap_interval = 1 keeps every level once and recomputes nothing: the
    forward levels are the same kernel outputs, so the gradient is bit-identical."""
    true, og, wg, q, r = case(shape, k, nt, 37)
    m, e = true.m32(), true.eta32()
    g1 = W.wp_gradient(ctx.handle, wg, m, e, q, true.src, r, true.rec, 1)
    g7 = W.wp_gradient(ctx.handle, wg, m, e, q, true.src, r, true.rec, 7)
    assert np.abs(g1).max() > 0
    assert np.array_equal(g1, g7)


def test_full_history_autograd_and_receivers(ctx):
    from paper_1808_01995_gb300.autograd import AcousticPropagator, misfit
    true, og, wg, q, r = case((22, 27, 25), 4, 40, 43)
    m0, e = true.m32(), true.eta32()
    d_ref = W.wp_forward(ctx.handle, wg, m0, e, q, true.src, true.rec)
    grads = []
    for S in (1, 6):
        prop = AcousticPropagator(true.shape, true.spacing, true.origin, 4, wg.dt, wg.nt, true.src, true.rec, S, ctx)
        m = torch.from_numpy(m0).cuda().requires_grad_(True)
        d = prop(m, torch.from_numpy(e).cuda(), torch.from_numpy(q).cuda())
        assert np.array_equal(d.detach().cpu().numpy(), d_ref)
        misfit(d, torch.zeros_like(d)).backward()
        grads.append(m.grad.cpu().numpy())
    assert np.array_equal(grads[0], grads[1])


def test_automatic_snapshot_interval(ctx):
    """snap_interval = 0: the whole history when it fits, else the smallest interval
    that fits the context's budget; the gradient is the same either way."""
    true, og, wg, q, r = case((24, 26, 28), 4, 60, 47)
    m, e = true.m32(), true.eta32()
    g1 = W.wp_gradient(ctx.handle, wg, m, e, q, true.src, r, true.rec, 1)
    g_auto = W.wp_gradient(ctx.handle, wg, m, e, q, true.src, r, true.rec, 0)
    assert np.array_equal(g_auto, g1)
    field = 24 * 26 * 32 * 4  # pitched field bytes (x padded to 32)
    small = W.Context(0, hbm_budget_bytes=50 * field)
    try:
        g_tight = W.wp_gradient(small.handle, wg, m, e, q, true.src, r, true.rec, 0)
        assert W.wp_bytes_in_use(small.handle) <= 50 * field
    finally:
        small.close()
    assert np.array_equal(g_tight, g1)
    tiny = W.Context(0, hbm_budget_bytes=12 * field)
    try:
        with pytest.raises(W.WpError):
            W.wp_gradient(tiny.handle, wg, m, e, q, true.src, r, true.rec, 0)
    finally:
        tiny.close()
