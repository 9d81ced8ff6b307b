"""Large 3D workload (512 x 512 x 400 interior + 40-point layer, SO16, 3000 steps,
25 Hz, 256 x 256 receivers, salt body over a 1.5 -> 4 km/s gradient, snapshots
every 20 steps): forward data and gradient on the central 64^3 crop against the
FP64 oracle, and, when the device has room for the snapshots, the full-size
gradient against centred finite differences of the FP32 forward."""
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


def test_salt_crop_forward_and_gradient_match_oracle(ctx):
    k, nt, S = 16, 3000, 20
    true = synth.crop(synth.salt_3d(), 64, nt=nt)
    start = synth.crop(synth.salt_3d(with_salt=False), 64, nt=nt)
    start.eta = true.eta.copy()
    dt = 0.9 * O.cfl_dt(true.spacing, k, max(true.vmax, start.vmax))
    og = O.Grid(true.shape, true.spacing, true.origin, k, dt, nt)
    wg = W.Grid(true.shape, true.spacing, true.origin, k, dt, nt)
    q = true.wavelet(dt, nt)
    e32 = true.eta32()
    d_obs = O.forward(og, true.m32(), e32, q, true.src, true.rec)
    got = W.wp_forward(ctx.handle, wg, true.m32(), e32, q, true.src, true.rec)
    err_f = rel_l2(got, d_obs)
    m0 = start.m32()
    d0 = O.forward(og, m0, e32, q, true.src, true.rec)
    res = (d0 - d_obs).astype(np.float32)
    g_ref = O.gradient(og, m0, e32, q, true.src, res, true.rec, checkpoint_every=S)
    g = W.wp_gradient(ctx.handle, wg, m0, e32, q, true.src, res, true.rec, S)
    err_g = rel_l2(g, g_ref)
    print(f"salt 64^3 crop ({true.shape}), SO16, nt={nt}: forward rel L2 {err_f:.3e}, gradient rel L2 {err_g:.3e}")
    assert err_f < 1e-4
    assert err_g < 1e-3


def test_salt_full_size_gradient_by_finite_differences(ctx):
    from paper_1808_01995_gb300.autograd import AcousticPropagator, misfit
    true = synth.salt_3d()
    k, nt, S = 16, 3000, 20
    dt = 0.9 * W.wp_cfl_dt(W.Grid(true.shape, true.spacing, true.origin, k), true.vmax)
    grid = W.Grid(true.shape, true.spacing, true.origin, k, dt, nt)
    need = W.wp_estimate_bytes(grid, 1, len(true.rec), 1, S) + 4 * int(np.prod(true.shape)) * 4
    free, _ = torch.cuda.mem_get_info()
    if need > 0.9 * free:
        pytest.skip(f"needs ~{need / 2**30:.0f} GiB of device memory, {free / 2**30:.0f} GiB free")
    prop = AcousticPropagator(true.shape, true.spacing, true.origin, k, dt, nt, true.src, true.rec, S, ctx)
    eta = torch.from_numpy(true.eta32()).cuda()
    wav = torch.from_numpy(true.wavelet(dt, nt)).cuda()
    m = torch.from_numpy(true.m32()).cuda().requires_grad_(True)
    J = misfit(prop(m, eta, wav), torch.zeros((nt, len(true.rec)), device="cuda"))
    J.backward()
    del J  # releases the resident snapshots before the finite-difference runs
    import gc
    gc.collect()
    rng = np.random.default_rng(29)
    dm = torch.from_numpy((0.005 * true.m32() * rng.standard_normal(true.shape)).astype(np.float32)).cuda()
    pred = float((m.grad.double() * dm.double()).sum())
    with torch.no_grad():
        d0 = torch.zeros((nt, len(true.rec)), device="cuda")
        jp = float(misfit(prop(m + dm, eta, wav), d0).double())
        jm = float(misfit(prop(m - dm, eta, wav), d0).double())
    err = abs((jp - jm) / 2 - pred) / abs(pred)
    print(f"salt full size {true.shape}, SO16, nt={nt}: directional derivative vs centred FD {err:.3e}")
    assert np.isfinite(m.grad.cpu().numpy()).all()
    assert err < 1e-2
