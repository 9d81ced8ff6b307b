"""Multi-shot FWI driver (Sec. 3.4): the objective and gradient summed over shots
against the sum of the FP64 oracle's per-shot values; the fixed-step update with
bounds; the accumulation and update kernels against a float64 reference."""
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


def test_axpy_and_model_update_kernels(ctx):
    rng = np.random.default_rng(0)
    x = rng.standard_normal(100003).astype(np.float32)
    y = rng.standard_normal(100003).astype(np.float32)
    tx, ty = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    W.wp_axpy_dev(ctx.handle, -0.37, tx, ty)
    ref = y.astype(np.float64) - 0.37 * x.astype(np.float64)
    assert np.abs(ty.cpu().numpy() - ref).max() <= 1e-6 * np.abs(ref).max()
    m = (1e-7 * (2 + rng.random(5000))).astype(np.float32)
    g = rng.standard_normal(5000).astype(np.float32)
    tm, tg = torch.from_numpy(m).cuda(), torch.from_numpy(g).cuda()
    lo, hi = np.float32(1.5e-7), np.float32(2.5e-7)
    W.wp_update_model_dev(ctx.handle, 3e-8, tg, tm, float(lo), float(hi))
    ref = np.clip(m.astype(np.float64) - 3e-8 * g.astype(np.float64), lo, hi)
    assert np.abs(tm.cpu().numpy() - ref).max() <= 1e-6 * hi


def test_multishot_gradient_matches_oracle_sum_and_descends(ctx):
    from paper_1808_01995_gb300.fwi import MultiShotFWI, Shot
    shape, k, nt = (26, 30, 34), 8, 70
    true = synth.random_case(shape, k, nsrc=4, nrec=24, nbl=5, seed=41, vmin=1800, vmax=2600)
    rng = np.random.default_rng(12)
    m0 = (true.m * (1.0 + 0.04 * smooth_random(shape, rng))).astype(np.float32)
    dt = 0.85 * O.cfl_dt(true.spacing, k, 1.0 / math.sqrt(float(m0.min())) * 1.05)
    og = O.Grid(shape, true.spacing, true.origin, k, dt, nt)
    grid = W.Grid(shape, true.spacing, true.origin, k, dt, nt)
    e32 = true.eta32()
    q = synth.ricker(30.0, dt, nt).astype(np.float32)[:, None]
    shots, J_ref, g_ref = [], 0.0, np.zeros(shape)
    for s in range(4):
        src = true.src[s:s + 1]
        d_obs = O.forward(og, true.m32(), e32, q, src, true.rec).astype(np.float32)
        d0 = O.forward(og, m0, e32, q, src, true.rec)
        J_ref += 0.5 * float(((d0 - d_obs) ** 2).sum())
        g_ref += O.gradient(og, m0, e32, q, src, (d0 - d_obs).astype(np.float32), true.rec)
        shots.append(Shot(torch.from_numpy(q).cuda(), src, true.rec, torch.from_numpy(d_obs).cuda()))
    fwi = MultiShotFWI(grid, torch.from_numpy(e32).cuda(), shots, snap_interval=9, slots=2)
    try:
        m = torch.from_numpy(m0).cuda()
        J, g = fwi.objective_and_gradient(m)
        assert abs(J - J_ref) <= 1e-4 * J_ref
        err = rel_l2(g.cpu().numpy(), g_ref)
        print(f"4-shot gradient vs sum of oracle gradients: rel L2 {err:.3e}")
        assert err < 1e-3
        # fixed-step descent with bounds on m
        step = 0.01 * float(m.abs().max()) / float(g.abs().max())
        lo, hi = float(true.m.min()) * 0.8, float(true.m.max()) * 1.2
        Js = []
        for _ in range(3):
            Jk, _ = fwi.fixed_step(m, step, lo, hi)
            Js.append(Jk)
        Jend, _ = fwi.objective_and_gradient(m)
        Js.append(Jend)
        print("misfit over three fixed steps:", Js)
        assert all(b < a for a, b in zip(Js, Js[1:]))
        assert float(m.min()) >= lo * (1 - 1e-6) and float(m.max()) <= hi * (1 + 1e-6)
    finally:
        fwi.close()
