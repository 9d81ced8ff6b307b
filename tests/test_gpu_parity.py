"""GPU parity: the CUDA path (called through the C ABI) against the FP64 oracle on
identical seeded inputs.

Tolerances: one update within 1e-5 relative (max norm) of the oracle;
receiver data, adjoint data and many-step fields within 1e-4 relative L2;
the GPU dot test within 1e-5; gradients within 1e-3 relative L2.
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
    yield c.handle
    c.close()


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def grids(model, dt, nt, k=None):
    k = k or model.space_order
    return (O.Grid(model.shape, model.spacing, model.origin, k, dt, nt),
            W.Grid(model.shape, model.spacing, model.origin, k, dt, nt))


def f32(x):
    return np.asarray(x, np.float32)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, np.float32))).cuda()


def smooth_random(shape, rng, passes=2):
    u = rng.standard_normal(shape)
    for _ in range(passes):
        for a in range(len(shape)):
            u = (np.roll(u, 1, a) + 2 * u + np.roll(u, -1, a)) / 4
    return u


# ragged shapes spanning several 32 x 16 tiles and z chunks
SHAPES_3D = [(37, 45, 70), (20, 17, 33), (9, 33, 64)]
SHAPES_2D = [(45, 70), (141, 141), (17, 33)]


@pytest.mark.parametrize("shape", SHAPES_3D + SHAPES_2D)
@pytest.mark.parametrize("k", [2, 4, 8, 12, 16])
def test_one_update_matches_oracle(ctx, shape, k):
    model = synth.random_case(shape, k, nbl=4, seed=len(shape) * 100 + k)
    dt = 0.9 * O.cfl_dt(model.spacing, k, model.vmax)
    og, wg = grids(model, dt, 1)
    rng = np.random.default_rng(k)
    up = f32(smooth_random(shape, rng))
    u = f32(smooth_random(shape, rng))
    m32, e32 = model.m32(), model.eta32()
    ref = O.step(og, m32, e32, up, u)
    tp, tu = dev(up), dev(u)
    W.wp_propagate_dev(ctx, wg, dev(m32), dev(e32), tp, tu, 1)
    got = tu.cpu().numpy()
    assert np.array_equal(tp.cpu().numpy(), u)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < 1e-5, err


@pytest.mark.parametrize("shape,k", [((37, 45, 70), 8), ((20, 17, 33), 16), ((45, 70), 4), ((64, 40), 12)])
def test_hundred_updates_match_oracle(ctx, shape, k):
    model = synth.random_case(shape, k, nbl=5, seed=7)
    dt = 0.9 * O.cfl_dt(model.spacing, k, model.vmax)
    og, wg = grids(model, dt, 1)
    rng = np.random.default_rng(1)
    u0 = f32(smooth_random(shape, rng, 4))
    m32, e32 = model.m32(), model.eta32()
    rp, ru = O.run(og, m32, e32, u0, u0, 100)
    tp, tu = dev(u0), dev(u0)
    W.wp_propagate_dev(ctx, wg, dev(m32), dev(e32), tp, tu, 100)
    assert rel_l2(tu.cpu().numpy(), ru) < 1e-4
    assert rel_l2(tp.cpu().numpy(), rp) < 1e-4


def _forward_case(model, k, nt, dt=None):
    dt = dt or 0.9 * O.cfl_dt(model.spacing, k, model.vmax)
    og, wg = grids(model, dt, nt, k)
    q = model.wavelet(dt, nt)
    return og, wg, q


@pytest.mark.parametrize("shape", [(30, 41, 38), (47, 66)])
@pytest.mark.parametrize("k", range(2, 17, 2))
def test_forward_matches_oracle(ctx, shape, k):
    model = synth.random_case(shape, k, nsrc=3, nrec=25, nbl=6, seed=k)
    og, wg, q = _forward_case(model, k, 80)
    m32, e32 = model.m32(), model.eta32()
    ref = O.forward(og, m32, e32, q, model.src, model.rec)
    got = W.wp_forward(ctx, wg, m32, e32, q, model.src, model.rec)
    assert got.shape == ref.shape
    assert rel_l2(got, ref) < 1e-4


def test_forward_circle_2d_config(ctx):
    """2D forward case of the paper's shape: 101^2 + 20-point layer, SO4, 500 ms,
    10 Hz source at (z=20 m, x=500 m), 101 receivers along z = 20 m."""
    model = synth.circle_2d()
    dt, nt = model.time_axis(O.cfl_dt(model.spacing, 4, model.vmax))
    assert nt == 227 and abs(dt - 0.5 / 227) < 1e-15
    og, wg = grids(model, dt, nt)
    q = model.wavelet(dt, nt)
    m32, e32 = model.m32(), model.eta32()
    ref = O.forward(og, m32, e32, q, model.src, model.rec)
    got = W.wp_forward(ctx, wg, m32, e32, q, model.src, model.rec)
    err = rel_l2(got, ref)
    per_trace = [rel_l2(got[:, i], ref[:, i]) for i in range(0, 101, 10)]
    print(f"circle2d forward rel L2 {err:.3e}, worst sampled trace {max(per_trace):.3e}")
    assert err < 1e-4


def test_forward_device_and_host_calls_agree(ctx):
    model = synth.random_case((26, 35, 40), 8, nsrc=2, nrec=30, nbl=5, seed=3)
    og, wg, q = _forward_case(model, 8, 40)
    m32, e32 = model.m32(), model.eta32()
    host = W.wp_forward(ctx, wg, m32, e32, q, model.src, model.rec)
    out = torch.zeros((40, 30), device="cuda")
    W.wp_forward_dev(ctx, wg, dev(m32), dev(e32), dev(q), model.src, model.rec, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), host)
    # deterministic: a second call gives the same bits
    again = W.wp_forward(ctx, wg, m32, e32, q, model.src, model.rec)
    assert np.array_equal(again, host)


@pytest.mark.parametrize("shape,k", [((30, 41, 38), 8), ((47, 66), 4), ((22, 19, 35), 16), ((40, 44), 2)])
def test_adjoint_matches_oracle(ctx, shape, k):
    model = synth.random_case(shape, k, nsrc=3, nrec=21, nbl=6, seed=40 + k)
    og, wg, _ = _forward_case(model, k, 70)
    rng = np.random.default_rng(5)
    y = f32(rng.standard_normal((70, 21)))
    m32, e32 = model.m32(), model.eta32()
    ref = O.adjoint(og, m32, e32, y, model.rec, model.src)
    got = W.wp_adjoint(ctx, wg, m32, e32, y, model.rec, model.src)
    assert rel_l2(got, ref) < 1e-4


@pytest.mark.parametrize("shape,k", [((30, 41, 38), 8), ((47, 66), 4), ((25, 27, 29), 16), ((50, 52), 12)])
def test_gpu_dot_test(ctx, shape, k):
    model = synth.random_case(shape, k, nsrc=4, nrec=17, nbl=6, seed=60 + k)
    og, wg, _ = _forward_case(model, k, 90)
    rng = np.random.default_rng(8)
    x = f32(rng.standard_normal((90, 4)))
    y = f32(rng.standard_normal((90, 17)))
    m32, e32 = model.m32(), model.eta32()
    Fx = W.wp_forward(ctx, wg, m32, e32, x, model.src, model.rec).astype(np.float64)
    Fty = W.wp_adjoint(ctx, wg, m32, e32, y, model.rec, model.src).astype(np.float64)
    a, b = float((Fx * y).sum()), float((x * Fty).sum())
    assert abs(a - b) / abs(a) < 1e-5


@pytest.mark.parametrize("shape,k,S", [((24, 27, 30), 8, 7), ((40, 45), 4, 1), ((40, 45), 4, 50),
                                        ((18, 21, 23), 16, 4), ((33, 36), 12, 9)])
def test_gradient_matches_oracle(ctx, shape, k, S):
    true = synth.random_case(shape, k, nsrc=1, nrec=15, nbl=5, seed=70 + k, vmin=1800, vmax=2600)
    rng = np.random.default_rng(11)
    m0 = (true.m * (1.0 + 0.03 * smooth_random(shape, rng))).astype(np.float32)
    nt = 50
    dt = 0.8 * O.cfl_dt(true.spacing, k, 1.0 / math.sqrt(float(m0.min())))
    og, wg = grids(true, dt, nt)
    q = true.wavelet(dt, nt)
    e32 = true.eta32()
    d_obs = O.forward(og, true.m32(), e32, q, true.src, true.rec)
    d0 = O.forward(og, m0, e32, q, true.src, true.rec)
    res = f32(d0 - d_obs)
    ref = O.gradient(og, m0, e32, q, true.src, res, true.rec)
    got = W.wp_gradient(ctx, wg, m0, e32, q, true.src, res, true.rec, S)
    assert rel_l2(got, ref) < 1e-3


def test_gradient_independent_of_snapshot_interval(ctx):
    model = synth.random_case((20, 23, 26), 8, nsrc=1, nrec=9, nbl=4, seed=5)
    og, wg, q = _forward_case(model, 8, 31)
    rng = np.random.default_rng(2)
    res = f32(rng.standard_normal((31, 9)))
    m32, e32 = model.m32(), model.eta32()
    gs = [W.wp_gradient(ctx, wg, m32, e32, q, model.src, res, model.rec, S) for S in (1, 5, 31, 100)]
    for g in gs[1:]:
        assert np.array_equal(g, gs[0])


# ---------------------------------------------------------------------------
# edge cases and errors
# ---------------------------------------------------------------------------

def test_edge_cases(ctx):
    model = synth.random_case((12, 13, 14), 4, nsrc=2, nrec=3, nbl=2, seed=9)
    og, wg, q = _forward_case(model, 4, 10)
    m32, e32 = model.m32(), model.eta32()
    # nt = 0
    g0 = W.Grid(model.shape, model.spacing, model.origin, 4, wg.dt, 0)
    assert W.wp_forward(ctx, g0, m32, e32, np.zeros((0, 2)), model.src, model.rec).shape == (0, 3)
    # no sources: zero data
    d = W.wp_forward(ctx, wg, m32, e32, np.zeros((10, 0)), None, model.rec)
    assert np.array_equal(d, np.zeros((10, 3), np.float32))
    # no receivers
    assert W.wp_forward(ctx, wg, m32, e32, q, model.src, None).shape == (10, 0)
    # a grid smaller than the stencil radius (k = 16 on 3 x 4 x 5)
    tiny = synth.random_case((3, 4, 5), 16, nsrc=1, nrec=2, nbl=0, seed=1)
    tog, twg, tq = _forward_case(tiny, 16, 6)
    ref = O.forward(tog, tiny.m32(), tiny.eta32(), tq, tiny.src, tiny.rec)
    got = W.wp_forward(ctx, twg, tiny.m32(), tiny.eta32(), tq, tiny.src, tiny.rec)
    assert rel_l2(got, ref) < 1e-5
    # no damping anywhere (no damped tiles)
    und = synth.random_case((20, 33, 40), 8, nsrc=1, nrec=5, nbl=0, seed=2)
    uog, uwg, uq = _forward_case(und, 8, 30)
    assert not und.eta.any()
    ref = O.forward(uog, und.m32(), und.eta32(), uq, und.src, und.rec)
    assert rel_l2(W.wp_forward(ctx, uwg, und.m32(), und.eta32(), uq, und.src, und.rec), ref) < 1e-4


def _status(fn):
    with pytest.raises(W.WpError) as e:
        fn()
    return e.value.status


def test_errors_are_reported_and_context_stays_usable(ctx):
    model = synth.random_case((12, 13, 14), 4, nsrc=1, nrec=3, nbl=2, seed=9)
    og, wg, q = _forward_case(model, 4, 10)
    m32, e32 = model.m32(), model.eta32()
    too_big = W.Grid(wg.shape, wg.spacing, wg.origin, 4, 1.5 * O.cfl_dt(model.spacing, 4, model.vmax), 10)
    assert _status(lambda: W.wp_forward(ctx, too_big, m32, e32, q, model.src, model.rec)) == W.WP_ECFL
    bad = m32.copy()
    bad[3, 4, 5] = np.nan
    assert _status(lambda: W.wp_forward(ctx, wg, bad, e32, q, model.src, model.rec)) == W.WP_ENONFINITE
    qbad = q.copy()
    qbad[2, 0] = np.inf
    assert _status(lambda: W.wp_forward(ctx, wg, m32, e32, qbad, model.src, model.rec)) == W.WP_ENONFINITE
    neg = m32.copy()
    neg[0, 0, 0] = -1.0
    assert _status(lambda: W.wp_forward(ctx, wg, neg, e32, q, model.src, model.rec)) == W.WP_EINVAL
    outside = model.rec.copy()
    outside[1, 2] = model.origin[2] - 1.0
    assert _status(lambda: W.wp_forward(ctx, wg, m32, e32, q, model.src, outside)) == W.WP_EINVAL
    odd = W.Grid(wg.shape, wg.spacing, wg.origin, 5, wg.dt, 10)
    assert _status(lambda: W.wp_forward(ctx, odd, m32, e32, q, model.src, model.rec)) == W.WP_EINVAL
    # after all that the context still computes the right answer
    ref = O.forward(og, m32, e32, q, model.src, model.rec)
    assert rel_l2(W.wp_forward(ctx, wg, m32, e32, q, model.src, model.rec), ref) < 1e-4


def test_budget_exhaustion_is_reported():
    model = synth.random_case((12, 13, 14), 4, nsrc=1, nrec=3, nbl=2, seed=9)
    og, wg, q = _forward_case(model, 4, 10)
    with W.Context(0, hbm_budget_bytes=0) as c:
        assert _status(lambda: W.wp_forward(c.handle, wg, model.m32(), model.eta32(), q, model.src,
                                            model.rec)) == W.WP_ENOMEM
    with W.Context(0, hbm_budget_bytes=64 << 20) as c:
        big = W.Grid((400, 400, 400), (10.0,) * 3, (0.0,) * 3, 4, 1e-3, 5)
        m = np.full(big.shape, 1 / 2000 ** 2, np.float32)
        assert _status(lambda: W.wp_forward(c.handle, big, m, np.zeros_like(m), np.zeros((5, 0)), None,
                                            None)) == W.WP_ENOMEM


# ---------------------------------------------------------------------------
# full-size workload (3D sweep, 256^3 + 40-point layer = 336^3, SO8), in the
# launch configuration the benchmark times
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def layers_so8():
    return synth.layers_3d(space_order=8)


def test_full_size_updates_match_oracle(ctx, layers_so8):
    model = layers_so8
    dt, nt = model.time_axis(O.cfl_dt(model.spacing, 8, model.vmax))
    og, wg = grids(model, dt, 1)
    rng = np.random.default_rng(12)
    u0 = f32(smooth_random(model.shape, rng, 1))
    m32, e32 = model.m32(), model.eta32()
    rp, ru = O.run(og, m32, e32, u0, u0, 6)
    tp, tu = dev(u0), dev(u0)
    W.wp_propagate_dev(ctx, wg, dev(m32), dev(e32), tp, tu, 6)
    got = tu.cpu().numpy()
    err = rel_l2(got, ru)
    print(f"336^3 SO8, 6 updates: rel L2 {err:.3e}")
    assert err < 1e-5


def test_full_size_dot_test(ctx, layers_so8):
    model = layers_so8
    dt, nt = model.time_axis(O.cfl_dt(model.spacing, 8, model.vmax))
    wg = W.Grid(model.shape, model.spacing, model.origin, 8, dt, nt)
    rng = np.random.default_rng(13)
    x = f32(rng.standard_normal((nt, len(model.src))))
    y = f32(rng.standard_normal((nt, len(model.rec))))
    m = dev(model.m32())
    e = dev(model.eta32())
    Fx = torch.zeros((nt, len(model.rec)), device="cuda")
    Fty = torch.zeros((nt, len(model.src)), device="cuda")
    W.wp_forward_dev(ctx, wg, m, e, dev(x), model.src, model.rec, Fx)
    W.wp_adjoint_dev(ctx, wg, m, e, dev(y), model.rec, model.src, Fty)
    a = float((Fx.double().cpu().numpy() * y).sum())
    b = float((x * Fty.double().cpu().numpy()).sum())
    err = abs(a - b) / abs(a)
    print(f"336^3 SO8 nt={nt}: dot test {err:.3e}")
    assert err < 1e-5


@pytest.mark.parametrize("k", [8, 4, 16])
def test_full_size_forward_matches_oracle(ctx, k):
    """The benchmark's shot exactly: 336^3, 1000 steps, 16384 off-grid receivers,
    the device-array call the benchmark times; every trace against the FP64 oracle
    run over the whole grid (a few tens of seconds on the host cores)."""
    model = synth.layers_3d(space_order=k)
    dt = 0.9 * O.cfl_dt(model.spacing, k, model.vmax)
    nt = model.nt
    og, wg = grids(model, dt, nt, k)
    m32, e32 = model.m32(), model.eta32()
    q = model.wavelet(dt, nt)
    out = torch.zeros((nt, len(model.rec)), device="cuda")
    W.wp_forward_dev(ctx, wg, dev(m32), dev(e32), dev(q), model.src, model.rec, out)
    got = out.cpu().numpy()
    ref = O.forward(og, m32, e32, q, model.src, model.rec)
    err = rel_l2(got, ref)
    # the traces nearest the source carry most of the energy; check the far ones too
    far = np.argsort(np.linalg.norm(ref, axis=0))[: len(model.rec) // 2]
    err_far = rel_l2(got[:, far], ref[:, far])
    print(f"336^3 SO{k} nt={nt}: rel L2 {err:.3e} (weaker half of the traces {err_far:.3e})")
    assert err < 1e-4
    assert err_far < 1e-4
