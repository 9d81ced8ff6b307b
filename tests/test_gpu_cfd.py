"""The CFD examples of Sec. 5 on the GPU against the FP64 oracle (oracle/cfd.py).

FP32 against FP64: 1e-5 relative L2 over at most a few hundred explicit steps (each
step's rounding is ~6e-8 relative, and the three schemes are contractive or
neutral where run).  Cases: the examples' own set-ups (hat function, spikes in the
right-hand side), ragged random fields, zero steps, the minimal 3 x 3 grid,
invalid input, and the benchmark size (8192^2) checked at sampled points: after n
steps a point depends only on the initial values within n cells, so the oracle
run on that window (one cell wider, its edges held fixed) gives the exact answer.
"""
import numpy as np
import pytest

from oracle import cfd
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


def hat(n, lo=0.5, hi=1.0, length=2.0):
    x = np.linspace(0, length, n)
    f = np.ones((n, n), dtype=np.float32)
    sel = (x >= lo) & (x <= hi)
    f[np.ix_(sel, sel)] = 2.0
    return f


def test_convection_example(ctx):
    n = 81
    dx = dy = 2.0 / (n - 1)
    c, sigma, nt = 1.0, 0.2, 100
    dt = sigma * dx
    u0 = hat(n)
    u = W.wp_convection_2d(ctx.handle, u0, dx, dy, dt, c, nt)
    ref = cfd.convection(u0, dx, dy, dt, c, nt)
    assert rel_l2(u, ref) < 1e-5
    assert np.array_equal(u[0], u0[0]) and np.array_equal(u[:, -1], u0[:, -1])


def test_burgers_example(ctx):
    n = 41
    dx = dy = 2.0 / (n - 1)
    nu, sigma, nt = 0.01, 0.0009, 120
    dt = sigma * dx * dy / nu
    u0 = hat(n)
    v0 = hat(n)
    u, v = W.wp_burgers_2d(ctx.handle, u0, v0, dx, dy, dt, nu, nt)
    ru, rv = cfd.burgers(u0, v0, dx, dy, dt, nu, nt)
    assert rel_l2(u, ru) < 1e-5 and rel_l2(v, rv) < 1e-5


def test_poisson_example(ctx):
    ny, nx, nit = 50, 50, 100
    dx, dy = 2.0 / (nx - 1), 1.0 / (ny - 1)
    b = np.zeros((ny, nx), dtype=np.float32)
    b[ny // 4, nx // 4] = 100.0
    b[3 * ny // 4, 3 * nx // 4] = -100.0
    p0 = np.zeros((ny, nx), dtype=np.float32)
    p = W.wp_poisson_2d(ctx.handle, p0, b, dx, dy, nit)
    ref = cfd.poisson(p0, b, dx, dy, nit)
    assert rel_l2(p, ref) < 1e-5


@pytest.mark.parametrize("ny,nx,steps", [(257, 300, 37), (3, 3, 5), (64, 129, 200), (131, 33, 1)])
def test_ragged_random_fields(ctx, ny, nx, steps):
    rng = np.random.default_rng(ny * 7 + nx)
    dx, dy = 0.013, 0.017
    u0 = rng.uniform(1.0, 2.0, (ny, nx)).astype(np.float32)
    v0 = rng.uniform(0.5, 1.5, (ny, nx)).astype(np.float32)
    c = 1.0
    dt = 0.45 / (c / dx + c / dy)
    assert rel_l2(W.wp_convection_2d(ctx.handle, u0, dx, dy, dt, c, steps), cfd.convection(u0, dx, dy, dt, c, steps)) < 1e-5
    nu = 0.001
    dtb = 0.4 / (2.0 / dx + 2.0 / dy + 2 * nu * (1 / dx**2 + 1 / dy**2))
    u, v = W.wp_burgers_2d(ctx.handle, u0, v0, dx, dy, dtb, nu, steps)
    ru, rv = cfd.burgers(u0, v0, dx, dy, dtb, nu, steps)
    assert rel_l2(u, ru) < 1e-5 and rel_l2(v, rv) < 1e-5
    b = rng.standard_normal((ny, nx)).astype(np.float32)
    assert rel_l2(W.wp_poisson_2d(ctx.handle, u0, b, dx, dy, steps), cfd.poisson(u0, b, dx, dy, steps)) < 1e-5


def test_zero_steps_device_arrays_and_errors(ctx):
    rng = np.random.default_rng(3)
    u0 = rng.uniform(1, 2, (20, 30)).astype(np.float32)
    assert np.array_equal(W.wp_convection_2d(ctx.handle, u0, 0.1, 0.1, 0.01, 1.0, 0), u0)
    u_host = W.wp_convection_2d(ctx.handle, u0, 0.1, 0.1, 0.01, 1.0, 9)
    out = torch.full(u0.shape, float("nan"), device="cuda")
    W.wp_convection_2d_dev(ctx.handle, torch.from_numpy(u0).cuda(), 0.1, 0.1, 0.01, 1.0, 9, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), u_host)
    uh, vh = W.wp_burgers_2d(ctx.handle, u0, u0 * 0.5, 0.1, 0.1, 0.001, 0.01, 7)
    uo, vo = torch.empty(u0.shape, device="cuda"), torch.empty(u0.shape, device="cuda")
    W.wp_burgers_2d_dev(ctx.handle, torch.from_numpy(u0).cuda(), torch.from_numpy(u0 * 0.5).cuda(), 0.1, 0.1, 0.001,
                        0.01, 7, uo, vo)
    torch.cuda.synchronize()
    assert np.array_equal(uo.cpu().numpy(), uh) and np.array_equal(vo.cpu().numpy(), vh)
    ph = W.wp_poisson_2d(ctx.handle, u0, u0, 0.1, 0.2, 11)
    po = torch.empty(u0.shape, device="cuda")
    W.wp_poisson_2d_dev(ctx.handle, torch.from_numpy(u0).cuda(), torch.from_numpy(u0).cuda(), 0.1, 0.2, 11, po)
    torch.cuda.synchronize()
    assert np.array_equal(po.cpu().numpy(), ph)
    with pytest.raises(W.WpError):
        W.wp_convection_2d(ctx.handle, u0, 0.1, 0.1, 0.1, 1.0, 3)      # Courant 2 > 1
    with pytest.raises(W.WpError):
        W.wp_convection_2d(ctx.handle, u0[:2], 0.1, 0.1, 0.01, 1.0, 3)  # ny < 3
    bad = u0.copy()
    bad[4, 5] = np.inf
    with pytest.raises(W.WpError):
        W.wp_poisson_2d(ctx.handle, bad, u0, 0.1, 0.1, 3)
    with pytest.raises(W.WpError):
        W.wp_convection_2d_dev(ctx.handle, torch.from_numpy(bad).cuda(), 0.1, 0.1, 0.01, 1.0, 3, out)
    assert np.isfinite(W.wp_convection_2d(ctx.handle, u0, 0.1, 0.1, 0.01, 1.0, 3)).all()


def _window(j, i, n, shape):
    r = n + 1
    j0, j1 = max(0, j - r), min(shape[0], j + r + 1)
    i0, i1 = max(0, i - r), min(shape[1], i + r + 1)
    return (slice(j0, j1), slice(i0, i1)), (j - j0, i - i0)


def test_benchmark_size_at_sampled_points(ctx):
    """8192^2 fields, 50 steps of each scheme, 24 sampled points (corners, edges,
    interior) against the oracle on their dependency windows."""
    ny = nx = 8192
    n = 50
    rng = np.random.default_rng(11)
    dx, dy = 1.0 / (nx - 1), 1.0 / (ny - 1)
    u0 = rng.uniform(1.0, 2.0, (ny, nx)).astype(np.float32)
    v0 = rng.uniform(0.5, 1.5, (ny, nx)).astype(np.float32)
    b = rng.standard_normal((ny, nx)).astype(np.float32)
    c = 1.0
    dt = 0.45 / (c / dx + c / dy)
    nu = 1e-7
    dtb = 0.4 / (2.0 / dx + 2.0 / dy + 2 * nu * (1 / dx**2 + 1 / dy**2))
    uc = W.wp_convection_2d(ctx.handle, u0, dx, dy, dt, c, n)
    ub, vb = W.wp_burgers_2d(ctx.handle, u0, v0, dx, dy, dtb, nu, n)
    pp = W.wp_poisson_2d(ctx.handle, u0, b, dx, dy, n)
    pts = [(1, 1), (1, nx - 2), (ny - 2, 1), (ny - 2, nx - 2), (0, 17), (ny - 1, 500), (4000, 0), (123, nx - 1)]
    pts += [tuple(int(t) for t in rng.integers(1, [ny - 1, nx - 1])) for _ in range(16)]
    for j, i in pts:
        sl, (jj, ii) = _window(j, i, n, (ny, nx))
        ref = cfd.convection(u0[sl], dx, dy, dt, c, n)[jj, ii]
        assert abs(uc[j, i] - ref) <= 1e-5 * abs(ref)
        ru, rv = cfd.burgers(u0[sl], v0[sl], dx, dy, dtb, nu, n)
        assert abs(ub[j, i] - ru[jj, ii]) <= 1e-5 * abs(ru[jj, ii]) and abs(vb[j, i] - rv[jj, ii]) <= 1e-5 * abs(rv[jj, ii])
        rp = cfd.poisson(u0[sl], b[sl], dx, dy, n)[jj, ii]
        assert abs(pp[j, i] - rp) <= 1e-5 * max(abs(rp), 1e-3)
