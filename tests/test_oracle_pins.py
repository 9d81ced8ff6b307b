"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each check is a closed form, an
exact discrete solution, brute force on tiny grids, an adjoint identity, a
Taylor expansion, a complex-step derivative, or a number the paper prints
(tests/golden/paper_verification.json).
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_1808_01995_gb300 import synth

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_verification.json")))


# ---------------------------------------------------------------------------
# independent helpers (exact arithmetic, dense matrices) used only by the pins
# ---------------------------------------------------------------------------

def taylor_weights(k):
    """a_0..a_p from the Taylor moment conditions, solved in exact fractions:
    sum_{j=1}^p 2 a_j j^(2i) = 2 [i == 1] for i = 1..p, a_0 = -2 sum a_j."""
    p = k // 2
    A = [[Fraction(2 * j ** (2 * i)) for j in range(1, p + 1)] + [Fraction(2 if i == 1 else 0)]
         for i in range(1, p + 1)]
    for c in range(p):                       # Gauss-Jordan in fractions
        piv = next(r for r in range(c, p) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        for r in range(p):
            if r != c and A[r][c] != 0:
                f = A[r][c] / A[c][c]
                A[r] = [x - f * y for x, y in zip(A[r], A[c])]
    a = [A[i][p] / A[i][i] for i in range(p)]
    return [-2 * sum(a)] + a


def lap_symbol_max(w, nth=20001):
    th = np.linspace(0.0, math.pi, nth)
    s = -float(w[0]) - 2.0 * sum(float(w[j]) * np.cos(j * th) for j in range(1, len(w)))
    return float(s.max())


def dense_interp(shape, spacing, origin, pts):
    """Multilinear interpolation matrix (npts x N), written independently."""
    nd = len(shape)
    N = int(np.prod(shape))
    P = np.zeros((len(pts), N))
    for i, c in enumerate(pts):
        base, frac = [], []
        for a in range(nd):
            t = min(max((c[a] - origin[a]) / spacing[a], 0.0), shape[a] - 1.0)
            b = min(int(math.floor(t)), shape[a] - 2)
            base.append(b)
            frac.append(t - b)
        for corner in np.ndindex(*([2] * nd)):
            wgt = 1.0
            idx = []
            for a in range(nd):
                wgt *= frac[a] if corner[a] else 1.0 - frac[a]
                idx.append(base[a] + corner[a])
            P[i, np.ravel_multi_index(idx, shape)] += wgt
    return P


def dense_laplacian(shape, spacing, k):
    w = [float(x) for x in taylor_weights(k)]
    N = int(np.prod(shape))
    L = np.zeros((N, N))
    for p in np.ndindex(*shape):
        i = np.ravel_multi_index(p, shape)
        for a in range(len(shape)):
            L[i, i] += w[0] / spacing[a] ** 2
            for j in range(1, k // 2 + 1):
                for s in (-j, j):
                    q = list(p)
                    q[a] += s
                    if 0 <= q[a] < shape[a]:
                        L[i, np.ravel_multi_index(q, shape)] += w[j] / spacing[a] ** 2
    return L


def dense_F(grid, m, eta, src, rec):
    """F = P_r A(m)^{-1} dt^2 P_s^T as a dense (nt*nrec) x (nt*nsrc) matrix, A the
    block lower-triangular matrix of the time-stepping (Sec. 2.2.2)."""
    shape, nt, dt = grid.shape, grid.nt, grid.dt
    N = int(np.prod(shape))
    L = dense_laplacian(shape, grid.spacing, grid.space_order)
    m = np.asarray(m, float).ravel()
    eta = np.asarray(eta, float).ravel()
    D = np.diag(m + eta * dt / 2)
    E = np.diag(m - eta * dt / 2)
    M = 2 * np.diag(m) + dt * dt * L
    A = np.zeros((nt * N, nt * N))
    for n in range(nt):
        A[n * N:(n + 1) * N, n * N:(n + 1) * N] = D
        if n >= 1:
            A[n * N:(n + 1) * N, (n - 1) * N:n * N] = -M
        if n >= 2:
            A[n * N:(n + 1) * N, (n - 2) * N:(n - 1) * N] = E
    Ps = dense_interp(shape, grid.spacing, grid.origin, src)
    Pr = dense_interp(shape, grid.spacing, grid.origin, rec)
    Inj = np.kron(np.eye(nt), dt * dt * Ps.T)
    Smp = np.kron(np.eye(nt), Pr)
    return Smp @ np.linalg.solve(A, Inj)


def grid_of(model, dt, nt, k=None):
    return O.Grid(model.shape, model.spacing, model.origin, k or model.space_order, dt, nt)


# ---------------------------------------------------------------------------
# (i) finite-difference weights
# ---------------------------------------------------------------------------

EXACT = {
    2: [Fraction(-2), Fraction(1)],
    4: [Fraction(-5, 2), Fraction(4, 3), Fraction(-1, 12)],
    8: [Fraction(-205, 72), Fraction(8, 5), Fraction(-1, 5), Fraction(8, 315), Fraction(-1, 560)],
}


@pytest.mark.parametrize("k", [2, 4, 8])
def test_weights_match_textbook_rationals(k):
    w = O.fd_weights(k)
    assert np.allclose(w, [float(x) for x in EXACT[k]], rtol=0, atol=1e-15)


@pytest.mark.parametrize("k", range(2, 17, 2))
def test_weights_solve_taylor_moment_conditions(k):
    exact = taylor_weights(k)
    w = O.fd_weights(k)
    assert len(w) == k // 2 + 1
    assert np.allclose(w, [float(x) for x in exact], rtol=1e-14, atol=1e-15)
    if k == 16:
        assert exact[0] == Fraction(-1077749, 352800)
    # the three-point rule of the second derivative, [1, -2, 1]
    if k == 2:
        assert list(w) == [-2.0, 1.0]


@pytest.mark.parametrize("k", [2, 4, 8, 12, 16])
def test_stencil_order_of_accuracy_on_polynomials(k):
    """The stencil differentiates x^q exactly for q <= k+1 and not x^(k+2)."""
    w = O.fd_weights(k)
    p = k // 2
    for q in range(0, k + 3):
        approx = w[0] * 0.0 ** q + sum(w[j] * ((j * 1.0) ** q + (-j * 1.0) ** q) for j in range(1, p + 1))
        exact = 2.0 if q == 2 else 0.0
        if q <= k + 1:
            assert abs(approx - exact) < 1e-9 * (p ** q + 1)
        elif q == k + 2:
            assert abs(approx - exact) > 1e-6


# ---------------------------------------------------------------------------
# CFL limit
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("k,A", [(2, 4.0), (4, 16.0 / 3.0), (8, 6.502), (12, 7.073), (16, 7.427)])
def test_cfl_bound_matches_symbol_maximum(k, A):
    w = taylor_weights(k)
    smax = lap_symbol_max(w)
    assert abs(smax - A) < 2e-3
    h = (7.0, 11.0, 13.0)
    dt = O.cfl_dt(h, k, 2500.0)
    lam = sum(smax / hh ** 2 for hh in h)
    assert abs(2500.0 ** 2 * dt * dt * lam - 4.0) < 1e-6


@pytest.mark.parametrize("factor,stable", [(0.97, True), (1.05, False)])
def test_cfl_stability_threshold(factor, stable):
    k, n, h, c = 4, 40, 10.0, 2000.0
    dt = factor * O.cfl_dt((h, h), k, c)
    g = O.Grid((n, n), (h, h), (0.0, 0.0), k, dt, 1)
    rng = np.random.default_rng(3)
    u0 = rng.standard_normal((n, n))
    up, u = O.run(g, np.full((n, n), 1 / c ** 2), np.zeros((n, n)), u0, u0, 600)
    growth = np.abs(u).max() / np.abs(u0).max()
    assert (growth < 10.0) == stable


# ---------------------------------------------------------------------------
# (ii) exact discrete standing wave, convergence orders
# ---------------------------------------------------------------------------

def _mode(n, L, q):
    nd = len(q)
    x = np.arange(n) * (L / (n - 1))
    S = np.ones((n,) * nd)
    for a in range(nd):
        sh = [1] * nd
        sh[a] = n
        S = S * np.sin(math.pi * q[a] / L * x).reshape(sh)
    return S


def _standing(n, k, L, c, dt, nsteps, q, chunks=8, discrete=False):
    nd = len(q)
    h = L / (n - 1)
    shape = (n,) * nd
    S = _mode(n, L, q)
    m = np.full(shape, 1.0 / c ** 2)
    eta = np.zeros(shape)
    if discrete:
        w = taylor_weights(k)
        lam = sum((-float(w[0]) - 2 * sum(float(w[j]) * math.cos(j * math.pi * qq / L * h)
                                           for j in range(1, k // 2 + 1))) / h ** 2 for qq in q)
        om_dt = math.acos(1.0 - 0.5 * c * c * dt * dt * lam)
        phase = lambda nn: math.cos(om_dt * nn)
    else:
        om = c * math.sqrt(sum((math.pi * qq / L) ** 2 for qq in q))
        phase = lambda nn: math.cos(om * nn * dt)
    up, u = S * phase(-1), S * phase(0)
    per = nsteps // chunks
    err, done = 0.0, 0
    for _ in range(chunks):
        g = O.Grid(shape, (h,) * nd, (0.0,) * nd, k, dt, per)
        up, u = O.run(g, m, eta, up, u, per, halo="odd")
        done += per
        err = max(err, np.abs(u - S * phase(done)).max() / np.abs(S).max())
    return err


@pytest.mark.parametrize("k,q", [(2, (1, 2)), (4, (2, 1)), (8, (3, 2)), (16, (2, 3)), (4, (1, 2, 1)), (12, (2, 1, 3))])
def test_exact_discrete_standing_wave(k, q):
    """u = prod sin(kappa_a x_a) cos(omega~ n dt), cos(omega~ dt) = 1 - c^2 dt^2 lambda_h / 2,
    is the exact solution of the scheme with odd-reflection ghosts."""
    n = 18 if len(q) == 2 else 14
    L, c = 400.0, 1500.0
    dt = 0.8 * O.cfl_dt((L / (n - 1),) * len(q), k, c)
    nsteps = 240
    err = _standing(n, k, L, c, dt, nsteps, q, chunks=6, discrete=True)
    # FP64 rounding only: at most 2e-15 of the amplitude per step (measured: at most
    # 4.1e-16 per step, k = 16; 1e-13 after the 240 steps)
    assert err < 2e-15 * nsteps


@pytest.mark.parametrize("k,ns", [(2, (9, 13, 17, 25, 33)), (4, (9, 13, 17, 25, 33)), (6, (9, 11, 13, 17)), (8, (9, 11, 13, 15))])
def test_space_convergence_order(k, ns):
    """Error against sin(kx) cos(c|k|t) falls like h^k (400 m box, 150 ms, dt = 0.00625 ms)."""
    ref = GOLDEN["space_convergence"]
    assert k in ref["orders"]
    L, c, T, dt = 400.0, 1500.0, 0.15, 6.25e-6
    nsteps = int(round(T / dt))
    nsteps -= nsteps % 8
    hs, errs = [], []
    for n in ns:
        hs.append(L / (n - 1))
        errs.append(_standing(n, k, L, c, dt, nsteps, (3, 2)))
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert abs(slope - k) < 0.5, (slope, errs)


def test_time_convergence_order():
    """Error falls like dt^2 (paper: slope 1.94, 400 m box, 150 ms)."""
    ref = GOLDEN["time_convergence"]
    L, T = ref["box_m"], ref["t_end_s"]
    n, k, c = 41, 16, 1500.0
    dts = [4e-4, 2e-4, 1e-4, 5e-5]
    errs = [_standing(n, k, L, c, dt, int(round(T / dt)), (3, 2), chunks=1) for dt in dts]
    slope = np.polyfit(np.log(dts), np.log(errs), 1)[0]
    assert abs(slope - 2.0) < 0.1
    assert abs(slope - ref["slope"]) < 0.15


# ---------------------------------------------------------------------------
# (vii) interpolation invariants
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(9, 11), (5, 7, 6)])
def test_interpolation_invariants(shape):
    nd = len(shape)
    h = (10.0, 7.5, 12.0)[:nd]
    o = (-40.0, 3.0, -7.0)[:nd]
    g = O.Grid(shape, h, o, 4, 1e-3, 1)
    rng = np.random.default_rng(5)
    ext = np.array([(shape[a] - 1) * h[a] for a in range(nd)])
    pts = rng.uniform(0, 1, (50, nd)) * ext + np.array(o)
    pts[0] = np.array(o) + ext                     # last node
    idx, w = O.interp(g, pts)
    assert np.allclose(w.sum(axis=1), 1.0, atol=1e-14)
    assert (w >= -1e-15).all()
    # linear fields are reproduced exactly
    coords = np.meshgrid(*[o[a] + h[a] * np.arange(shape[a]) for a in range(nd)], indexing="ij")
    lin = 3.0 + sum((a + 1.5) * coords[a] for a in range(nd))
    vals = (w * lin.ravel()[idx]).sum(axis=1)
    truth = 3.0 + sum((a + 1.5) * pts[:, a] for a in range(nd))
    assert np.allclose(vals, truth, rtol=1e-13, atol=1e-10)
    # on-node points reduce to sampling
    nodes = np.array([[o[a] + h[a] * (shape[a] - 1 - a) for a in range(nd)], [o[a] for a in range(nd)]])
    idx2, w2 = O.interp(g, nodes)
    for i in range(2):
        assert abs(w2[i].max() - 1.0) < 1e-14
    # matches an independent dense construction
    P = dense_interp(shape, h, o, pts)
    Q = np.zeros_like(P)
    for i in range(len(pts)):
        np.add.at(Q[i], idx[i], w[i])
    assert np.abs(P - Q).max() < 1e-14
    with pytest.raises(ValueError):
        O.interp(g, np.array([np.array(o) - 1e-3]))


# ---------------------------------------------------------------------------
# (iii) brute force on tiny grids
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape,k,h", [((6, 7), 4, (10.0, 12.5)), ((5, 4, 6), 2, (9.0, 10.0, 11.0)),
                                        ((7, 6), 8, (10.0, 10.0))])
def test_forward_and_adjoint_equal_dense_operator(shape, k, h):
    model = synth.random_case(shape, k, nsrc=2, nrec=3, nbl=2, seed=11, h=h)
    dt = 0.8 * O.cfl_dt(model.spacing, k, model.vmax)
    nt = 6
    grid = grid_of(model, dt, nt)
    F = dense_F(grid, model.m, model.eta, model.src, model.rec)
    rng = np.random.default_rng(7)
    q = rng.standard_normal((nt, len(model.src)))
    d = O.forward(grid, model.m, model.eta, q, model.src, model.rec)
    ref = (F @ q.ravel()).reshape(nt, -1)
    assert np.abs(d - ref).max() <= 1e-13 * np.abs(ref).max()
    y = rng.standard_normal((nt, len(model.rec)))
    qh = O.adjoint(grid, model.m, model.eta, y, model.rec, model.src)
    ref_a = (F.T @ y.ravel()).reshape(nt, -1)
    assert np.abs(qh - ref_a).max() <= 1e-13 * np.abs(ref_a).max()


# ---------------------------------------------------------------------------
# (iv) dot tests
# ---------------------------------------------------------------------------

def _dot(model, k, nt, seed):
    dt = 0.9 * O.cfl_dt(model.spacing, k, model.vmax)
    grid = grid_of(model, dt, nt, k)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((nt, len(model.src)))
    y = rng.standard_normal((nt, len(model.rec)))
    Fx = O.forward(grid, model.m, model.eta, x, model.src, model.rec)
    Fty = O.adjoint(grid, model.m, model.eta, y, model.rec, model.src)
    a, b = float((Fx * y).sum()), float((x * Fty).sum())
    return abs(a - b) / abs(a)


@pytest.mark.parametrize("k", range(2, 17, 2))
def test_dot_test_2d(k):
    model = synth.random_case((40, 37), k, nsrc=3, nrec=11, nbl=6, seed=k)
    err = _dot(model, k, 60, k)
    paper = GOLDEN["dot_test_2d"]["relative_error"]
    assert err <= 1e-12
    assert err <= 1e3 * max(paper)


@pytest.mark.parametrize("k", range(2, 17, 2))
def test_dot_test_3d(k):
    model = synth.random_case((14, 13, 15), k, nsrc=2, nrec=9, nbl=3, seed=100 + k)
    err = _dot(model, k, 25, k)
    paper = GOLDEN["dot_test_3d"]["relative_error"]
    assert err <= 1e-12
    assert err <= 1e3 * max(paper)


@pytest.mark.parametrize("shape", [(12, 10), (6, 7, 5)])
def test_dot_test_injection_interpolation_alone(shape):
    """With nt = 1 the maps reduce to P_r diag(dt^2/D) P_s^T and its transpose."""
    model = synth.random_case(shape, 4, nsrc=5, nrec=6, nbl=2, seed=21)
    assert _dot(model, 4, 1, 3) <= 1e-14


# ---------------------------------------------------------------------------
# (v) Taylor test, (vi) complex step, checkpointing
# ---------------------------------------------------------------------------

def _fwi_problem(shape=(30, 34), k=8, nt=80, seed=2):
    true = synth.random_case(shape, k, nsrc=1, nrec=12, nbl=5, seed=seed, vmin=1800, vmax=2200)
    rng = np.random.default_rng(seed)
    m0 = true.m * (1.0 + 0.03 * rng.standard_normal(true.shape))
    dt = 0.8 * O.cfl_dt(true.spacing, k, 1.0 / math.sqrt(min(m0.min(), true.m.min())) * 1.06)
    grid = grid_of(true, dt, nt)
    q = synth.ricker(40.0, dt, nt)[:, None]
    d_obs = O.forward(grid, true.m, true.eta, q, true.src, true.rec)
    return true, m0, grid, q, d_obs


def _J(grid, m, eta, q, src, rec, d_obs):
    d = O.forward(grid, m, eta, q, src, rec)
    return 0.5 * float(((d - d_obs) ** 2).sum()), d


def test_taylor_gradient_test():
    ref = GOLDEN["gradient_test"]
    true, m0, grid, q, d_obs = _fwi_problem()
    J0, d0 = _J(grid, m0, true.eta, q, true.src, true.rec, d_obs)
    g = O.gradient(grid, m0, true.eta, q, true.src, d0 - d_obs, true.rec)
    rng = np.random.default_rng(9)
    dm = 0.005 * m0 * rng.standard_normal(m0.shape)
    hs = np.logspace(math.log10(ref["h_range"][0]), math.log10(ref["h_range"][1]), 7)
    e0, e1 = [], []
    gdm = float((g * dm).sum())
    for h in hs:
        Jh, _ = _J(grid, m0 + h * dm, true.eta, q, true.src, true.rec, d_obs)
        e0.append(abs(Jh - J0))
        e1.append(abs(Jh - J0 - h * gdm))
    s0 = np.polyfit(np.log(hs), np.log(e0), 1)[0]
    s1 = np.polyfit(np.log(hs), np.log(e1), 1)[0]
    assert abs(s0 - 1.0) < 0.1 and abs(s0 - ref["slope_eps0"]) < 0.15
    assert abs(s1 - 2.0) < 0.1 and abs(s1 - ref["slope_eps1"]) < 0.15


@pytest.mark.parametrize("shape,k", [((9, 10), 4), ((6, 5, 7), 8)])
def test_gradient_matches_complex_step(shape, k):
    true = synth.random_case(shape, k, nsrc=1, nrec=4, nbl=2, seed=31)
    rng = np.random.default_rng(4)
    m0 = true.m * (1.0 + 0.05 * rng.standard_normal(true.shape))
    dt = 0.8 * O.cfl_dt(true.spacing, k, 1.0 / math.sqrt(m0.min()))
    nt = 14
    grid = grid_of(true, dt, nt)
    q = rng.standard_normal((nt, 1))
    d_obs = rng.standard_normal((nt, len(true.rec))) * 1e-3
    d0 = O.forward(grid, m0, true.eta, q, true.src, true.rec)
    g = O.gradient(grid, m0, true.eta, q, true.src, d0 - d_obs, true.rec)
    gmax = np.abs(g).max()
    eps = 1e-30 * float(m0.mean())
    flat = rng.choice(m0.size, 12, replace=False).tolist() + [0, m0.size - 1]
    for i in flat:
        mc = m0.astype(np.complex128)
        mc.flat[i] += 1j * eps
        dc = O.forward_complex(grid, mc, true.eta, q, true.src, true.rec)
        Jc = 0.5 * ((dc - d_obs) ** 2).sum()
        assert abs(Jc.imag / eps - g.flat[i]) <= 1e-12 * gmax


def test_gradient_independent_of_checkpoint_interval():
    true, m0, grid, q, d_obs = _fwi_problem(shape=(16, 18), k=4, nt=23)
    _, d0 = _J(grid, m0, true.eta, q, true.src, true.rec, d_obs)
    gs = [O.gradient(grid, m0, true.eta, q, true.src, d0 - d_obs, true.rec, checkpoint_every=c)
          for c in (1, 4, 7, 23)]
    for g in gs[1:]:
        assert np.array_equal(g, gs[0])


def test_degenerate_cases():
    model = synth.random_case((8, 9), 4, nsrc=2, nrec=3, nbl=1, seed=1)
    dt = 0.5 * O.cfl_dt(model.spacing, 4, model.vmax)
    g0 = grid_of(model, dt, 0)
    assert O.forward(g0, model.m, model.eta, np.zeros((0, 2)), model.src, model.rec).shape == (0, 3)
    g = grid_of(model, dt, 5)
    d = O.forward(g, model.m, model.eta, np.zeros((5, 0)), np.zeros((0, 2)), model.rec)
    assert np.array_equal(d, np.zeros((5, 3)))
    # grid smaller than the stencil radius: the zero values outside act alone
    tiny = synth.random_case((3, 4), 16, nsrc=1, nrec=2, nbl=0, seed=2)
    dtt = 0.5 * O.cfl_dt(tiny.spacing, 16, tiny.vmax)
    gt = grid_of(tiny, dtt, 4)
    F = dense_F(gt, tiny.m, tiny.eta, tiny.src, tiny.rec)
    q = np.arange(4.0).reshape(4, 1) + 1
    dd = O.forward(gt, tiny.m, tiny.eta, q, tiny.src, tiny.rec)
    assert np.abs(dd.ravel() - F @ q.ravel()).max() <= 1e-13 * np.abs(dd).max()
