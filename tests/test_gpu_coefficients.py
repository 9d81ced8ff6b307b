"""Coefficient setup (A1) checked exactly through one time step.

With u^{-1} = u^0 = 0 the first update is the injection alone: an on-node source
puts b q^0 on its node (weight 1), with b = dt^2 / (m + eta dt/2) rounded once to
float, and a receiver on the same node reads it back.  So every trace sample must
equal float(float(b) * q) with b evaluated in FP64 here, bit for bit, in the
physical domain and in the damping layer (eta > 0).
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


@pytest.mark.parametrize("shape,k", [((30, 34, 38), 8), ((41, 37), 4)])
def test_injection_weight_is_the_correctly_rounded_b(ctx, shape, k):
    case = synth.random_case(shape, k, nsrc=1, nrec=1, nbl=6, seed=13, vmin=1500, vmax=4500)
    m, e = case.m32(), case.eta32()
    assert (e > 0).any() and (e == 0).any()
    rng = np.random.default_rng(21)
    flat = rng.choice(int(np.prod(shape)), size=160, replace=False)
    idx = np.stack(np.unravel_index(flat, shape), axis=1)
    coords = np.asarray(case.origin) + idx * np.asarray(case.spacing)   # on nodes, exact in binary
    dt = 0.9 * O.cfl_dt(case.spacing, k, case.vmax)
    grid = W.Grid(shape, case.spacing, case.origin, k, dt, 1)
    q = rng.uniform(0.5, 2.0, size=(1, len(coords))).astype(np.float32)
    d = W.wp_forward(ctx.handle, grid, m, e, q, coords, coords)
    mm = m[tuple(idx.T)].astype(np.float64)
    ee = e[tuple(idx.T)].astype(np.float64)
    b = (dt * dt / (mm + ee * dt * 0.5)).astype(np.float32)
    expect = (b * q[0]).astype(np.float32)
    assert np.array_equal(d[0], expect)
