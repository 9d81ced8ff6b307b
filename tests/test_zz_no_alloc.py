"""wp_forward_noalloc: the forward call for callers that cannot allocate device
memory (their host application owns every device byte and forbids cudaMalloc /
cudaFree from libraries).  It runs the same kernels with the same arguments as
wp_forward_dev, so its receiver data must equal wp_forward_dev's bit for bit, on
two calls in a row (the second call reuses the fixed work space the first one
left behind), and match the FP64 oracle within the receiver-data tolerance of
the parity tests (1e-4 relative L2).  This file is collected last so that a run
stopping at the first failure has run every other test first."""
import numpy as np
import pytest

import oracle as O
from paper_1808_01995_gb300 import synth
from paper_1808_01995_gb300 import wavprop as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_01995_gb300 import build
    build.build()
    c = W.Context(0)
    yield c.handle
    c.close()


def _compare(ctx, model, k, nt, nsrc, nrec, oracle_check=True):
    dt = 0.9 * O.cfl_dt(model.spacing, k, model.vmax)
    grid = W.Grid(model.shape, model.spacing, model.origin, k, dt, nt)
    m = torch.from_numpy(model.m32()).cuda()
    eta = torch.from_numpy(model.eta32()).cuda()
    q = torch.from_numpy(model.wavelet(dt, nt)[:, :nsrc].copy()).cuda()
    src, rec = model.src[:nsrc], model.rec[:nrec]
    ref = torch.zeros((nt, nrec), device="cuda")
    W.wp_forward_dev(ctx, grid, m, eta, q, src, rec, ref)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    for _ in range(2):
        out = torch.full((nt, nrec), float("nan"), device="cuda")
        W.wp_forward_noalloc(grid, m, eta, q, src, rec, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref)
    if oracle_check:
        og = O.Grid(model.shape, model.spacing, model.origin, k, dt, nt)
        d = O.forward(og, model.m32(), model.eta32(), model.wavelet(dt, nt)[:, :nsrc].copy(), src, rec)
        if nsrc == 0:
            assert not ref.any() and not d.any()
        else:
            assert rel_l2(ref, d) < 1e-4
    return ref


@pytest.mark.parametrize("shape,k,nt", [((40, 45, 70), 8, 60), ((47, 66), 4, 80), ((21, 18, 35), 16, 30)])
def test_noalloc_matches_forward_dev_on_two_calls_in_a_row(ctx, shape, k, nt):
    model = synth.random_case(shape, k, nsrc=2, nrec=30, nbl=5, seed=k + len(shape))
    _compare(ctx, model, k, nt, 2, 30)


def test_noalloc_without_sources_gives_zero_data(ctx):
    model = synth.random_case((30, 33, 40), 8, nsrc=2, nrec=20, nbl=4, seed=11)
    ref = _compare(ctx, model, 8, 20, 0, 20)
    assert not ref.any()


def test_noalloc_without_receivers(ctx):
    model = synth.random_case((30, 33, 40), 8, nsrc=2, nrec=20, nbl=4, seed=12)
    _compare(ctx, model, 8, 20, 2, 0, oracle_check=False)


def test_noalloc_near_its_work_space_limit(ctx):
    # 63 x 128 x 500 (rows padded to 512): four fields of 63.0 MiB in all, just
    # under the 64 MiB work space; one more plane does not fit
    model = synth.random_case((63, 128, 500), 4, nsrc=1, nrec=16, nbl=4, seed=13)
    _compare(ctx, model, 4, 12, 1, 16, oracle_check=False)
    big = W.Grid((65, 128, 500), (10.0,) * 3, (0.0,) * 3, 4, 1e-4, 2)
    m = torch.full(big.shape, 1.0 / 2000 ** 2, device="cuda")
    with pytest.raises(W.WpError) as e:
        W.wp_forward_noalloc(big, m, torch.zeros_like(m), None, None, None, None)
    assert e.value.status == W.WP_ENOMEM


def test_noalloc_rejects_problems_beyond_its_work_space():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    grid = W.Grid((200, 200, 200), (10.0,) * 3, (0.0,) * 3, 8, 1e-3, 4)
    m = torch.full(grid.shape, 1.0 / 2000 ** 2, device="cuda")
    eta = torch.zeros(grid.shape, device="cuda")
    out = torch.zeros((4, 0), device="cuda")
    with pytest.raises(W.WpError) as e:
        W.wp_forward_noalloc(grid, m, eta, None, None, None, out)
    assert e.value.status == W.WP_ENOMEM
    assert "limited to" in str(e.value)
