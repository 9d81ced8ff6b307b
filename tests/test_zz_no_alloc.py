"""wp_forward_noalloc: the forward call for callers that cannot allocate device
memory (their host application owns every device byte and forbids cudaMalloc /
cudaFree from libraries).  Its output must match wp_forward_dev's within the
receiver-data tolerance of the parity tests, on two calls in a row (the second
call reuses the fixed work space the first one left behind).  This file is
collected last so that a run stopping at the first failure has run every other
test first."""
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


@pytest.mark.parametrize("shape,k,nt", [((40, 45, 70), 8, 60), ((47, 66), 4, 80), ((21, 18, 35), 16, 30)])
def test_noalloc_matches_forward_dev_on_two_calls_in_a_row(ctx, shape, k, nt):
    model = synth.random_case(shape, k, nsrc=2, nrec=30, nbl=5, seed=k + len(shape))
    dt = 0.9 * O.cfl_dt(model.spacing, k, model.vmax)
    grid = W.Grid(model.shape, model.spacing, model.origin, k, dt, nt)
    m = torch.from_numpy(model.m32()).cuda()
    eta = torch.from_numpy(model.eta32()).cuda()
    q = torch.from_numpy(model.wavelet(dt, nt)).cuda()
    ref = torch.zeros((nt, 30), device="cuda")
    W.wp_forward_dev(ctx, grid, m, eta, q, model.src, model.rec, ref)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    for _ in range(2):
        out = torch.full((nt, 30), float("nan"), device="cuda")
        W.wp_forward_noalloc(grid, m, eta, q, model.src, model.rec, out)
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), ref) < 1e-4


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
