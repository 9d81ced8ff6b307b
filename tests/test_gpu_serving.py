"""Shot server on the GPU: each result is the same alone and in the mix, work of
concurrent slots overlaps, and faulty requests fail alone."""
import math

import numpy as np
import pytest

from paper_1808_01995_gb300 import serving as S
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


def specs(n=8):
    return synth.serving_requests(count=n, seed=77, size_scale=0.3)


def test_results_are_the_same_alone_and_in_the_mix(ctx):
    sp = specs(8)
    alone = []
    for spec in sp:
        r = S.make_request(spec)
        alone.append(S.run_request(ctx.handle, r))
    mix = [S.make_request(spec) for spec in sp]
    srv = S.ShotServer(slots=4, hbm_budget_bytes=16 << 30)
    try:
        for r in mix:
            srv.submit(r)
        assert srv.drain(600)
    finally:
        srv.close()
    kinds = set()
    for (res, J), r in zip(alone, mix):
        assert r.status == "done", r.error
        kinds.add(r.kind)
        assert rel_l2(r.result, res) <= 1e-6
        if r.kind == "gradient":
            assert abs(r.misfit - J) <= 1e-9 * abs(J)
    assert kinds == {"forward", "gradient"}
    # the slots really ran side by side
    spans = sorted((r.t_admit, r.t_done) for r in mix)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))


def test_faulty_requests_fail_alone(ctx):
    sp = specs(4)
    good = [S.make_request(s) for s in sp[:3]]
    nan_req = S.make_request(sp[3], ident=100)
    nan_req.m = nan_req.m.copy()
    nan_req.m.flat[5] = np.nan
    cfl_req = S.make_request(sp[0], ident=101)
    cfl_req.grid = W.Grid(cfl_req.grid.shape, cfl_req.grid.spacing, cfl_req.grid.origin,
                          cfl_req.grid.space_order, cfl_req.grid.dt * 3.0, cfl_req.grid.nt)
    expected = [S.run_request(ctx.handle, S.make_request(s)) for s in sp[:3]]
    srv = S.ShotServer(slots=3, hbm_budget_bytes=16 << 30)
    try:
        for r in [nan_req] + good + [cfl_req]:
            srv.submit(r)
        assert srv.drain(600)
    finally:
        srv.close()
    assert nan_req.status == "error" and nan_req.error_status == W.WP_ENONFINITE
    assert cfl_req.status == "error" and cfl_req.error_status == W.WP_ECFL
    for r, (res, _) in zip(good, expected):
        assert r.status == "done"
        assert rel_l2(r.result, res) <= 1e-6


def test_small_budget_is_respected(ctx):
    sp = specs(6)
    reqs = [S.make_request(s) for s in sp]
    est = [S.estimate_bytes(r) for r in reqs]
    budget = int(2.2 * max(est))
    srv = S.ShotServer(slots=4, hbm_budget_bytes=budget)
    try:
        for r in reqs:
            srv.submit(r)
        assert srv.drain(600)
    finally:
        srv.close()
    assert all(r.status == "done" for r in reqs), [r.error for r in reqs]
    assert srv.peak_reserved <= budget
