"""Failure detection on the GPU without a GPU fault.

- Device side: every wait inside the stencil kernels (TMA copies landing, ring
  slots freed) is bounded.  A context's wait limit set to 0 makes each kernel's
  first work item start with a wait on a barrier that nothing completes, which
  gives up at once; the kernel then skips its stores, lets its own copies land
  and reports through the context's error word, and the call returns WP_EDEVICE.
  The same context, with the limit restored, and a fresh context still compute
  the right answer.
- Host side: a context deadline shorter than the call makes it return
  WP_ETIMEOUT while its kernels are still running; the context then refuses
  further calls, and a fresh context computes the right answer once the device
  has drained.
- Device-array calls refuse host pointers and buffers of the wrong size before
  anything is launched.
Nothing here faults, traps or hangs the GPU: every wait ends by its limit and
the queued kernels always complete.
"""
import numpy as np
import pytest

import oracle as O
from paper_1808_01995_gb300 import synth
from paper_1808_01995_gb300 import wavprop as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_01995_gb300 import build
    build.build()


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def case(shape, k, nt, seed):
    model = synth.random_case(shape, k, nsrc=2, nrec=24, nbl=4, seed=seed)
    dt = 0.9 * O.cfl_dt(model.spacing, k, model.vmax)
    og = O.Grid(model.shape, model.spacing, model.origin, k, dt, nt)
    wg = W.Grid(model.shape, model.spacing, model.origin, k, dt, nt)
    q = model.wavelet(dt, nt)
    return model, og, wg, q


def run_dev(h, wg, model, q):
    out = torch.zeros((wg.nt, len(model.rec)), device="cuda")
    W.wp_forward_dev(h, wg, torch.from_numpy(model.m32()).cuda(), torch.from_numpy(model.eta32()).cuda(),
                     torch.from_numpy(q).cuda(), model.src, model.rec, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("k", [8, 16])
def test_wait_limit_zero_reports_edevice_and_context_recovers(k):
    model, og, wg, q = case((40, 45, 70), k, 40, seed=30 + k)
    ref = O.forward(og, model.m32(), model.eta32(), q, model.src, model.rec)
    with W.Context(0) as c:
        good = run_dev(c.handle, wg, model, q)
        assert rel_l2(good, ref) < 1e-4
        W.wp_set_wait_limit(c.handle, 0.0)
        with pytest.raises(W.WpError) as e:
            run_dev(c.handle, wg, model, q)
        assert e.value.status == W.WP_EDEVICE
        assert "device error" in str(e.value)
        # the same context, limit restored: bit-identical to the run before
        W.wp_set_wait_limit(c.handle, 2.0)
        assert np.array_equal(run_dev(c.handle, wg, model, q), good)
    with W.Context(0) as c2:
        assert np.array_equal(run_dev(c2.handle, wg, model, q), good)


def test_wait_limit_is_validated():
    with W.Context(0) as c:
        for bad in (-1.0, float("nan"), 61.0):
            with pytest.raises(W.WpError) as e:
                W.wp_set_wait_limit(c.handle, bad)
            assert e.value.status == W.WP_EINVAL


def test_host_deadline_reports_etimeout_and_a_fresh_context_works():
    # a 3D forward of about a second of device work against a 1 ms deadline
    model = synth.layers_3d(space_order=8, n=176, nt=1)
    k, nt = 8, 3000
    dt = 0.9 * W.wp_cfl_dt(W.Grid(model.shape, model.spacing, model.origin, k), model.vmax)
    wg = W.Grid(model.shape, model.spacing, model.origin, k, dt, nt)
    m = torch.from_numpy(model.m32()).cuda()
    eta = torch.from_numpy(model.eta32()).cuda()
    q = torch.from_numpy(model.wavelet(dt, nt)).cuda()
    out = torch.zeros((nt, len(model.rec)), device="cuda")
    c = W.Context(0)
    try:
        W.wp_set_timeout(c.handle, 1e-3)
        with pytest.raises(W.WpError) as e:
            W.wp_forward_dev(c.handle, wg, m, eta, q, model.src, model.rec, out)
        assert e.value.status == W.WP_ETIMEOUT
        # the timed-out context refuses further work
        with pytest.raises(W.WpError) as e2:
            W.wp_forward_dev(c.handle, wg, m, eta, q, model.src, model.rec, out)
        assert e2.value.status == W.WP_ETIMEOUT
    finally:
        # its kernels are still queued and write `out`: let the device drain first
        torch.cuda.synchronize()
        c.close()
        torch.cuda.synchronize()
    # a fresh context on the same device computes the shot; a short run is checked
    # against the oracle (the 3000-step run only for completing)
    with W.Context(0) as c2:
        W.wp_forward_dev(c2.handle, wg, m, eta, q, model.src, model.rec, out)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        small, og, sg, sq = case((30, 33, 36), 8, 25, seed=5)
        ref = O.forward(og, small.m32(), small.eta32(), sq, small.src, small.rec)
        assert rel_l2(run_dev(c2.handle, sg, small, sq), ref) < 1e-4


def test_device_calls_refuse_host_and_short_buffers():
    model, og, wg, q = case((20, 21, 22), 4, 10, seed=3)
    m = torch.from_numpy(model.m32()).cuda()
    eta = torch.from_numpy(model.eta32()).cuda()
    qd = torch.from_numpy(q).cuda()
    with W.Context(0) as c:
        out = torch.zeros((wg.nt, len(model.rec)), device="cuda")
        launches = W.wp_kernel_launches(c.handle)
        # wrong sizes and host tensors are refused by the binding
        with pytest.raises(ValueError):
            W.wp_forward_dev(c.handle, wg, m, eta, qd, model.src, model.rec, out[:-1])
        with pytest.raises(ValueError):
            W.wp_forward_dev(c.handle, wg, m[:-1], eta, qd, model.src, model.rec, out)
        with pytest.raises(TypeError):
            W.wp_forward_dev(c.handle, wg, m, eta, torch.from_numpy(q), model.src, model.rec, out)
        # a host pointer handed straight to the C ABI is refused by the library
        import ctypes
        g = wg.c()
        qh = np.ascontiguousarray(q, np.float32)
        src = np.ascontiguousarray(model.src, np.float64)
        rec = np.ascontiguousarray(model.rec, np.float64)
        rc = W.lib().wp_forward_dev(c.handle, ctypes.byref(g), m.data_ptr(), eta.data_ptr(), qh.ctypes.data,
                                    len(src), src.ctypes.data, len(rec), rec.ctypes.data, out.data_ptr(), None)
        assert rc == W.WP_EINVAL
        assert "host pointer" in W.wp_last_error()
        rc = W.lib().wp_forward_noalloc(ctypes.byref(g), m.data_ptr(), eta.data_ptr(), qh.ctypes.data, len(src),
                                        src.ctypes.data, len(rec), rec.ctypes.data, out.data_ptr(), None)
        assert rc == W.WP_EINVAL
        assert W.wp_kernel_launches(c.handle) == launches  # nothing was launched
        # and the context still works
        ref = O.forward(og, model.m32(), model.eta32(), q, model.src, model.rec)
        W.wp_forward_dev(c.handle, wg, m, eta, qd, model.src, model.rec, out)
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), ref) < 1e-4


def test_state_outliving_its_context_is_detached():
    # a forward state kept (e.g. by an autograd graph held in a traceback) after
    # its context is destroyed: the context releases the state's memory, backward
    # on it is refused, and freeing it afterwards touches nothing of the context
    model, og, wg, q = case((20, 22, 24), 4, 12, seed=4)
    m = torch.from_numpy(model.m32()).cuda()
    eta = torch.from_numpy(model.eta32()).cuda()
    qd = torch.from_numpy(q).cuda()
    d = torch.zeros((wg.nt, len(model.rec)), device="cuda")
    c = W.Context(0)
    st = W.wp_forward_save(c.handle, wg, m, eta, qd, model.src, model.rec, 4, d)
    g = torch.zeros_like(m)
    W.wp_backward(st, d, g)
    c.close()
    with pytest.raises(W.WpError) as e:
        W.wp_backward(st, d, g)
    assert e.value.status == W.WP_EINVAL
    W.wp_state_free(st)
    # a new context still works
    with W.Context(0) as c2:
        ref = O.forward(og, model.m32(), model.eta32(), q, model.src, model.rec)
        assert rel_l2(run_dev(c2.handle, wg, model, q), ref) < 1e-4
