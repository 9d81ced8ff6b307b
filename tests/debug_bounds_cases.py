"""Small propagator cases run in a child process by test_gpu_debug_bounds.py.

Usage: python debug_bounds_cases.py OUT.npz  (the library is the one WAVPROP_LIB
names, or the in-tree build).  Each case's result goes into OUT.npz under its
name; a case that raises stores its status and message instead.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_1808_01995_gb300 import synth  # noqa: E402
from paper_1808_01995_gb300 import wavprop as W  # noqa: E402


def cfl(model, k):
    return 0.9 * W.wp_cfl_dt(W.Grid(model.shape, model.spacing, model.origin, k), model.vmax)


def cases():
    # ragged 3D grids, sources and receivers on the first and last nodes, all the
    # order families, a 2D grid, the gradient paths and the no-allocation call
    for shape, k, nt in [((23, 37, 45), 4, 24), ((30, 41, 70), 8, 24), ((21, 18, 35), 16, 16), ((47, 66), 4, 30)]:
        model = synth.random_case(shape, k, nsrc=3, nrec=20, nbl=4, seed=k + len(shape))
        dt = cfl(model, k)
        grid = W.Grid(model.shape, model.spacing, model.origin, k, dt, nt)
        q = model.wavelet(dt, nt)
        tag = f"{'x'.join(map(str, shape))}_so{k}"
        yield f"forward_{tag}", lambda c, g=grid, mo=model, q=q: W.wp_forward(c, g, mo.m32(), mo.eta32(), q, mo.src,
                                                                              mo.rec)
        rng = np.random.default_rng(k)
        d = rng.standard_normal((nt, len(model.rec))).astype(np.float32)
        yield f"adjoint_{tag}", lambda c, g=grid, mo=model, d=d: W.wp_adjoint(c, g, mo.m32(), mo.eta32(), d, mo.rec,
                                                                              mo.src)
        yield f"gradient_{tag}", lambda c, g=grid, mo=model, q=q, d=d: W.wp_gradient(c, g, mo.m32(), mo.eta32(), q,
                                                                                     mo.src, d, mo.rec, 5)
    model = synth.random_case((28, 30, 34), 8, nsrc=2, nrec=12, nbl=5, seed=7)
    dt = cfl(model, 8)
    grid = W.Grid(model.shape, model.spacing, model.origin, 8, dt, 20)
    q = model.wavelet(dt, 20)
    d = np.random.default_rng(3).standard_normal((20, 12)).astype(np.float32)
    yield "checkpointed_so8", lambda c: W.wp_gradient_checkpointed(c, grid, model.m32(), model.eta32(), q, model.src,
                                                                    d, model.rec, 3)

    def noalloc(c):
        out = torch.zeros((20, 12), device="cuda")
        W.wp_forward_noalloc(grid, torch.from_numpy(model.m32()).cuda(), torch.from_numpy(model.eta32()).cuda(),
                             torch.from_numpy(q).cuda(), model.src, model.rec, out)
        torch.cuda.synchronize()
        return out.cpu().numpy()
    yield "noalloc_so8", noalloc


def main(out_path):
    res = {}
    with W.Context(0) as ctx:
        for name, fn in cases():
            try:
                res[name] = np.asarray(fn(ctx.handle))
            except W.WpError as e:
                res[name + "__error"] = np.array([e.status])
                res[name + "__message"] = np.array([str(e)])
    np.savez(out_path, **res)


if __name__ == "__main__":
    main(sys.argv[1])
