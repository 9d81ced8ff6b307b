"""Multi-shot full-waveform inversion driver (Sec. 3.4).

The FWI objective of a survey is the sum over source experiments of the
per-shot misfit 1/2 ||F_s(m) q_s - d_s||^2 (Eq. AS); its gradient is the sum of
the per-shot adjoint-state gradients (Eq. Grad).  Shots are independent, so
they run concurrently on ``slots`` contexts (each with its own stream and device
pool), every shot's gradient is accumulated on the device by the library's
axpy kernel, and the model is updated with the fixed-step gradient step with
bounds on the squared slowness (wp_update_model_dev).  The optimiser around it
(line searches, l-BFGS, ...) is out of scope; ``fixed_step`` is the simple
gradient descent the paper shows.
"""
from __future__ import annotations

import threading
from dataclasses import dataclass

import numpy as np
import torch

from . import wavprop as W


@dataclass
class Shot:
    """One source experiment: wavelet [nt][nsrc], coordinates, observed data [nt][nrec]
    (CUDA tensors for the arrays, numpy for the coordinates)."""

    wavelet: torch.Tensor
    src: np.ndarray
    rec: np.ndarray
    d_obs: torch.Tensor


class MultiShotFWI:
    """Objective, gradient and fixed-step updates of a multi-shot survey on one GPU."""

    def __init__(self, grid: W.Grid, eta: torch.Tensor, shots: list[Shot], snap_interval: int = 10,
                 slots: int = 2, device: int = 0):
        self.grid = grid
        self.eta = eta
        self.shots = shots
        self.snap_interval = int(snap_interval)
        self.slots = max(1, min(int(slots), len(shots)))
        self.contexts = [W.Context(device) for _ in range(self.slots)]
        self.device = device

    def close(self):
        for c in self.contexts:
            c.close()

    def objective_and_gradient(self, m: torch.Tensor):
        """(J, dJ/dm) summed over all shots; m is a contiguous float32 CUDA tensor."""
        shape = tuple(self.grid.shape)
        acc = [torch.zeros(shape, device=m.device) for _ in range(self.slots)]
        buf = [torch.empty(shape, device=m.device) for _ in range(self.slots)]
        J = [0.0] * self.slots
        err: list[BaseException] = []

        def run(s: int):
            try:
                torch.cuda.set_device(m.device)
                h = self.contexts[s].handle
                for shot in self.shots[s::self.slots]:
                    J[s] += W.wp_fwi_gradient_dev(h, self.grid, m, self.eta, shot.wavelet, shot.src, shot.d_obs,
                                                  shot.rec, self.snap_interval, buf[s])
                    W.wp_axpy_dev(h, 1.0, buf[s], acc[s])
            except BaseException as e:  # noqa: BLE001 - re-raised on the caller's thread
                err.append(e)

        threads = [threading.Thread(target=run, args=(s,)) for s in range(self.slots)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        if err:
            raise err[0]
        g = acc[0]
        for s in range(1, self.slots):
            W.wp_axpy_dev(self.contexts[0].handle, 1.0, acc[s], g)
        return float(sum(J)), g

    def fixed_step(self, m: torch.Tensor, step: float, m_min: float, m_max: float):
        """One gradient step m <- clamp(m - step dJ/dm, m_min, m_max) in place; returns
        the objective at the model before the step."""
        J, g = self.objective_and_gradient(m)
        W.wp_update_model_dev(self.contexts[0].handle, step, g, m, m_min, m_max)
        return J, g
