"""Inverse design: the overlap objective and its adjoint gradient as a
torch.autograd.Function.  Argument marshalling only: the forward run, the
checkpoints, the recompute and the reverse-time adjoint all run in libfdtd
(fdtd_adjoint_gradient).

A Problem fixes everything but the permittivity of a design box: the grid,
the background eps, a point current source, the output plane k0 with its
mode profile, the number of steps and the objective window.  OverlapLoss
maps the design-box eps (a float64 tensor, (nz, ny, nx) of the box) to
L = sum over the window of (sum m(i,j) Ez(i,j,k0))^2; its backward returns
dL/deps of the box from the adjoint sweep done in the forward call.
"""
import numpy as np
import torch

from . import fdtd
from . import workloads as wl


class Problem:
    def __init__(self, shape_zyx, eps_bg, box_lo, box_hi, source, k0, mode, n_steps, window,
                 checkpoint_every=100, scheme="systolic", dt=wl.DT_DEFAULT):
        self.shape = tuple(int(v) for v in shape_zyx)
        self.eps_bg = np.broadcast_to(np.asarray(eps_bg, np.float64), self.shape).copy()
        self.box_lo, self.box_hi = tuple(box_lo), tuple(box_hi)  # (x, y, z)
        self.source = source  # (component, i, j, k, J)
        self.k0, self.window, self.n_steps = int(k0), int(window), int(n_steps)
        self.mode = torch.as_tensor(np.asarray(mode, np.float32))
        self.checkpoint_every, self.scheme, self.dt = int(checkpoint_every), scheme, float(dt)

    def eps_with(self, eps_box):
        e = self.eps_bg.copy()
        (x0, y0, z0), (x1, y1, z1) = self.box_lo, self.box_hi
        e[z0:z1, y0:y1, x0:x1] = np.asarray(eps_box, np.float64)
        return e

    def run(self, eps_box):
        """(L, dL/deps of the box) for this design."""
        sim = fdtd.Sim(self.shape, self.eps_with(eps_box), self.dt, scheme=self.scheme,
                       max_source_steps=self.n_steps, steps_per_launch=min(self.n_steps, 1024))
        try:
            sim.add_source(*self.source)
            return fdtd.adjoint_gradient(sim, self.k0, self.mode, self.window, self.n_steps, self.box_lo,
                                         self.box_hi, self.checkpoint_every)
        finally:
            sim.close()


class OverlapLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps_box, problem):
        L, grad = problem.run(eps_box.detach().cpu().numpy())
        ctx.save_for_backward(grad.to(eps_box.device))
        return torch.tensor(L, dtype=torch.float64, device=eps_box.device)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None
