"""Adjoint gradient on the GPU, through the C ABI: against the FP64 oracle's
adjoint and its central finite differences, across schedules and
checkpoint intervals, and through torch.autograd."""
import numpy as np
import pytest
import torch

from oracle import adjoint as adj
from paper_2502_20610_gb300 import adjoint as gadj
from paper_2502_20610_gb300 import fdtd
from paper_2502_20610_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DT = wl.DT_DEFAULT


def small_problem(scheme="systolic", K=20, steps=80):
    shape = (24, 22, 26)                       # nz, ny, nx
    lo, hi = (9, 7, 8), (17, 15, 14)           # x, y, z: an 8 x 8 x 6 design box
    bg = np.full(shape, 2.1)
    rng_eps = 2.1 + 10.0 * (0.5 + 0.5 * np.asarray(wl.uniform_pm1(3, 8 * 8 * 6)).reshape(6, 8, 8))
    mode = np.asarray(wl.uniform_pm1(4, 22 * 26)).reshape(22, 26)
    src = (2, 13, 11, 4, wl.sine_source(steps, DT, 10.0))
    p = gadj.Problem(shape, bg, lo, hi, src, k0=20, mode=mode, n_steps=steps, window=30, checkpoint_every=K,
                     scheme=scheme)
    return p, rng_eps


def oracle_grad(p, eps_box):
    obj = adj.Objective(p.k0, p.mode.numpy().astype(np.float64), p.window)
    c, i, j, k, J = p.source
    f0 = np.zeros((6,) + p.shape)
    L, g = adj.gradient(p.shape, p.eps_with(eps_box), f0, p.n_steps, [(c, i, j, k, J)], obj, DT)
    (x0, y0, z0), (x1, y1, z1) = p.box_lo, p.box_hi
    return L, g[z0:z1, y0:y1, x0:x1]


@pytest.mark.parametrize("scheme,K", [("systolic", 20), ("naive", 7), ("systolic", 80)])
def test_gradient_matches_oracle_adjoint(cuda_device, scheme, K):
    p, eps_box = small_problem(scheme, K)
    L, g = p.run(eps_box)
    Lo, go = oracle_grad(p, eps_box)
    g = g.cpu().numpy()
    assert abs(L - Lo) <= 1e-4 * Lo
    assert np.linalg.norm(g - go) <= 2e-3 * np.linalg.norm(go), np.linalg.norm(g - go) / np.linalg.norm(go)


def test_gradient_is_independent_of_checkpoint_interval(cuda_device):
    # recompute is deterministic and both schedules are bit-identical
    p1, eps_box = small_problem("systolic", 1)
    p2, _ = small_problem("naive", 33)
    L1, g1 = p1.run(eps_box)
    L2, g2 = p2.run(eps_box)
    assert L1 == L2 and torch.equal(g1, g2)


def test_autograd_and_finite_differences(cuda_device):
    p, eps_box = small_problem("systolic", 25)
    x = torch.tensor(eps_box, dtype=torch.float64, requires_grad=True)
    L = gadj.OverlapLoss.apply(x, p)
    (g,) = torch.autograd.grad(3.0 * L, x)
    _, g_direct = p.run(eps_box)
    assert torch.allclose(g, 3.0 * g_direct.cpu(), rtol=0, atol=0)
    # central differences of the FP64 oracle on voxels of the box
    obj = adj.Objective(p.k0, p.mode.numpy().astype(np.float64), p.window)
    c, i, j, k, J = p.source
    f0 = np.zeros((6,) + p.shape)
    rng = np.random.default_rng(5)
    for _ in range(4):
        q = tuple(int(rng.integers(0, s)) for s in eps_box.shape)
        h = 1e-4 * eps_box[q]
        ep, em = eps_box.copy(), eps_box.copy()
        ep[q] += h
        em[q] -= h
        fd = (adj.objective(p.shape, p.eps_with(ep), f0, p.n_steps, [(c, i, j, k, J)], obj, DT) -
              adj.objective(p.shape, p.eps_with(em), f0, p.n_steps, [(c, i, j, k, J)], obj, DT)) / (2 * h)
        got = float(g_direct[q])
        assert abs(got - fd) <= 5e-3 * max(abs(fd), 1e-2 * float(g_direct.abs().max())), (q, got, fd)
