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
    # the GPU steps with c = fl32(dt/eps); the oracle takes the same
    # coefficients (quantize=True), so what remains is FP32 arithmetic
    obj = adj.Objective(p.k0, p.mode.numpy().astype(np.float64), p.window)
    c, i, j, k, J = p.source
    f0 = np.zeros((6,) + p.shape)
    L, g = adj.gradient(p.shape, p.eps_with(eps_box), f0, p.n_steps, [(c, i, j, k, J)], obj, DT, quantize=True)
    (x0, y0, z0), (x1, y1, z1) = p.box_lo, p.box_hi
    return L, g[z0:z1, y0:y1, x0:x1]


# FP32 bound of the gradient: forward state and adjoint state each carry a
# rounding error that grows at most linearly in the steps (the Yee map and
# its transpose do not amplify: energy-norm stable), u32 = 2^-24 per
# operation, ~10 operations per value and step, so after N = 80 steps each
# is within ~N * 10 * u32 = 4.8e-5 of its FP64 value relative to its size,
# and the gradient (their products summed in FP64) within ~1e-4 of it.
GRAD_TOL = 1e-4


@pytest.mark.parametrize("scheme,K", [("systolic", 20), ("naive", 7), ("systolic", 80)])
def test_gradient_matches_oracle_adjoint(cuda_device, scheme, K):
    p, eps_box = small_problem(scheme, K)
    L, g = p.run(eps_box)
    Lo, go = oracle_grad(p, eps_box)
    g = g.cpu().numpy()
    rel = np.linalg.norm(g - go) / np.linalg.norm(go)
    print(f"{scheme} K={K}: |L-Lo|/Lo = {abs(L - Lo) / Lo:.2e}, gradient rel-L2 = {rel:.2e}")
    assert abs(L - Lo) <= 1e-4 * Lo
    assert rel <= GRAD_TOL, rel


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
    # central differences of the FP64 oracle on 16 seeded random voxels of
    # the box (distinct, drawn from the splitmix64 stream of the inputs)
    obj = adj.Objective(p.k0, p.mode.numpy().astype(np.float64), p.window)
    c, i, j, k, J = p.source
    f0 = np.zeros((6,) + p.shape)
    n_box = eps_box.size
    order = np.argsort(wl.splitmix64(17, 0, n_box))
    voxels = [np.unravel_index(int(v), eps_box.shape) for v in order[:16]]
    assert len(set(voxels)) == 16
    worst = 0.0
    eps64 = np.asarray(eps_box, np.float64)  # perturb in FP64 (a float32 step would be rounded)
    for q in voxels:
        q = tuple(int(v) for v in q)
        h = 1e-5 * eps64[q]  # truncation error ~(h/eps)^2 stays far below the tolerance
        ep, em = eps64.copy(), eps64.copy()
        ep[q] += h
        em[q] -= h
        fd = (adj.objective(p.shape, p.eps_with(ep), f0, p.n_steps, [(c, i, j, k, J)], obj, DT) -
              adj.objective(p.shape, p.eps_with(em), f0, p.n_steps, [(c, i, j, k, J)], obj, DT)) / (2 * h)
        got = float(g_direct[q])
        scale = max(abs(fd), 1e-2 * float(g_direct.abs().max()))
        worst = max(worst, abs(got - fd) / scale)
        assert abs(got - fd) <= 1e-3 * scale, (q, got, fd)
    print(f"16 voxels: largest |adjoint - central difference| / scale = {worst:.2e}")


def test_midsize_gradient_16_voxels_central_differences(cuda_device):
    """A mid-size problem (64 x 64 x 48 cells, 1000 steps, checkpoints every
    100, a 16 x 16 x 8 design box): the GPU gradient on 16 seeded random
    voxels of the box against central differences of the FP64 oracle's
    objective (eps perturbed by 1e-5 relative, in FP64)."""
    nz, ny, nx = 48, 64, 64
    steps = 1000
    lo, hi = (24, 24, 16), (40, 40, 24)       # x, y, z
    bg = np.full((nz, ny, nx), 2.1)
    u = np.asarray(wl.uniform_pm1(31, 16 * 16 * 8), np.float64).reshape(8, 16, 16)
    eps_box = 2.1 + 10.0 * (0.5 + 0.5 * u)
    mode = np.asarray(wl.uniform_pm1(32, ny * nx)).reshape(ny, nx)
    src = (2, 32, 32, 10, wl.sine_source(steps, DT, 20.0))
    p = gadj.Problem((nz, ny, nx), bg, lo, hi, src, k0=32, mode=mode, n_steps=steps, window=150,
                     checkpoint_every=100, scheme="systolic")
    L, g = p.run(eps_box)
    g = g.cpu().numpy()
    obj = adj.Objective(p.k0, p.mode.numpy().astype(np.float64), p.window)
    c, i, j, k, J = p.source
    f0 = np.zeros((6, nz, ny, nx))
    Lo = adj.objective_window(p.shape, p.eps_with(eps_box), f0, steps, [(c, i, j, k, J)], obj, DT, quantize=True)
    assert abs(L - Lo) <= 1e-4 * Lo, (L, Lo)
    order = np.argsort(wl.splitmix64(33, 0, eps_box.size))
    worst = 0.0
    for v in order[:16]:
        q = tuple(int(t) for t in np.unravel_index(int(v), eps_box.shape))
        h = 1e-5 * eps_box[q]
        ep, em = eps_box.copy(), eps_box.copy()
        ep[q] += h
        em[q] -= h
        fd = (adj.objective_window(p.shape, p.eps_with(ep), f0, steps, [(c, i, j, k, J)], obj, DT) -
              adj.objective_window(p.shape, p.eps_with(em), f0, steps, [(c, i, j, k, J)], obj, DT)) / (2 * h)
        scale = max(abs(fd), 1e-2 * float(np.abs(g).max()))
        worst = max(worst, abs(g[q] - fd) / scale)
        assert abs(g[q] - fd) <= 1e-3 * scale, (q, g[q], fd)
    print(f"mid-size, 16 voxels: largest |adjoint - central difference| / scale = {worst:.2e}")
