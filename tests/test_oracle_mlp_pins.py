"""Pins of the FP64 reference network and learned-boundary step (oracle/mlp.py).

* The hand-written backward pass against central finite differences of the
  loss (an independent derivative).
* Closed forms: with zero weights f = b3 and dL/db3 = 2 (b3 - mean y) / 6;
  with tanh and W2 = W3 = 0 the network ignores its input.
* The stencil layout puts a single non-zero field value where the layout
  says, and the centre at c*27 + 13.
* The scale-equivariant correction is homogeneous of degree 1.
* A network whose output is zero leaves the plain PEC box (the Yee oracle),
  and so does a layer of thickness 0.
"""
import numpy as np

from oracle import YeeOracle
from oracle import mlp
from paper_2502_20610_gb300 import workloads as wl

DT = wl.DT_DEFAULT


def test_backward_matches_central_differences():
    rng = np.random.default_rng(1)
    theta = mlp.init_params(2)
    x = rng.standard_normal((7, mlp.N_IN))
    y = rng.standard_normal((7, mlp.N_OUT))
    g = mlp.grad(theta, x, y)
    idx = np.concatenate([rng.choice(mlp.N_PARAMS, 60, replace=False),
                          np.arange(mlp.N_PARAMS - 6, mlp.N_PARAMS)])  # includes every b3
    h = 1e-6
    for q in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[q] += h
        tm[q] -= h
        fd = (mlp.loss(tp, x, y) - mlp.loss(tm, x, y)) / (2 * h)
        assert abs(fd - g[q]) <= 1e-7 * max(1.0, abs(fd)) + 1e-9, (q, fd, g[q])


def test_zero_weights_closed_form():
    theta = np.zeros(mlp.N_PARAMS)
    b3 = np.array([0.5, -1.0, 2.0, 0.0, 0.25, -0.75])
    theta[-6:] = b3
    rng = np.random.default_rng(3)
    x = rng.standard_normal((5, mlp.N_IN))
    y = rng.standard_normal((5, mlp.N_OUT))
    out, _ = mlp.forward(theta, x)
    assert np.array_equal(out, np.broadcast_to(b3, (5, 6)))
    g = mlp.grad(theta, x, y)
    assert np.allclose(g[-6:], 2.0 * (b3 - y.mean(0)) / 6.0, rtol=0, atol=1e-15)
    p = mlp.unpack(mlp.init_params(4))
    p["W3"][:] = 0.0
    p["W2"][:] = 0.0
    out, _ = mlp.forward(mlp.pack(p), x)
    assert np.allclose(out, p["b3"], atol=0)


def test_stencil_layout():
    shape = (5, 6, 7)
    cur = np.zeros((6,) + shape)
    prev = np.zeros((6,) + shape)
    cur[4, 2, 3, 5] = 7.0    # Hy at (x=5, y=3, z=2)
    prev[1, 3, 3, 4] = -2.0  # Ey at (x=4, y=3, z=3)
    x = mlp.stencil_inputs(cur, prev, [(4, 3, 2), (0, 0, 0)])
    # centre (4,3,2): Hy at dx=+1 -> (4*27 + 1*9 + 1*3 + 2); Ey(n-1) at dz=+1 -> 162 + 1*27 + 2*9 + 1*3 + 1
    assert x[0, 4 * 27 + 9 + 3 + 2] == 7.0
    assert x[0, 162 + 27 + 18 + 3 + 1] == -2.0
    assert np.count_nonzero(x[0]) == 2 and np.count_nonzero(x[1]) == 0
    cur[2, 2, 3, 4] = 1.5
    assert mlp.stencil_inputs(cur, prev, [(4, 3, 2)])[0, 2 * 27 + 13] == 1.5


def test_correction_is_scale_equivariant():
    theta = mlp.init_params(5)
    x = np.random.default_rng(6).standard_normal((4, mlp.N_IN))
    a = mlp.correction(theta, x)
    for s in (2.0 ** -20, 3.0, 1e6):
        assert np.allclose(mlp.correction(theta, s * x), s * a, rtol=1e-12, atol=0)
    assert np.array_equal(mlp.correction(theta, np.zeros((1, mlp.N_IN))), np.zeros((1, 6)))


def test_layer_cells_and_degenerate_networks():
    shape = (10, 11, 12)
    cells = mlp.layer_cells(shape, 2)
    assert len(cells) == 10 * 11 * 12 - 6 * 7 * 8
    eps = wl.random_eps(shape, 7)
    f0 = wl.random_fields(shape, 7)
    o = YeeOracle(shape, DT, eps, quantize_ce_f32=True)
    o.set_fields(f0)
    o.step(5)
    # zero output layer: the plain PEC box
    p = mlp.unpack(mlp.init_params(8))
    p["W3"][:] = 0.0
    cur, _ = mlp.learned_run(shape, eps, f0, 5, mlp.pack(p), thickness=2, dt=DT)
    assert np.array_equal(cur, o.fields())
    # thickness 0: the plain box too
    cur, _ = mlp.learned_run(shape, eps, f0, 5, mlp.init_params(9), thickness=0, dt=DT)
    assert np.array_equal(cur, o.fields())
    # a non-zero network changes exactly the tangential values on the faces:
    # E on the low faces, H on the high ones
    cur, _ = mlp.learned_run(shape, eps, f0, 1, mlp.init_params(9), thickness=2, dt=DT)
    o1 = YeeOracle(shape, DT, eps, quantize_ce_f32=True)
    o1.set_fields(f0)
    o1.step(1)
    changed = cur != o1.fields()
    nz, ny, nx = shape
    expect = np.zeros_like(changed)
    expect[1:3, :, :, 0] = True       # Ey, Ez at x = 0
    expect[[0, 2], :, 0, :] = True    # Ex, Ez at y = 0
    expect[0:2, 0, :, :] = True       # Ex, Ey at z = 0
    expect[4:6, :, :, nx - 1] = True  # Hy, Hz at x = nx-1
    expect[[3, 5], :, ny - 1, :] = True
    expect[3:5, nz - 1, :, :] = True
    assert not changed[~expect].any() and changed[expect].mean() > 0.9
