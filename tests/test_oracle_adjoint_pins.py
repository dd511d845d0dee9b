"""Pins of the FP64 adjoint reference (oracle/adjoint.py).

* Dot-product test: the transposed step is the transpose of the forward
  step, <F v, u> = <v, F^T u>, for random states (catches a wrong sign, a
  misplaced coefficient or mask, a curl that is not the other's transpose).
* The numpy forward step equals the C oracle's (source-free), so the
  adjoint differentiates the map the oracle computes.
* Central finite differences of the oracle's own objective on single
  voxels (including one next to the source and one on a wall), the
  independent definition of the gradient.
* The identity the GPU's adjoint sweep rests on: in the variables
  (M c lambda_E, -dt lambda_H) the transposed step is the forward step, and
  the gradient computed that way equals the oracle's reverse sweep.
"""
import numpy as np

from oracle import YeeOracle
from oracle import adjoint as adj
from paper_2502_20610_gb300 import workloads as wl

DT = wl.DT_DEFAULT


def test_transposed_step_is_the_transpose():
    shape = (7, 8, 9)
    rng = np.random.default_rng(1)
    c = DT / wl.random_eps(shape, 2)
    M = adj.pec_mask(shape)
    v = (rng.standard_normal((3,) + shape), rng.standard_normal((3,) + shape))
    u = (rng.standard_normal((3,) + shape), rng.standard_normal((3,) + shape))
    Fv = adj.yee_step(v[0], v[1], c, DT, M)
    Tu = adj.transposed_step(u[0], u[1], c, DT, M)
    lhs = (Fv[0] * u[0]).sum() + (Fv[1] * u[1]).sum()
    rhs = (v[0] * Tu[0]).sum() + (v[1] * Tu[1]).sum()
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs))
    # a wrong transpose (curl_f used on both sides) fails it
    bad = (u[0] - DT * adj.curl_f(u[1] + adj.curl_f(M * c[None] * u[0])), u[1] + adj.curl_f(M * c[None] * u[0]))
    rhs_bad = (v[0] * bad[0]).sum() + (v[1] * bad[1]).sum()
    assert abs(lhs - rhs_bad) > 1e-6 * abs(lhs)


def test_numpy_step_is_the_oracle_step():
    shape = (6, 7, 8)
    eps = wl.random_eps(shape, 3)
    f0 = wl.random_fields(shape, 3, zero_pec_walls=False)
    o = YeeOracle(shape, DT, eps)
    o.set_fields(f0)
    o.step(1)
    E, H = adj.yee_step(np.asarray(f0[:3], np.float64), np.asarray(f0[3:], np.float64), o.ce(), DT,
                        adj.pec_mask(shape))
    assert np.allclose(o.fields(), np.concatenate([E, H]), rtol=0, atol=1e-13)


def test_gradient_matches_central_differences():
    shape = (10, 12, 14)
    eps = wl.random_eps(shape, 4, lo=2.1, hi=12.1)
    steps = 60
    src = [(2, 6, 5, 2, wl.sine_source(steps, DT, 8.0))]
    mode = np.asarray(wl.uniform_pm1(5, 12 * 14)).reshape(12, 14)
    obj = adj.Objective(k0=8, mode=mode, window=20)
    f0 = np.zeros((6,) + shape)
    L, g = adj.gradient(shape, eps, f0, steps, src, obj, DT)
    assert L > 0
    for (k, j, i) in [(5, 6, 7), (2, 5, 6), (3, 4, 7), (9, 11, 13), (0, 3, 3), (6, 0, 9)]:
        h = 1e-5 * eps[k, j, i]
        ep, em = eps.copy(), eps.copy()
        ep[k, j, i] += h
        em[k, j, i] -= h
        fd = (adj.objective(shape, ep, f0, steps, src, obj, DT) - adj.objective(shape, em, f0, steps, src, obj, DT)) / (2 * h)
        assert abs(fd - g[k, j, i]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(g).max()), ((k, j, i), fd, g[k, j, i])


def test_windowed_objective_equals_the_history_objective():
    # the no-history form used for finite differences on larger grids
    shape = (9, 10, 11)
    eps = wl.random_eps(shape, 6, lo=2.1, hi=12.1)
    steps = 40
    src = [(1, 5, 4, 3, wl.sine_source(steps, DT, 9.0))]
    mode = np.asarray(wl.uniform_pm1(7, 10 * 11)).reshape(10, 11)
    obj = adj.Objective(k0=6, mode=mode, window=13)
    f0 = np.zeros((6,) + shape)
    a = adj.objective(shape, eps, f0, steps, src, obj, DT)
    b = adj.objective_window(shape, eps, f0, steps, src, obj, DT)
    assert a > 0 and abs(a - b) <= 1e-14 * a


def test_transposed_step_is_the_forward_step_in_scaled_variables():
    shape = (6, 7, 8)
    rng = np.random.default_rng(4)
    c = DT / wl.random_eps(shape, 5)
    M = adj.pec_mask(shape)
    le, lh = rng.standard_normal((3,) + shape), rng.standard_normal((3,) + shape)
    te, th = adj.transposed_step(le, lh, c, DT, M)
    fe, fh = adj.yee_step(M * c[None] * le, -DT * lh, c, DT, M)
    assert np.allclose(fe, M * c[None] * te, rtol=0, atol=1e-12)
    assert np.allclose(fh, -DT * th, rtol=0, atol=1e-12)


def test_gradient_in_scaled_variables_equals_the_reverse_sweep():
    # the GPU's form: E~ = M c lambda_E stepped by the forward map, the
    # objective's source added as M c dg/dE, dL/deps = -(1/dt) sum E~ . dE
    shape = (10, 9, 11)
    eps = wl.random_eps(shape, 6, lo=2.1, hi=12.1)
    steps = 30
    src = [(2, 5, 4, 3, wl.sine_source(steps, DT, 9.0))]
    mode = np.asarray(wl.uniform_pm1(7, 9 * 11)).reshape(9, 11)
    obj = adj.Objective(k0=6, mode=mode, window=11)
    f0 = np.zeros((6,) + shape)
    L, g = adj.gradient(shape, eps, f0, steps, src, obj, DT)
    _, hist, c = adj.forward(shape, eps, f0, steps, src, obj, DT)
    M = adj.pec_mask(shape)

    def source_of(n):
        s = np.zeros((3,) + shape)
        if obj.weight(n, steps):
            s[2, obj.k0] = 2.0 * obj.overlap(hist[n]) * obj.mode
        return M * c[None] * s

    et, ht = source_of(steps), np.zeros((3,) + shape)
    g2 = np.zeros(shape)
    for n in range(steps - 1, -1, -1):
        g2 -= (et * (hist[n + 1] - hist[n])).sum(0) / DT
        et, ht = adj.yee_step(et, ht, c, DT, M)
        et = et + source_of(n)
    assert np.abs(g2 - g).max() <= 1e-12 * np.abs(g).max()
