"""FP64 reference of the learned boundary's network and of one learned-boundary
step.

TEST INFRASTRUCTURE ONLY: imported by tests/ (and nothing in the product
path).  Plain numpy, float64, written from the definitions:

Network (the learned absorbing boundary: 2 hidden layers of 64, input the
3x3x3 stencil of the 6 fields at steps n and n-1):
    f(x) = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3,   x in R^324, f in R^6.
Parameter vector (FP32 on the GPU), in this order:
    W1 [64][324], b1 [64], W2 [64][64], b2 [64], W3 [6][64], b3 [6]
    (25350 values; W row-major, row = output unit).
Input layout: x[(s*6 + c)*27 + (dz+1)*9 + (dy+1)*3 + (dx+1)], s = 0 for the
fields at step n, 1 for step n-1, c = Ex..Hz, stencil offsets in -1..1;
cells outside the domain read 0.
Scale equivariance: r = sqrt(mean(x^2)); the network sees x / r and predicts
a correction of the centre cell's six values, in units of r, to the Yee
step of the domain on its own (PEC walls), Yee_D:
    S^{n+1}(centre) = Yee_D(S^n)(centre) + r * f(x / r)   (r < 1e-30: + 0).
Loss of a batch: mean over samples and the 6 outputs of (f(x_hat) - y_hat)^2,
with y_hat = (S^{n+1}_ref - Yee_D(S^n))(centre) / r.

Learned-boundary step (the layer = cells within `thickness` of a wall):
    every cell takes the Yee step, then every layer cell adds the network's
    correction from the stencils of S^n and S^{n-1} to the components its
    walls get wrong: tangential E on a low face, tangential H on a high face
    (every other value of the Yee step is already the reference's).
"""
import numpy as np

N_IN, N_H, N_OUT = 324, 64, 6
R_MIN = 1e-30  # a smaller stencil RMS counts as a zero stencil
SIZES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
         ("W3", (N_OUT, N_H)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = theta[o:o + n].reshape(shape)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SIZES])


def forward(theta, x):
    """f(x) for a batch x [B, 324]; returns (y [B, 6], cache)."""
    p = unpack(theta)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ p["W1"].T + p["b1"]
    h1 = np.tanh(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.tanh(z2)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (x, h1, h2)


def loss(theta, x, y_hat):
    y, _ = forward(theta, x)
    return float(np.mean((y - y_hat) ** 2))


def grad(theta, x, y_hat):
    """Gradient of loss() with respect to the parameter vector (chain rule,
    layer by layer, d tanh(z)/dz = 1 - tanh(z)^2)."""
    p = unpack(theta)
    y, (x, h1, h2) = forward(theta, x)
    B = x.shape[0]
    dy = 2.0 * (y - y_hat) / (B * N_OUT)
    g = {"W3": dy.T @ h2, "b3": dy.sum(0)}
    dz2 = (dy @ p["W3"]) * (1.0 - h2 ** 2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * (1.0 - h1 ** 2)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(0)
    return pack(g)


def init_params(seed):
    """Small random network: uniform(-a, a) weights with a = 1/sqrt(fan_in),
    zero biases (seeded, numpy generator)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in SIZES:
        if name.startswith("W"):
            a = 1.0 / np.sqrt(shape[1])
            p[name] = rng.uniform(-a, a, shape)
        else:
            p[name] = np.zeros(shape)
    return pack(p)


def stencil_inputs(cur, prev, cells):
    """x [B, 324] for cells [B, 3] (x, y, z indices) from two (6, nz, ny, nx)
    states; outside the domain reads 0."""
    cur = np.asarray(cur, dtype=np.float64)
    prev = np.asarray(prev, dtype=np.float64)
    _, nz, ny, nx = cur.shape
    pad = [np.pad(a, ((0, 0), (1, 1), (1, 1), (1, 1))) for a in (cur, prev)]
    cells = np.asarray(cells)
    out = np.empty((len(cells), N_IN), dtype=np.float64)
    for q, (i, j, k) in enumerate(cells):
        for s in range(2):
            blk = pad[s][:, k:k + 3, j:j + 3, i:i + 3]  # [6, dz, dy, dx] around (i, j, k)
            out[q, s * 162:(s + 1) * 162] = blk.reshape(6, 27).ravel()
    return out


def correction(theta, x):
    """r f(x / r) for stencil inputs x [B, 324] (0 where r < R_MIN)."""
    x = np.asarray(x, dtype=np.float64)
    r = np.sqrt(np.mean(x ** 2, axis=1))
    live = r >= R_MIN
    safe = np.where(live, r, 1.0)
    f, _ = forward(theta, x / safe[:, None])
    return np.where(live[:, None], r[:, None] * f, 0.0)


def tangent_mask(cells, shape_zyx):
    """[B, 6] booleans: tangential E on the low faces, tangential H on the
    high faces that each cell (x, y, z) lies on."""
    nz, ny, nx = shape_zyx
    c = np.asarray(cells)
    x, y, z = c[:, 0], c[:, 1], c[:, 2]
    m = np.zeros((len(c), 6), bool)
    for lo, comps in ((x == 0, (1, 2)), (y == 0, (0, 2)), (z == 0, (0, 1)),
                      (x == nx - 1, (4, 5)), (y == ny - 1, (3, 5)), (z == nz - 1, (3, 4))):
        for k in comps:
            m[:, k] |= lo
    return m


def layer_cells(shape_zyx, thickness):
    """(x, y, z) indices of the cells within `thickness` of a wall, in
    x-fastest order."""
    nz, ny, nx = shape_zyx
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    d = np.minimum.reduce([i, nx - 1 - i, j, ny - 1 - j, k, nz - 1 - k])
    sel = d < thickness
    return np.stack([i[sel], j[sel], k[sel]], axis=1)


def learned_run(shape, eps, fields0, steps, theta, thickness=4, sources=(), dt=None, quantize=True,
                prev0=None, sigma=None):
    """FP64 learned-boundary run: the Yee oracle (conductivity `sigma` per
    cell if given: the layer's base) steps every cell, then the layer cells
    add the network's correction.  Returns (S^n, S^{n-1})."""
    from .yee import YeeOracle
    o = YeeOracle(shape, dt, eps, quantize_ce_f32=quantize)
    if sigma is not None:
        o.set_eps_sigma(eps, sigma, quantize)
    o.set_fields(fields0)
    for (c, i, j, k, J) in sources:
        o.add_source(c, i, j, k, J)
    cells = layer_cells(shape, thickness)
    mask = tangent_mask(cells, shape)
    prev = np.zeros((6,) + tuple(shape)) if prev0 is None else np.asarray(prev0, dtype=np.float64)
    cur = o.fields()
    for _ in range(steps):
        x = stencil_inputs(cur, prev, cells)
        corr = np.where(mask, correction(theta, x), 0.0)
        o.step(1)
        nxt = o.fields()
        nxt[:, cells[:, 2], cells[:, 1], cells[:, 0]] += corr.T
        o.set_fields(nxt)
        prev, cur = cur, nxt
    return cur, prev
