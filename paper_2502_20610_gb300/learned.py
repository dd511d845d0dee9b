"""Learned absorbing boundary: data, training and evaluation, driving the
library's kernels through the C ABI (fdtd_learned_record, fdtd_mlp_train,
FDTD_BOUNDARY_LEARNED).  Orchestration only; every arithmetic step runs in
libfdtd's CUDA kernels.

Set-up: the learned boundary replaces a thick graded absorber.  A reference domain is the learned domain D (n^3 cells, its outer
`thickness` cells a graded base layer) surrounded by `pad` more cells whose
outer `absorber` cells conduct (graded, order 3); the network learns, for
D's face cells, the correction from D's own Yee step (PEC walls) to the
reference run's next state, from the stencils of the last two states with
everything outside D read as 0 -- exactly what it will see when D stands
alone with the learned layer at its walls.

Reflection of a boundary: run the same source in D with that boundary and
in the reference domain; the error is the energy of the difference in D's
interior (cells not in the layer) summed over the run, relative to the
reference's energy there.  The thick absorber is the yardstick (its own
error is zero by definition); a plain PEC wall, a graded absorber as thin as the
learned layer, and the learned layer are compared on it.
"""
import numpy as np

from . import fdtd
from . import workloads as wl

DT = wl.DT_DEFAULT


def graded_profile(n, thickness, sigma_max, order):
    """sigma_max * sum_a (depth_a / thickness)^order on an n^3 box, depth_a =
    thickness - i inside the low layer, i - (n-1-thickness) inside the high
    one (the library's graded absorber profile), as float64 (n, n, n)."""
    i = np.arange(n)
    d = np.where(i < thickness, thickness - i, np.where(i >= n - thickness, i - (n - 1 - thickness), 0))
    w = np.where(d > 0, (d / thickness) ** order, 0.0)
    return sigma_max * (w[:, None, None] + w[None, :, None] + w[None, None, :])


class Setup:
    """Geometry of a learned-boundary experiment (all sizes in cells).

    The learned domain D is n^3 with a `thickness`-cell layer at its walls:
    graded conductivity `base_sigma` (order 3) whose PEC termination the
    network corrects.  The reference is D, layer included, inside `pad`
    more cells whose outer `absorber` cells conduct (the thick absorber)."""

    def __init__(self, n=48, thickness=4, pad=32, absorber=(32, 0.5, 3), eps_bg=2.1, base_sigma=0.3):
        self.n, self.thickness, self.pad = n, thickness, pad
        self.absorber = absorber
        self.eps_bg = eps_bg
        self.base_sigma = base_sigma
        self.N = n + 2 * pad

    @property
    def lo(self):
        return (self.pad,) * 3

    @property
    def hi(self):
        return (self.pad + self.n,) * 3

    def ref_sigma(self, with_layer=True):
        sig = graded_profile(self.N, *self.absorber)
        if with_layer and self.base_sigma > 0:
            p, n = self.pad, self.n
            sig[p:p + n, p:p + n, p:p + n] += graded_profile(n, self.thickness, self.base_sigma, 3)
        return sig

    def ref_sim(self, scheme="systolic", max_source_steps=0, with_layer=True):
        """The reference domain; with_layer=False is the yardstick: the thick
        absorber alone."""
        shape = (self.N,) * 3
        return fdtd.Sim(shape, self.eps_bg, DT, scheme=scheme, boundary="graded",
                        absorber=self.ref_sigma(with_layer), max_source_steps=max_source_steps)

    def sim(self, kind, params=None, max_source_steps=0, sigma=None):
        """The n^3 domain with boundary kind "learned", "pec" or "thin": a
        graded absorber of the layer's thickness with peak conductivity
        `sigma` (default: the learned boundary's base, i.e. the learned layer
        without its network)."""
        shape = (self.n,) * 3
        if kind == "learned":
            return fdtd.Sim(shape, self.eps_bg, DT, scheme="naive", boundary="learned",
                            learned=(self.thickness, params, self.base_sigma, 3), max_source_steps=max_source_steps)
        if kind == "thin":
            s = self.base_sigma if sigma is None else sigma
            return fdtd.Sim(shape, self.eps_bg, DT, scheme="naive", boundary="graded",
                            absorber=(self.thickness, s, 3), max_source_steps=max_source_steps)
        return fdtd.Sim(shape, self.eps_bg, DT, scheme="naive", max_source_steps=max_source_steps)


def _sources(setup, seed, count, steps, wavelengths=(10.0, 20.0)):
    """Seeded pulse sources inside D (away from its layer), in D coordinates."""
    u = wl.uniform_pm1(seed, 5 * count)
    out = []
    m = setup.thickness + 4
    for q in range(count):
        x, y, z = (int(m + (setup.n - 2 * m - 1) * (0.5 + 0.5 * u[5 * q + a])) for a in range(3))
        comp = int(3 * (0.5 + 0.5 * u[5 * q + 3])) % 3
        lam = wavelengths[0] + (wavelengths[1] - wavelengths[0]) * (0.5 + 0.5 * u[5 * q + 4])
        out.append((comp, x, y, z, wl.gaussian_pulse_source(steps, DT, wavelength=lam)))
    return out


def record(setup, seed=1, runs=2, sources_per_run=3, steps=300, per_step=1000, warm=20, noise=0.0):
    """Training pairs from reference runs with seeded pulse sources (and,
    if noise > 0, seeded broadband initial fields of that amplitude, so the
    network also sees the reference's response to fine-grained patterns).
    Returns (x [m, 324], y [m, 6]) CUDA tensors."""
    import torch
    xs, ys = [], []
    for r in range(runs):
        ref = setup.ref_sim(max_source_steps=steps + warm + 1)
        if noise > 0:
            f0 = noise * wl.random_fields((setup.N,) * 3, seed * 1000 + r + 500)
            ref.write_fields(torch.as_tensor(f0.astype(np.float32)).to(ref.device))
        for (c, x, y, z, J) in _sources(setup, seed * 1000 + r, sources_per_run, steps + warm + 1):
            ref.add_source(c, x + setup.pad, y + setup.pad, z + setup.pad, J)
        ref.step(warm)
        X, Y = fdtd.learned_record(ref, setup.lo, setup.hi, setup.thickness, steps, per_step, seed=seed * 7 + r)
        ref.close()
        xs.append(X)
        ys.append(Y)
    return torch.cat(xs), torch.cat(ys)


def train(x, y, epochs=20, batch=4096, lr=1e-3, seed=0, init_seed=0):
    """A network trained on the GPU from a small random start."""
    import torch
    from . import fdtd as f
    n = f.mlp_param_count()
    rng = np.random.default_rng(init_seed)
    sizes = [(64, 324), (64,), (64, 64), (64,), (6, 64), (6,)]
    parts = []
    for s in sizes:
        if len(s) == 2:
            a = 1.0 / np.sqrt(s[1])
            parts.append(rng.uniform(-a, a, s).ravel())
        else:
            parts.append(np.zeros(s))
    theta = np.concatenate(parts).astype(np.float32)
    assert theta.size == n
    params = torch.from_numpy(theta).to(x.device)
    loss = f.mlp_train(params, x, y, epochs, batch=batch, lr=lr, seed=seed)
    return params, loss


def reflection(setup, kind, params=None, seed=99, steps=400, ref_fields=None, sigma=None):
    """Relative error energy of boundary `kind` against the thick absorber
    over `steps` steps of a seeded pulse; returns (error, reference trace)
    where the trace (the reference's interior fields per step) can be
    passed back in to reuse it."""
    import torch
    src = _sources(setup, seed, 1, steps)
    t = setup.thickness
    inner = slice(t, setup.n - t)
    if ref_fields is None:
        ref = setup.ref_sim(scheme="naive", max_source_steps=steps, with_layer=False)
        for (c, x, y, z, J) in src:
            ref.add_source(c, x + setup.pad, y + setup.pad, z + setup.pad, J)
        p0, p1 = setup.pad + t, setup.pad + setup.n - t
        ref_fields = []
        for _ in range(steps):
            ref.step(1)
            ref_fields.append(ref.read_fields()[:, p0:p1, p0:p1, p0:p1].double())
        ref.close()
    sim = setup.sim(kind, params, max_source_steps=steps, sigma=sigma)
    for (c, x, y, z, J) in src:
        sim.add_source(c, x, y, z, J)
    num = den = 0.0
    for s in range(steps):
        sim.step(1)
        f = sim.read_fields()[:, inner, inner, inner].double()
        num += float(((f - ref_fields[s]) ** 2).sum())
        den += float((ref_fields[s] ** 2).sum())
    sim.close()
    return num / den, ref_fields


def reflection_lockstep(setup, boundaries, source, steps):
    """Reflection errors of several boundaries at once against the thick
    absorber (the yardstick), stepping every domain together so that no
    trace of the reference is stored (for large grids).

    boundaries: {name: (kind, params, sigma)} for setup.sim; source: (comp,
    x, y, z, J) in D coordinates.  Returns {name: error}: the energy of
    (field - yardstick's field) in D's interior summed over `steps` steps,
    relative to the yardstick's energy there (FP64 sums on the device)."""
    import torch
    t = setup.thickness
    inner = slice(t, setup.n - t)
    p0, p1 = setup.pad + t, setup.pad + setup.n - t
    c, x, y, z, J = source
    ref = setup.ref_sim(scheme="naive", max_source_steps=steps, with_layer=False)
    ref.add_source(c, x + setup.pad, y + setup.pad, z + setup.pad, J)
    sims = {}
    for name, (kind, params, sigma) in boundaries.items():
        s = setup.sim(kind, params, max_source_steps=steps, sigma=sigma)
        s.add_source(c, x, y, z, J)
        sims[name] = s
    num = {name: torch.zeros((), dtype=torch.float64, device=ref.device) for name in sims}
    den = torch.zeros((), dtype=torch.float64, device=ref.device)
    for _ in range(steps):
        ref.step(1)
        r = ref.read_fields()[:, p0:p1, p0:p1, p0:p1]
        den += (r.double() ** 2).sum()
        for name, s in sims.items():
            s.step(1)
            f = s.read_fields()[:, inner, inner, inner]
            num[name] += ((f.double() - r.double()) ** 2).sum()
    ref.close()
    for s in sims.values():
        s.close()
    return {name: float(num[name] / den) for name in sims}
