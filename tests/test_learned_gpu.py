"""Learned boundary on the GPU, through the C ABI.

* Network forward pass and gradient (the training kernels) against the FP64
  reference of oracle/mlp.py.
* Training on the GPU fits a teacher network's data.
* Recorded training pairs are stencils of the reference run, normalised.
* One learned-boundary run against the FP64 learned-boundary step.
* The gain: trained on thick-absorber runs, the 4-cell learned layer
  reflects less than a PEC wall and than a graded absorber of the same
  4 cells (measured against the thick absorber).
"""
import numpy as np
import pytest
import torch

from helpers import rel_l2_per_field
from oracle import mlp
from paper_2502_20610_gb300 import fdtd
from paper_2502_20610_gb300 import learned
from paper_2502_20610_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DT = wl.DT_DEFAULT


def test_forward_matches_fp64(cuda_device):
    theta = mlp.init_params(3)
    x = np.random.default_rng(4).standard_normal((1000, mlp.N_IN))
    ref, _ = mlp.forward(theta, x)
    p = torch.tensor(theta, dtype=torch.float32, device="cuda")
    got = fdtd.mlp_forward(p, torch.tensor(x, dtype=torch.float32, device="cuda"), batch=256).cpu().numpy()
    assert np.abs(got - ref).max() < 1e-5 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("n", [1, 257, 4096])
def test_gradient_matches_fp64(cuda_device, n):
    theta = mlp.init_params(5)
    rng = np.random.default_rng(6)
    x = rng.standard_normal((n, mlp.N_IN))
    y = rng.standard_normal((n, mlp.N_OUT))
    g_ref = mlp.grad(theta, x, y)
    l_ref = mlp.loss(theta, x, y)
    p = torch.tensor(theta, dtype=torch.float32, device="cuda")
    g, l = fdtd.mlp_grad(p, torch.tensor(x, dtype=torch.float32, device="cuda"),
                         torch.tensor(y, dtype=torch.float32, device="cuda"))
    g = g.cpu().numpy().astype(np.float64)
    assert abs(l - l_ref) <= 1e-5 * l_ref
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    # every block of the parameter vector
    for name, (a, b) in {"W1": (0, 20736), "b1": (20736, 20800), "W2": (20800, 24896), "b2": (24896, 24960),
                         "W3": (24960, 25344), "b3": (25344, 25350)}.items():
        assert np.linalg.norm(g[a:b] - g_ref[a:b]) <= 1e-4 * np.linalg.norm(g_ref[a:b]) + 1e-9, name


def test_training_fits_a_teacher(cuda_device):
    rng = np.random.default_rng(7)
    x = rng.standard_normal((32768, mlp.N_IN)) / np.sqrt(mlp.N_IN) * 3
    teacher = mlp.init_params(8)
    y, _ = mlp.forward(teacher, x)
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    yd = torch.tensor(y, dtype=torch.float32, device="cuda")
    p = torch.tensor(mlp.init_params(9), dtype=torch.float32, device="cuda")
    l0 = mlp.loss(mlp.init_params(9), x, y)
    last = fdtd.mlp_train(p, xd, yd, epochs=30, batch=1024, lr=2e-3, seed=1)
    l1 = mlp.loss(p.cpu().numpy().astype(np.float64), x, y)
    assert abs(last - l1) < 0.5 * l1 + 1e-6  # the kernels' epoch loss is the loss
    assert l1 < 0.05 * l0, (l0, l1)


def test_recorded_pairs_are_normalised_stencils(cuda_device):
    # reference run twice: once recording, once reading every state, then
    # each recorded row must be one layer cell's normalised stencil
    setup = learned.Setup(n=12, thickness=2, pad=6, absorber=(4, 0.5, 3))
    shape = (setup.N,) * 3
    src = (2, 11, 12, 13, wl.gaussian_pulse_source(40, DT, wavelength=8.0))
    a = setup.ref_sim(scheme="naive", max_source_steps=40)
    a.add_source(*src)
    a.step(5)
    x, y = fdtd.learned_record(a, setup.lo, setup.hi, setup.thickness, 3, 40, seed=5)
    b = setup.ref_sim(scheme="naive", max_source_steps=40)
    b.add_source(*src)
    b.step(5)
    states = [b.read_fields().cpu().numpy().astype(np.float64)]
    for _ in range(4):
        b.step(1)
        states.append(b.read_fields().cpu().numpy().astype(np.float64))
    from oracle import YeeOracle
    lo, hi = setup.lo[0], setup.hi[0]
    box = (setup.n,) * 3
    cells = mlp.layer_cells(box, setup.thickness)
    x, y = x.cpu().numpy(), y.cpu().numpy()
    for s in range(3):
        prev, cur, nxt = (st[:, lo:hi, lo:hi, lo:hi] for st in states[s:s + 3])
        cand = mlp.stencil_inputs(cur, prev, cells)
        r = np.sqrt(np.mean(cand ** 2, axis=1))
        inv = np.where(r >= mlp.R_MIN, 1.0 / np.where(r > 0, r, 1.0), 0.0)  # (near-)zero stencils stay 0
        cand_n = cand * inv[:, None]
        # the box's own PEC Yee step of S^n (no conductivity inside the box)
        o = YeeOracle(box, DT, setup.eps_bg, quantize_ce_f32=True)
        o.set_fields(cur)
        o.step(1)
        yee = o.fields()
        dy = (nxt - yee)[:, cells[:, 2], cells[:, 1], cells[:, 0]].T * inv[:, None]
        dy = np.where(mlp.tangent_mask(cells, box), dy, 0.0)
        for q in range(40):
            row = x[s * 40 + q]
            d = np.abs(cand_n - row).max(axis=1)
            best = int(np.argmin(d))
            assert d[best] < 1e-5, (s, q, d[best])
            assert np.abs(y[s * 40 + q] - dy[best]).max() < 1e-5 * max(1.0, np.abs(cand_n[best]).max())


@pytest.mark.parametrize("base", [0.0, 0.4])
def test_learned_step_matches_fp64_oracle(cuda_device, base):
    from oracle.yee import graded_sigma
    shape = (20, 22, 24)
    eps = wl.random_eps(shape, 10)
    f0 = wl.random_fields(shape, 10)
    p = mlp.unpack(mlp.init_params(11))
    p["W3"] *= 0.05  # a tame random network
    theta = mlp.pack(p)
    th32 = theta.astype(np.float32)
    src = [(2, 12, 11, 10, wl.sine_source(12, DT))]
    sim = fdtd.Sim(shape, eps, DT, scheme="naive", boundary="learned", learned=(4, th32, base, 3),
                   max_source_steps=12)
    sim.write_fields(torch.as_tensor(np.asarray(f0, np.float32)).cuda())
    sim.add_source(*src[0])
    sim.step(12)
    got = sim.read_fields().cpu().numpy()
    sim.close()
    ref, _ = mlp.learned_run(shape, eps, np.asarray(f0, np.float32).astype(np.float64), 12,
                             th32.astype(np.float64), thickness=4, sources=src, dt=DT,
                             sigma=graded_sigma(shape, 4, base, 3) if base > 0 else None)
    err = rel_l2_per_field(got, ref)
    assert max(err.values()) < 1e-4, err


def test_learned_layer_beats_pec_and_a_thin_absorber(cuda_device):
    # the 4-cell learned boundary (graded base, learned termination), trained
    # on pulses plus broadband initial noise (without the fine-grained
    # patterns the closed loop can meet patterns the network never saw and
    # grow them), measured against the 32-cell absorber
    setup = learned.Setup(n=48, thickness=4, pad=32, absorber=(32, 0.5, 3), base_sigma=0.3)
    x, y = learned.record(setup, seed=1, runs=4, sources_per_run=3, steps=250, per_step=1000, noise=0.05)  # 10^6 pairs
    assert torch.isfinite(x).all() and torch.isfinite(y).all()
    params, loss = learned.train(x, y, epochs=30, batch=4096, lr=1e-3)
    assert np.isfinite(loss)
    theta = params.cpu().numpy()
    e_learned, trace = learned.reflection(setup, "learned", theta, seed=99, steps=300)
    e_base, _ = learned.reflection(setup, "thin", seed=99, steps=300, ref_fields=trace)
    e_thin, _ = learned.reflection(setup, "thin", seed=99, steps=300, ref_fields=trace, sigma=0.5)
    e_pec, _ = learned.reflection(setup, "pec", seed=99, steps=300, ref_fields=trace)
    print(f"reflection error vs the 32-cell absorber: learned {e_learned:.3e}, its base alone {e_base:.3e}, "
          f"4-cell graded (sigma 0.5) {e_thin:.3e}, PEC {e_pec:.3e}; training loss {loss:.3e}")
    # The closed-loop reflection of a trained network varies with the
    # training seed (0.08 .. 0.21 over ten trainings on 0.75M and 1M pairs,
    # against 0.33 for the base alone and 0.26 for the 4-cell absorber cut),
    # so the bounds hold for every seed tried, not just this one (0.14).
    assert e_learned < 0.7 * e_base        # what the network adds to its own base
    assert e_learned < 0.85 * e_thin       # and against the thick absorber cut to 4 cells
    assert e_learned < e_pec
