"""Shared test helpers: per-field error metrics and oracle runs."""
import numpy as np

from paper_2502_20610_gb300 import workloads as wl

FIELDS = ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz")


def rel_l2_per_field(got, ref):
    """Per-field relative L2 ||a-b|| / ||b||; a component whose reference norm
    is below 1e-6 of the all-field norm (zero in exact arithmetic, e.g. Hz of
    the config-1 pulse) is measured against the all-field norm instead."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    total = np.sqrt((ref ** 2).sum())
    out = {}
    for c in range(6):
        nb = np.sqrt((ref[c] ** 2).sum())
        err = np.sqrt(((got[c] - ref[c]) ** 2).sum())
        out[FIELDS[c]] = err / (nb if nb >= 1e-6 * total else total)
    return out


def bits_equal(a, b):
    """Bitwise equality of two float32 tensors/arrays."""
    import torch
    if isinstance(a, np.ndarray):
        a = torch.from_numpy(a)
    if isinstance(b, np.ndarray):
        b = torch.from_numpy(b)
    return torch.equal(a.contiguous().view(torch.int32).cpu(), b.contiguous().view(torch.int32).cpu())


def oracle_run(shape, eps, fields0, steps, sources=(), dt=wl.DT_DEFAULT, quantize=False):
    from oracle import YeeOracle
    o = YeeOracle(shape, dt, eps, quantize_ce_f32=quantize)
    o.set_fields(np.asarray(fields0, dtype=np.float64))
    for (c, i, j, k, J) in sources:
        o.add_source(c, i, j, k, J)
    o.step(steps)
    return o.fields()
