"""The C-ABI library builds, loads and exports every symbol include/fdtd.h
declares; host-side argument checks (no GPU compute)."""
import ctypes

import numpy as np
import os
import re

import pytest

from paper_2502_20610_gb300 import build as libbuild
from paper_2502_20610_gb300 import fdtd
from paper_2502_20610_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return fdtd.load_library()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "fdtd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fdtd_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(fdtd.EXPORTS) == names


def test_workspace_size_and_argument_checks(lib):
    g, c, b = fdtd.make_params((32, 48, 64), wl.DT_DEFAULT, scheme="systolic")
    n = ctypes.c_size_t(0)
    assert lib.fdtd_workspace_size(ctypes.byref(g), ctypes.byref(c), ctypes.byref(b), ctypes.byref(n)) == 0
    assert n.value >= 7 * 32 * 48 * 64 * 4
    gn, cn, bn = fdtd.make_params((32, 48, 64), wl.DT_DEFAULT, scheme="naive")
    m = ctypes.c_size_t(0)
    assert lib.fdtd_workspace_size(ctypes.byref(gn), ctypes.byref(cn), ctypes.byref(bn), ctypes.byref(m)) == 0
    assert m.value < n.value  # no tile schedule for the naive scheme
    bad = fdtd.Grid(0, 4, 4)
    assert lib.fdtd_workspace_size(ctypes.byref(bad), ctypes.byref(c), ctypes.byref(b),
                                   ctypes.byref(n)) == fdtd.FDTD_ERR_INVALID_ARG
    c2 = fdtd.Coeffs.from_buffer_copy(c)
    c2.dt = -1.0
    assert lib.fdtd_workspace_size(ctypes.byref(g), ctypes.byref(c2), ctypes.byref(b),
                                   ctypes.byref(n)) == fdtd.FDTD_ERR_INVALID_ARG
    b2 = fdtd.Boundary.from_buffer_copy(b)
    b2.kind = 7
    assert lib.fdtd_workspace_size(ctypes.byref(g), ctypes.byref(c), ctypes.byref(b2),
                                   ctypes.byref(n)) == fdtd.FDTD_ERR_INVALID_ARG
    assert lib.fdtd_workspace_size(None, ctypes.byref(c), ctypes.byref(b), ctypes.byref(n)) == \
        fdtd.FDTD_ERR_INVALID_ARG


def _ws(lib, g, c, b):
    n = ctypes.c_size_t(0)
    st = lib.fdtd_workspace_size(ctypes.byref(g), ctypes.byref(c), ctypes.byref(b), ctypes.byref(n))
    return st, n.value


def test_storage_option_checks(lib):
    shape = (32, 48, 64)
    st32, n32 = _ws(lib, *fdtd.make_params(shape, wl.DT_DEFAULT, scheme="naive"))
    for storage in ("f16", "bf16"):
        st, n16 = _ws(lib, *fdtd.make_params(shape, wl.DT_DEFAULT, scheme="naive", storage=storage))
        assert st == 0 and st32 == 0
        # 6 fields at 2 bytes + FP32 dt/eps + one FP32 transfer component
        assert n16 < n32 and n16 >= (6 * 2 + 4 + 4) * 32 * 48 * 64
        st, _ = _ws(lib, *fdtd.make_params(shape, wl.DT_DEFAULT, storage=storage, tile="31x15x12"))
        assert st == 0
        # the shared-memory systolic kernels hold FP32 only
        st, _ = _ws(lib, *fdtd.make_params(shape, wl.DT_DEFAULT, storage=storage, tile="31x15x15"))
        assert st == fdtd.FDTD_ERR_UNSUPPORTED
        for bad in (3.0, -2.0, float("inf"), float("nan"), 2.0 ** 120):
            sc = [1.0] * 6
            sc[4] = bad
            st, _ = _ws(lib, *fdtd.make_params(shape, wl.DT_DEFAULT, storage=storage, field_scale=sc))
            assert st == fdtd.FDTD_ERR_INVALID_ARG, bad
        st, _ = _ws(lib, *fdtd.make_params(shape, wl.DT_DEFAULT, storage=storage,
                                           field_scale=[0.0, 0.5, 2.0, 2.0 ** -20, 1.0, 8.0]))
        assert st == 0
    g, c, b = fdtd.make_params(shape, wl.DT_DEFAULT)
    c.storage = 3
    assert _ws(lib, g, c, b)[0] == fdtd.FDTD_ERR_INVALID_ARG


def test_boundary_option_checks(lib):
    shape = (40, 40, 40)
    ok = fdtd.make_params(shape, wl.DT_DEFAULT, boundary="graded", absorber=(8, 0.5, 3))
    st, n_abs = _ws(lib, *ok)
    assert st == 0
    assert n_abs > _ws(lib, *fdtd.make_params(shape, wl.DT_DEFAULT))[1]  # one more FP32 array
    assert _ws(lib, *fdtd.make_params(shape, wl.DT_DEFAULT, scheme="naive", boundary="graded",
                                      absorber=(8, 0.5, 3), storage="f16"))[0] == 0
    for bad in ((0, 0.5, 3), (8, -1.0, 3), (8, float("nan"), 3), (8, 0.5, -1), (8, 0.5, 17)):
        assert _ws(lib, *fdtd.make_params(shape, wl.DT_DEFAULT, boundary="graded", absorber=bad))[0] == \
            fdtd.FDTD_ERR_INVALID_ARG, bad
    # the lossy update is built for the default register tile only
    for tile in ("31x15x8", "31x15x15", "31x7x15"):
        assert _ws(lib, *fdtd.make_params(shape, wl.DT_DEFAULT, boundary="graded", absorber=(8, 0.5, 3),
                                          tile=tile))[0] == fdtd.FDTD_ERR_UNSUPPORTED
    assert _ws(lib, *fdtd.make_params(shape, wl.DT_DEFAULT, boundary="learned"))[0] == fdtd.FDTD_ERR_INVALID_ARG
    model = np.zeros(fdtd.mlp_param_count(), np.float32)
    st, n_l = _ws(lib, *fdtd.make_params(shape, wl.DT_DEFAULT, scheme="naive", boundary="learned",
                                         learned=(4, model)))
    n_plain = _ws(lib, *fdtd.make_params(shape, wl.DT_DEFAULT, scheme="naive"))[1]
    assert st == 0 and n_l > n_plain
    # two band snapshots (S^n, S^{n-1}), each six FP32 components and its x
    # slab (the planes x = 0, 1, nx-2, nx-1 of the six components)
    nz, ny, nx = shape
    assert n_l - n_plain >= 2 * (6 * 4 * nx * ny * nz + 4 * 24 * ny * nz)
    # the layer update needs the previous level every step: naive scheme, FP32
    assert _ws(lib, *fdtd.make_params(shape, wl.DT_DEFAULT, boundary="learned",
                                      learned=(4, model)))[0] == fdtd.FDTD_ERR_UNSUPPORTED
    assert _ws(lib, *fdtd.make_params(shape, wl.DT_DEFAULT, scheme="naive", storage="f16", boundary="learned",
                                      learned=(4, model)))[0] == fdtd.FDTD_ERR_UNSUPPORTED
    assert _ws(lib, *fdtd.make_params(shape, wl.DT_DEFAULT, scheme="naive", boundary="learned",
                                      learned=(0, model)))[0] == fdtd.FDTD_ERR_INVALID_ARG
    assert _ws(lib, *fdtd.make_params(shape, wl.DT_DEFAULT, scheme="naive", boundary="learned",
                                      learned=(4, model, -0.1, 3)))[0] == fdtd.FDTD_ERR_INVALID_ARG
    st, n_b = _ws(lib, *fdtd.make_params(shape, wl.DT_DEFAULT, scheme="naive", boundary="learned",
                                         learned=(4, model, 0.3, 3)))
    assert st == 0 and n_b > n_l  # the base layer's ca array
    sig = np.zeros(shape)
    assert _ws(lib, *fdtd.make_params(shape, wl.DT_DEFAULT, boundary="graded", absorber=sig))[0] == 0


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.fdtd_step(None, 1) == fdtd.FDTD_ERR_INVALID_ARG
    assert lib.fdtd_current_step(None) == -1
    assert lib.fdtd_launch_count(None) == -1
    lib.fdtd_destroy(None)
    for s in range(7):
        assert lib.fdtd_status_string(s)
    assert lib.fdtd_status_string(99) == b"unknown status"


def test_missing_library_fails_loudly(tmp_path):
    """Without the built library the binding raises (there is no CPU path to
    fall back to).  A fresh interpreter, since the loaded library is cached."""
    import subprocess
    import sys
    missing = str(tmp_path / "libfdtd.so")
    code = ("import sys; sys.path.insert(0, %r); from paper_2502_20610_gb300 import fdtd; "
            "fdtd.load_library(%r)" % (ROOT, missing))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode != 0
    assert "is not built" in r.stderr and "no CPU fallback" in r.stderr


def test_product_path_has_no_oracle_import():
    """The library binding never reaches the oracle (no CPU fallback)."""
    pkg = os.path.join(ROOT, "paper_2502_20610_gb300")
    for name in os.listdir(pkg):
        if name.endswith(".py"):
            src = open(os.path.join(pkg, name)).read()
            assert not re.search(r"^\s*(from|import)\s+oracle", src, flags=re.M), name
            assert "yee_oracle" not in src, name
