"""CPU check of the systolic tile schedule (host logic, no GPU).

A model of the persistent kernel's global-memory traffic: tiles of 31x15x15
cells in skewed space sigma = p + t (Sec. 3, Fig. 7; Sec. 4) are handed out
in the library's topological order to a few virtual CTAs, which run in a
random interleaving.  Each step of a tile is split in two actions, as on the
GPU: (wait on the -x/-y/-z progress flags, read the lower shell) and (write
the top faces, publish).  Global memory is modelled as the time level each
cell currently holds; every read must find exactly the level the update
needs (a smaller level is a read-before-write race, a larger one an
overwrite-before-read race), and every (cell, step) must be computed once.
"""
import random

import numpy as np
import pytest

TX, TY, TZ = 31, 15, 15
SHAPES = [(31, 15, 15), (31, 7, 15), (31, 15, 12), (31, 15, 8)]  # the tile shapes the library is built with


def interval(I, J, K, N, T, n=(TX, TY, TZ)):
    A = (I * n[0], J * n[1], K * n[2])
    s = max(0, A[0] - N[0] + 1, A[1] - N[1] + 1, A[2] - N[2] + 1)
    e = min(T - 1, A[0] + n[0] - 1, A[1] + n[1] - 1, A[2] + n[2] - 1)
    return s, e


def tile_order(N, T_max, order=0, seed=0, n=(TX, TY, TZ)):
    """Same rule as the library: keep start <= end+1, sort by (start, I+J+K)."""
    gx = -(-(N[0] + T_max - 1) // n[0])
    gy = -(-(N[1] + T_max - 1) // n[1])
    gz = -(-(N[2] + T_max - 1) // n[2])
    rng = random.Random(seed)
    ent = []
    for K in range(gz):
        for J in range(gy):
            for I in range(gx):
                s, e = interval(I, J, K, N, T_max, n)
                if s > e + 1:
                    continue
                key = (s, K, J, I) if order == 2 else (s, I + J + K, rng.random() if order == 1 else 0, I, J, K)
                ent.append((key, (I, J, K)))
    ent.sort()
    return [t for _, t in ent], (gx, gy, gz)


def box(lo, hi):
    """Boolean-free index arrays of the integer box [lo, hi) (x,y,z)."""
    xs, ys, zs = (np.arange(lo[a], hi[a]) for a in range(3))
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return X.ravel(), Y.ravel(), Z.ravel()


def run_model(N, T, n_cta=6, seed=0, order=0, T_max=None, n=(TX, TY, TZ)):
    T_max = T_max or T
    tiles, (gx, gy, gz) = tile_order(N, T_max, order, seed, n)
    tiles = [t for t in tiles if interval(*t, N, T, n)[0] <= T]  # launch uses count_le[T]
    rng = random.Random(seed)
    lvl = np.full((N[2], N[1], N[0]), -1, dtype=np.int64)
    count = np.zeros((T,) + lvl.shape, dtype=np.int32)
    progress = {}
    errors = []

    def indom(x, y, z):
        return (x >= 0) & (x < N[0]) & (y >= 0) & (y < N[1]) & (z >= 0) & (z < N[2])

    def read(x, y, z, L, what):
        m = indom(x, y, z)
        got = lvl[z[m], y[m], x[m]]
        if not np.all(got == L):
            errors.append((what, L, np.unique(got).tolist()))

    def write(x, y, z, L):
        m = indom(x, y, z)
        lvl[z[m], y[m], x[m]] = L

    def wait_ok(I, J, K, L):
        for u in ((I - 1, J, K), (I, J - 1, K), (I, J, K - 1)):
            if min(u) < 0:
                continue
            s, e = interval(*u, N, T, n)
            if s > e + 1 or L < s - 1 or L > e:
                continue
            if progress.get(u, -10**9) < L + 1:
                return False
        return True

    def actions(tile):
        I, J, K = tile
        A = (I * n[0], J * n[1], K * n[2])
        s, e = interval(I, J, K, N, T, n)
        if s > 0:
            yield ("wait", s - 1)
        if s > e:
            yield ("publish", s)
            return
        lo = tuple(A[a] - s for a in range(3))
        yield ("read", box(lo, tuple(lo[a] + n[a] + 1 for a in range(3))), s - 1, "initial")
        if s > 0:
            yield ("publish", s)
        for t in range(s, e + 1):
            yield ("wait", t)
            b = tuple(A[a] - t for a in range(3))
            x, y, z = box(tuple(b[a] - 1 for a in range(3)), tuple(b[a] + n[a] for a in range(3)))
            shell = (x < b[0]) | (y < b[1]) | (z < b[2])
            yield ("read", (x[shell], y[shell], z[shell]), t, "shell")
            x, y, z = box(b, tuple(b[a] + n[a] for a in range(3)))
            m = indom(x, y, z)
            count[t, z[m], y[m], x[m]] += 1
            if t == T - 1:
                out = np.ones_like(x, dtype=bool)
            else:
                out = (x == b[0] + n[0] - 1) | (y == b[1] + n[1] - 1) | (z == b[2] + n[2] - 1)
            yield ("write", (x[out], y[out], z[out]), t)
            yield ("publish", t + 1)

    next_ticket = 0
    ctas = [None] * n_cta
    while True:
        for c in range(n_cta):
            if ctas[c] is None and next_ticket < len(tiles):
                tile = tiles[next_ticket]
                next_ticket += 1
                ctas[c] = [tile, actions(tile), None]
        live = [c for c in range(n_cta) if ctas[c] is not None]
        if not live:
            break
        rng.shuffle(live)
        progressed = False
        for c in live:
            tile, gen, pending = ctas[c]
            if pending is None:
                try:
                    pending = next(gen)
                except StopIteration:
                    ctas[c] = None
                    progressed = True
                    break
            if pending[0] == "wait" and not wait_ok(*tile, pending[1]):
                ctas[c][2] = pending
                continue
            if pending[0] == "read":
                read(*pending[1], pending[2], pending[3])
            elif pending[0] == "write":
                write(*pending[1], pending[2])
            elif pending[0] == "publish":
                progress[tile] = max(progress.get(tile, -10**9), pending[1])
            ctas[c][2] = None
            progressed = True
            break
        assert progressed, "deadlock in the tile schedule"
    return errors, count, lvl


CASES = [
    ((45, 33, 20), 25),   # several tiles per axis, T < N
    ((20, 17, 9), 60),    # T > N: tiles enter and leave the domain
    ((70, 16, 31), 7),    # short launch
    ((1, 1, 1), 5),       # degenerate grid
]


@pytest.mark.parametrize("N,T", CASES)
@pytest.mark.parametrize("order", [0, 1, 2])
@pytest.mark.parametrize("n", SHAPES)
def test_schedule_levels_and_coverage(N, T, order, n):
    errors, count, lvl = run_model(N, T, n_cta=5, seed=1 + order, order=order, n=n)
    assert not errors, errors[:5]
    assert np.all(count == 1), "every (cell, step) must be updated exactly once"
    assert np.all(lvl == T - 1), "after the launch global memory holds one uniform time level"


def test_schedule_shorter_launch_than_tile_list():
    # a launch of T steps with the tile list built for T_max > T
    errors, count, lvl = run_model((45, 33, 20), 9, n_cta=4, seed=5, T_max=40)
    assert not errors
    assert np.all(count == 1) and np.all(lvl == 8)


def test_paper_tile_arithmetic():
    # Sec. 4: 31x15x15 updated, 32x16x16 stored; ~32*16+32*16+16*16 cells
    # loaded and written per iteration; ~5.45x fewer global memory operations
    assert TX * TY * TZ == 6975
    assert (TX + 1) * (TY + 1) * (TZ + 1) == 8192
    faces = 32 * 16 + 32 * 16 + 16 * 16
    assert faces == 1280
    assert round(6975 / faces, 2) == 5.45
    # the exact shell of the ring is a little smaller than the paper's count
    assert 8192 - 6975 == 1217


# ---------------------------------------------------------------------------
# Face buffers of the register kernel.  The top x and y faces of a tile do not
# go to the field arrays but to two face buffers indexed by physical (x, y) and
# by z'' = (sigma_z mod P) (sigma_z = z + t, P a multiple of the tile's z
# extent), so a tile's faces and shells are z-blocks that start at a fixed,
# aligned position for the whole life of the tile.  The lower shell of a tile
# step is then read from three places: the z plane (with its x and y edges)
# from the field arrays, the y plane (without the x edge and the z row) from
# the y-face buffer, and the x plane (with its y edge, without the z row) from
# the x-face buffer.  The model stores, per buffer location, which cell and
# which level it holds, so a read that finds another cell's value (a wrapped
# index reused too early) is caught as well as a wrong level.

def run_face_model(N, T, P, n_cta=5, seed=0, order=0, n=(31, 15, 12)):
    tiles, _ = tile_order(N, T, order, seed, n)
    tiles = [t for t in tiles if interval(*t, N, T, n)[0] <= T]
    rng = random.Random(seed)
    nx, ny, nz = N
    F = np.full((nz, ny, nx), -1, dtype=np.int64)      # field arrays: level of the cell
    # face buffers: (level, physical z) held at (x, y, z'')
    X = np.full((nx, ny, P, 2), -9, dtype=np.int64)
    Y = np.full((ny, nx, P, 2), -9, dtype=np.int64)
    count = np.zeros((T,) + F.shape, dtype=np.int32)
    progress = {}
    errors = []

    def indom(x, y, z):
        return (x >= 0) & (x < nx) & (y >= 0) & (y < ny) & (z >= 0) & (z < nz)

    def zidx(z, t):
        return (z + t) % P

    def read_shell(b, t_level, lvl_t, tag):
        # b: low corner of the box whose lower shell is read; values must be at
        # level lvl_t; t_level: the step whose skew maps z to z'' (= lvl_t)
        x, y, z = box(tuple(b[a] - 1 for a in range(3)), tuple(b[a] + n[a] for a in range(3)))
        shell = (x < b[0]) | (y < b[1]) | (z < b[2])
        x, y, z = x[shell], y[shell], z[shell]
        m = indom(x, y, z)
        x, y, z = x[m], y[m], z[m]
        zpl = z == b[2] - 1
        ypl = (~zpl) & (y == b[1] - 1) & (x >= b[0])
        xpl = (~zpl) & (x == b[0] - 1)
        got = F[z[zpl], y[zpl], x[zpl]]
        if not np.all(got == lvl_t):
            errors.append((tag, "z shell", lvl_t, np.unique(got).tolist()))
        for sel, buf, (i0, i1) in ((ypl, Y, (y, x)), (xpl, X, (x, y))):
            if not sel.any():
                continue
            h = buf[i0[sel], i1[sel], zidx(z[sel], t_level)]
            if not (np.all(h[:, 0] == lvl_t) and np.all(h[:, 1] == z[sel])):
                errors.append((tag, "y shell" if buf is Y else "x shell", lvl_t,
                               np.unique(h[:, 0]).tolist()))

    def write_faces(b, t):
        # top z plane -> field arrays; top y and x planes -> face buffers
        x, y, z = box(b, tuple(b[a] + n[a] for a in range(3)))
        m = indom(x, y, z)
        x, y, z = x[m], y[m], z[m]
        if t == T - 1:
            F[z, y, x] = t
        else:
            zt = z == b[2] + n[2] - 1
            F[z[zt], y[zt], x[zt]] = t
        for sel, buf, (i0, i1) in (((y == b[1] + n[1] - 1), Y, (y, x)), ((x == b[0] + n[0] - 1), X, (x, y))):
            buf[i0[sel], i1[sel], zidx(z[sel], t), 0] = t
            buf[i0[sel], i1[sel], zidx(z[sel], t), 1] = z[sel]

    def wait_ok(I, J, K, L):
        for u in ((I - 1, J, K), (I, J - 1, K), (I, J, K - 1)):
            if min(u) < 0:
                continue
            s, e = interval(*u, N, T, n)
            if s > e + 1 or L < s - 1 or L > e:
                continue
            if progress.get(u, -10**9) < L + 1:
                return False
        return True

    def actions(tile):
        I, J, K = tile
        A = (I * n[0], J * n[1], K * n[2])
        s, e = interval(I, J, K, N, T, n)
        if s > 0:
            yield ("wait", s - 1)
        if s > e:
            yield ("publish", s)
            return
        b0 = tuple(A[a] - s + 1 for a in range(3))  # box at level s-1
        if s == 0:
            yield ("read_initial_fields", b0)
        else:
            yield ("read_shell", b0, s - 1, s - 1, "initial")
            yield ("publish", s)
        for t in range(s, e + 1):
            yield ("wait", t)
            b = tuple(A[a] - t for a in range(3))
            yield ("read_shell", b, t, t, "step")
            x, y, z = box(b, tuple(b[a] + n[a] for a in range(3)))
            m = indom(x, y, z)
            count[t, z[m], y[m], x[m]] += 1
            yield ("write", b, t)
            yield ("publish", t + 1)

    def initial_fields(b):
        x, y, z = box(tuple(b[a] - 1 for a in range(3)), tuple(b[a] + n[a] for a in range(3)))
        m = indom(x, y, z)
        got = F[z[m], y[m], x[m]]
        if not np.all(got == -1):
            errors.append(("initial s=0", np.unique(got).tolist()))

    next_ticket = 0
    ctas = [None] * n_cta
    while True:
        for c in range(n_cta):
            if ctas[c] is None and next_ticket < len(tiles):
                tile = tiles[next_ticket]
                next_ticket += 1
                ctas[c] = [tile, actions(tile), None]
        live = [c for c in range(n_cta) if ctas[c] is not None]
        if not live:
            break
        rng.shuffle(live)
        progressed = False
        for c in live:
            tile, gen, pending = ctas[c]
            if pending is None:
                try:
                    pending = next(gen)
                except StopIteration:
                    ctas[c] = None
                    progressed = True
                    break
            if pending[0] == "wait" and not wait_ok(*tile, pending[1]):
                ctas[c][2] = pending
                continue
            if pending[0] == "read_shell":
                read_shell(pending[1], pending[2], pending[3], pending[4])
            elif pending[0] == "read_initial_fields":
                initial_fields(pending[1])
            elif pending[0] == "write":
                write_faces(pending[1], pending[2])
            elif pending[0] == "publish":
                progress[tile] = max(progress.get(tile, -10**9), pending[1])
            ctas[c][2] = None
            progressed = True
            break
        assert progressed, "deadlock in the tile schedule"
    return errors, count, F


def face_period(nz, tz):
    """z'' period of the face buffers: nz rounded up to the tile's z extent."""
    return -(-nz // tz) * tz


FACE_CASES = [
    ((45, 33, 20), 25),
    ((20, 17, 9), 60),
    ((70, 16, 31), 7),
    ((40, 20, 37), 50),
    ((1, 1, 1), 5),
]


@pytest.mark.parametrize("N,T", FACE_CASES)
@pytest.mark.parametrize("order", [0, 1, 2])
@pytest.mark.parametrize("n", [(31, 15, 12), (31, 15, 8)])
def test_face_buffers_levels_and_coverage(N, T, order, n):
    P = face_period(N[2], n[2])
    errors, count, F = run_face_model(N, T, P, n_cta=5, seed=3 + order, order=order, n=n)
    assert not errors, errors[:5]
    assert np.all(count == 1)
    assert np.all(F == T - 1)


def test_face_buffer_period_shorter_than_the_grid_is_caught():
    # the model must see a wrapped index reused before its reader took it
    N, T, n = (40, 20, 37), 50, (31, 15, 12)
    errors, _, _ = run_face_model(N, T, 12, n_cta=5, seed=4, n=n)
    assert errors
