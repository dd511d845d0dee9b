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
