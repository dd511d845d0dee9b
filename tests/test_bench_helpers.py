"""bench.py's algorithmic byte counts against brute-force enumeration of the
cells a tile step reads and writes (CPU)."""
import itertools
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("tile", sorted(bench.TILE_SHAPES))
@pytest.mark.parametrize("eb", [4, 2])
def test_systolic_bytes_match_enumeration(tile, eb):
    tx, ty, tz = bench.TILE_SHAPES[tile]
    box = set(itertools.product(range(tx), range(ty), range(tz)))
    # the lower shell: cells one step upwind of the box in the skewed frame,
    # i.e. the (tx+1)(ty+1)(tz+1) box shifted down by one, minus the box
    shell = set(itertools.product(range(-1, tx), range(-1, ty), range(-1, tz))) - box
    # the top faces: box cells with a +1 neighbour outside the box
    top = {c for c in box if c[0] == tx - 1 or c[1] == ty - 1 or c[2] == tz - 1}
    want = ((6 * eb + 4.0) * len(shell) + 6.0 * eb * len(top)) / len(box)
    assert bench.systolic_bytes(tile, eb) == pytest.approx(want, rel=1e-12)


def test_default_tile_figures():
    assert bench.systolic_bytes(bench.DEFAULT_TILE, 4) == pytest.approx(9.528, abs=5e-4)
    assert bench.naive_bytes(4) == 76.0 and bench.naive_bytes(2) == 40.0
