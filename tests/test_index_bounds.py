"""Host-side check of the integer derivative pass's division-free periodic
wrap: on every grid that the host sends to the kernel instance wrapping by
one compare and select (near_indices: nx >= BX + 3, ny >= DBY + 3, nz >= 3),
every index that a tile forms lies in [-n, 2n), where that wrap equals the
remainder.  The index sets are restated from the kernel's loops: the
neighbour offsets (i + o, j + o, k + o, |o| <= 3, for every thread of a tile
that starts inside the grid) and the staging of the D_y / D_z sums (x in
i0 - 2 .. i0 + BX + 1, rows j0 - 2 .. j0 + DBY + 1, planes k - 2 .. k + 2)."""
import os
import pathlib
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
COMMON = os.path.join(os.path.dirname(HERE), "paper_2606_02053_gb300", "csrc", "common.cuh")


def constants():
    src = pathlib.Path(COMMON).read_text()
    bx = int(re.search(r"constexpr int BX = (\d+);", src).group(1))
    dby = int(re.search(r"#define COSMOS_DERIV_ROWS (\d+)", src).group(1))
    m = re.search(r"near_indices\(const DevGrid& g\) \{ return g\.nx >= BX \+ (\d+) && g\.ny >= DBY \+ (\d+) "
                  r"&& g\.nz >= (\d+); \}", src)
    assert m, "near_indices changed: restate this test"
    return bx, dby, tuple(int(v) for v in m.groups())


def wrap_near(a, n):
    return np.where(a < 0, a + n, np.where(a >= n, a - n, a))


def indices_along(n, tile):
    """Every index formed along one axis by the tiles (tile = BX along x,
    DBY along y, 1 along z)."""
    starts = np.arange(0, n, tile)
    lanes = np.arange(tile)
    nbr = (starts[:, None, None] + lanes[None, :, None] + np.arange(-3, 4)[None, None, :]).ravel()
    if tile > 1:  # staging: a 2-point halo around the tile, each with +-2 neighbours along y
        stage = (starts[:, None] + np.arange(-2, tile + 2)[None, :]).ravel()
        stage = (stage[:, None] + np.arange(-2, 3)[None, :]).ravel()
    else:
        stage = (starts[:, None] + np.arange(-2, 3)[None, :]).ravel()
    return np.concatenate([nbr, stage])


def test_division_free_wrap_is_exact_wherever_the_host_selects_it():
    bx, dby, (ax, ay, az) = constants()
    for n, tile, lo in ((range(bx + ax, bx + ax + 70), bx, bx + ax), (range(dby + ay, dby + ay + 40), dby, dby + ay),
                        (range(az, az + 20), 1, az)):
        for size in n:
            a = indices_along(size, tile)
            assert a.min() >= -size and a.max() < 2 * size, (size, tile, a.min(), a.max())
            assert np.array_equal(wrap_near(a, size), np.mod(a, size))


def test_the_bound_is_needed_below_the_threshold():
    """On small enough grids a tile's indices leave [-n, 2n), so the remainder
    path the host picks there is needed (the threshold is sufficient, and not
    far from necessary)."""
    bx, dby, _ = constants()
    for size, tile in ((bx // 2, bx), (dby // 2, dby), (2, 1)):
        a = indices_along(size, tile)
        assert a.min() < -size or a.max() >= 2 * size
