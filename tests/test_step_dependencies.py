"""Which strips a two-buffer step tile reads from, against the strips its items wait for (CPU).

A warp tile of strip s reads the previous step's post-collision values:
- the staged columns x0 - 1 .. x0 + W (W = strip width): its pulls;
- the pulled rho u_r of the columns beside the strip, which reach one
  column further (x0 - 2, x0 + W + 1);
- with periodic ends, the pulled rho u_r of column nx - 1 (columns nx - 2 ..
  nx, for column 0) and of column 0 (columns -1 .. 1, for column nx - 1).
Ghost columns are written by the edge node whose value the rule copies:
- column nx by column 0 (periodic), else by column nx - 1;
- column -1 by column nx - 1 (periodic), else by column 0 (inlet).
A tile only uses a beside value if the node next to it lies on the
lattice.  The persistent launch orders a tile after the tiles one strip
away (wrapped for periodic ends), or two strips away when the step kernel's
far-wrap condition holds: periodic ends, a one-column last strip, four
strips or more.  This model checks that every strip a tile depends on lies
within that distance, and that the wider wait is needed exactly there.
"""
import pytest


def writer_strip(col, nx, W, periodic):
    """Strip whose previous step wrote column col (-1 .. nx) of the stored state."""
    if col == nx:
        col = 0 if periodic else nx - 1
    elif col == -1:
        col = nx - 1 if periodic else 0
    return col // W


def needed_strips(s, nx, W, periodic):
    ns = -(-nx // W)
    x0, last = s * W, min(s * W + W, nx) - 1
    cols = set(range(x0 - 1, last + 2))  # the tile's own pulls
    if x0 > 0:  # the left beside node x0 - 1 is on the lattice
        cols |= {x0 - 2, x0 - 1, x0}
    if last + 1 < nx:  # the right beside node
        cols |= {last, last + 1, last + 2}
    if periodic:
        if x0 == 0:
            cols |= {nx - 2, nx - 1, nx}
        if last == nx - 1:
            cols |= {-1, 0, 1}
    return {writer_strip(c, nx, W, periodic) for c in cols if -1 <= c <= nx}, ns


def far_wrap(periodic, nx, nstrips, W):
    return periodic and (nx - 1) % W == 0 and nstrips >= 4


def distance(a, b, ns, periodic):
    d = abs(a - b)
    return min(d, ns - d) if periodic else d


@pytest.mark.parametrize("W", [32, 64])
@pytest.mark.parametrize("periodic", [False, True])
def test_tiles_depend_only_on_strips_their_items_wait_for(W, periodic):
    for nx in range(2, 12 * W + 3):
        ns = -(-nx // W)
        far = far_wrap(periodic, nx, ns, W)
        widest = 0
        for s in range(ns):
            strips, _ = needed_strips(s, nx, W, periodic)
            widest = max(widest, max(distance(s, t, ns, periodic) for t in strips))
        assert widest <= (2 if far else 1), (nx, W, periodic)
        if far:
            assert widest == 2, (nx, W)  # the wider wait is needed exactly where it is taken
