"""The AA in-place layout's cell ownership, checked on the CPU for small lattices.

A value is addressed as "population q arriving at node y" in one of two
representations: slot_0(q, y) = cell(opp(q), y - e_q) and slot_1(q, y) =
cell(q, y).  A step on representation P reads slot_P(q, x) and writes
slot_{1-P}(q, x + e_q) for every node x, and writes the boundary value for
a ghost g to slot_{1-P}(q, g + e_q).  The in-place update is race-free only
if:
- every node writes exactly the cells it reads;
- no two nodes share a cell;
- boundary cells are touched by no node in that step.
After the step, the node's post-collision value is slot_{1-P}(q, x + e_q),
distinct from every boundary cell.  These tests check the three rules and
that last property for every boundary cell a pulled population can need.
"""
import itertools

import pytest

EX = [0, 1, 0, -1, 0, 1, -1, -1, 1, 1, 0, -1, 0]
EY = [0, 0, 1, 0, -1, 1, 1, -1, -1, 0, 1, 0, -1]


def opp(q):
    for m in range(13):
        if (m < 9) == (q < 9) and EX[m] == -EX[q] and EY[m] == -EY[q]:
            return m
    raise AssertionError(q)


def slot(P, q, i, j):
    return (q, i, j) if P else (opp(q), i - EX[q], j - EY[q])


def nodes(nx, nr):
    return [(i, j) for j in range(nr) for i in range(nx)]


@pytest.mark.parametrize("nx,nr", [(1, 1), (2, 3), (5, 4), (7, 2)])
@pytest.mark.parametrize("P", [0, 1])
def test_each_node_writes_exactly_the_cells_it_reads(nx, nr, P):
    owner = {}
    for i, j in nodes(nx, nr):
        reads = {slot(P, q, i, j) for q in range(13)}
        writes = {slot(1 - P, q, i + EX[q], j + EY[q]) for q in range(13)}
        assert reads == writes and len(reads) == 13
        for c in reads:
            assert c not in owner, (c, owner.get(c), (i, j))
            owner[c] = (i, j)


@pytest.mark.parametrize("nx,nr", [(1, 1), (2, 3), (5, 4), (7, 2)])
@pytest.mark.parametrize("P", [0, 1])
def test_boundary_cells_are_nobodys_and_post_values_stay_readable(nx, nr, P):
    inside = set(nodes(nx, nr))
    touched = set()
    for i, j in inside:
        touched |= {slot(P, q, i, j) for q in range(13)}
    # every ghost g whose population q streams into a lattice node (the rules may give it a value)
    boundary = {slot(1 - P, q, gi + EX[q], gj + EY[q])
                for q in range(13) for gi, gj in itertools.product(range(-1, nx + 1), range(-1, nr + 1))
                if (gi, gj) not in inside and (gi + EX[q], gj + EY[q]) in inside}
    assert not boundary & touched  # no node reads or writes a boundary cell in the step
    post = {slot(1 - P, q, i + EX[q], j + EY[q]) for i, j in inside for q in range(13)}
    assert len(post) == 13 * len(inside) and not post & boundary
    # every cell lies inside the ghost ring of the padded planes
    for q, i, j in touched | boundary:
        assert -1 <= i <= nx and -1 <= j <= nr
