"""The seeded random-geometry generator of the batched workload.

Every problem it returns holds the bodies it drew (1 to 3), each at least 3
cells of the stretched grid from the box, the bodies at least 3 local cells
apart, and the oracle finds irregular points on it.  Checked for every seed
the benchmark's batch, the batch, parity and ILU tests and the learned part
use, so none of them runs on a body-free domain."""
import numpy as np
import pytest

from oracle import pyoracle as O
from paper_1901_08269_gb300 import workloads as W

BATCH_SEED = 20261203

SEEDS = ([(s, (33, 49, 65, 97, 129)) for s in range(BATCH_SEED, BATCH_SEED + 64)]
         + [(s, (33, 41, 49)) for s in list(range(100, 106)) + [7, 11]]
         + [(s, (33, 49)) for s in (3, 8)]
         + [(s, (33,)) for s in list(range(6)) + [100, 101]]
         + [(s, (65, 97, 129)) for s in range(1000, 1016)])


def _box_cells(grid, lo, hi):
    """Whole cells between the box ends and the interval [lo, hi]."""
    below = int(np.searchsorted(grid, lo, side="right")) - 1
    above = grid.size - int(np.searchsorted(grid, hi, side="left"))
    return below, above - 1


@pytest.mark.parametrize("seed,sizes", SEEDS)
def test_random_problem_has_bodies_and_irregular_points(seed, sizes):
    w = W.random_problem(seed, sizes=sizes)
    assert 1 <= len(w.bodies) <= 3
    axes = (w.x, w.y, w.z)
    for b in w.bodies:
        rad = max(b["p"])
        for d in range(3):
            lo, hi = b["c"][d] - rad, b["c"][d] + rad
            below, above = _box_cells(axes[d], lo, hi)
            assert below >= 3 and above >= 3, (seed, d, below, above)
    for a in range(len(w.bodies)):
        for c in range(a):
            ca, cc = np.asarray(w.bodies[a]["c"]), np.asarray(w.bodies[c]["c"])
            assert np.linalg.norm(ca - cc) > max(w.bodies[a]["p"]) + max(w.bodies[c]["p"])
    P = O.Problem(w.x, w.y, w.z, w.bodies)
    t = P.classify()
    assert P.n_irr > 0 and P.n_ibi > 0
    assert np.count_nonzero(t == O.SOLID) > 0


def test_random_problem_is_deterministic():
    a, b = W.random_problem(BATCH_SEED + 5), W.random_problem(BATCH_SEED + 5)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.z, b.z)
    assert [x["c"] for x in a.bodies] == [x["c"] for x in b.bodies]


def test_random_problem_raises_when_nothing_fits():
    # a grid of 9 nodes per axis leaves no interval 3 cells from both box
    # ends wide enough for a body of radius >= 0.1
    with pytest.raises(ValueError):
        W.random_problem(0, sizes=(9,))
