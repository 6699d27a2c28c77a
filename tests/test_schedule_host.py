"""The planner's host scheduling logic, without a GPU: the longest-processing-time
packing of work units onto persistent CTAs (the static form of the paper's Sec. 3.2 task
scheduling) and the split-k choice (Sec. 3.2, Fig. 2), through bsmm_schedule_lpt and
bsmm_schedule_pieces.

References: brute-force optimal makespans on tiny instances (LPT's classical bound of
4/3 - 1/(3m) times the optimum, Graham 1969), the trivial lower bounds, and hand-worked
tie cases."""
import itertools

import numpy as np
import pytest

import paper_1504_05046_gb300 as P


def _loads(cost, ptr, units, bins):
    return [float(sum(cost[u] for u in units[ptr[b]:ptr[b + 1]])) for b in range(bins)]


def test_lpt_ties_and_order():
    # equal costs go to the least-loaded bin, ties to the lowest bin; each bin lists its
    # units in ascending order
    ptr, units, mk = P.bsmm_schedule_lpt([5.0, 5.0, 5.0, 5.0], 2)
    assert ptr.tolist() == [0, 2, 4] and units.tolist() == [0, 2, 1, 3] and mk == 10.0
    # longest first: 7 -> bin 0, 5 -> bin 1, 3 -> bin 1 (5 < 7), 2 -> bin 0 (7 < 8)
    ptr, units, mk = P.bsmm_schedule_lpt([3.0, 7.0, 2.0, 5.0], 2)
    assert ptr.tolist() == [0, 2, 4] and units.tolist() == [1, 2, 0, 3] and mk == 9.0


@pytest.mark.parametrize("seed", range(30))
def test_lpt_is_a_partition_within_grahams_bound(seed):
    rng = np.random.default_rng(seed)
    n, m = int(rng.integers(1, 9)), int(rng.integers(1, 4))
    cost = rng.integers(1, 20, n).astype(float)
    ptr, units, mk = P.bsmm_schedule_lpt(cost, m)
    assert sorted(units.tolist()) == list(range(n))
    for b in range(m):
        seg = units[ptr[b]:ptr[b + 1]].tolist()
        assert seg == sorted(seg)
    loads = _loads(cost, ptr, units, m)
    assert mk == max(loads)
    assert mk >= max(cost.max(), cost.sum() / m) - 1e-9
    opt = min(max(np.bincount(np.array(a), weights=cost, minlength=m)) for a in itertools.product(range(m), repeat=n))
    assert mk <= (4.0 / 3.0 - 1.0 / (3.0 * m)) * opt + 1e-9


def test_pieces_forced_and_never():
    cost = np.array([10.0, 20.0, 30.0, 1.0])
    ln = np.array([5, 1, 0, 100])
    assert P.bsmm_schedule_pieces(cost, ln, 8, 0.0, ksplit=1).tolist() == [1, 1, 1, 1]
    assert P.bsmm_schedule_pieces(cost, ln, 8, 0.0, ksplit=3).tolist() == [3, 1, 1, 3]
    assert P.bsmm_schedule_pieces(cost, ln, 8, 0.0, ksplit=64).tolist() == [5, 1, 1, 64]


def test_pieces_automatic_leaves_balanced_work_alone():
    rng = np.random.default_rng(1)
    cost = rng.uniform(1.0, 2.0, 5000)
    assert (P.bsmm_schedule_pieces(cost, np.full(5000, 50), 76, 0.01) == 1).all()


def _pieces_makespan(cost, pieces, bins, overhead):
    pc = np.concatenate([np.full(k, c / k + (overhead if k > 1 else 0.0)) for c, k in zip(cost, pieces)])
    return P.bsmm_schedule_lpt(pc, bins)[2]


@pytest.mark.parametrize("units,bins", [(32, 76), (256, 1216), (10, 152), (100, 76)])
def test_pieces_automatic_fills_an_idle_grid(units, bins):
    """Few long units: the planner cuts them and the packed makespan drops by at least 10%
    (the rule's threshold) against the uncut packing."""
    rng = np.random.default_rng(units)
    cost = rng.uniform(0.9, 1.1, units) * 1e9
    ln = np.full(units, 4000)
    pieces = P.bsmm_schedule_pieces(cost, ln, bins, 1e6)
    assert ((pieces >= 1) & (pieces <= ln)).all()
    base = P.bsmm_schedule_lpt(cost, bins)[2]
    if units >= bins * 4:
        return
    assert (pieces > 1).any()
    assert _pieces_makespan(cost, pieces, bins, 1e6) <= 0.9 * base


def test_pieces_overhead_and_length_limit_cuts():
    cost = np.full(4, 1e6)
    # an overhead larger than the work: cutting never pays
    assert (P.bsmm_schedule_pieces(cost, np.full(4, 1000), 64, 1e9) == 1).all()
    # k-lists of one block cannot be cut
    assert (P.bsmm_schedule_pieces(cost, np.ones(4, np.int64), 64, 0.0) == 1).all()


def test_invalid_arguments():
    with pytest.raises(P.BsmmError):
        P.bsmm_schedule_lpt([1.0, -1.0], 2)
    with pytest.raises(P.BsmmError):
        P.bsmm_schedule_lpt([1.0], 0)
    with pytest.raises(P.BsmmError):
        P.bsmm_schedule_pieces([1.0], [-1], 4, 0.0)
    with pytest.raises(P.BsmmError):
        P.bsmm_schedule_pieces([1.0], [3], 4, 0.0, ksplit=-1)
