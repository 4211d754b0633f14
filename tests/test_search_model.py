"""A host model of the GPU's backward-search levels against the oracle's partition (§2.2).

The device search mixes three kinds of level: top-down over the reversed graph (on one
cluster or the whole GPU) and bottom-up, where every unmarked state reads its own successors
and is marked when one of them is, marks made during a pass already counting for states
read later in the same pass, in whatever order the threads happen to run.  This test runs
that schedule on the host -- random switches between the two kinds, a random order inside
every bottom-up pass, goal states blocked from the start in the S=1 search -- and checks
that the marked sets are the oracle's S=0 and S=1, in both partition modes.  It checks the
reasoning the kernels rely on (every mark is a path to the sources, so the same set is
reached), independently of the GPU.
"""
import numpy as np
import pytest

import oracle as O
from paper_1210_6412_gb300 import synth


def _search(n, rowptr, col, val, sources, blocked, rng):
    """Backward closure of `sources`: states with a path of positive entries into a source,
    never entering a blocked state.  Levels alternate at random between top-down (the
    frontier's reversed rows) and bottom-up passes (unmarked rows read in a random order,
    marks visible within the pass)."""
    rows = [set() for _ in range(n)]   # reversed graph: rows[c] = predecessors of c
    for s in range(n):
        for k in range(rowptr[s], rowptr[s + 1]):
            if val[k] > 0.0:
                rows[col[k]].add(s)
    marked = sources | blocked
    reached = sources.copy()
    frontier = list(np.flatnonzero(sources))
    while frontier:
        found = []
        if rng.random() < 0.5:                       # top-down
            for v in frontier:
                for u in rows[v]:
                    if not marked[u]:
                        marked[u] = reached[u] = True
                        found.append(u)
        else:                                        # bottom-up, marks seen within the pass
            for s in rng.permutation(n):
                if marked[s]:
                    continue
                for k in range(rowptr[s], rowptr[s + 1]):
                    c = col[k]
                    if val[k] > 0.0 and reached[c]:
                        marked[s] = reached[s] = True
                        found.append(s)
                        break
        frontier = found
    return reached


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
@pytest.mark.parametrize("mode", [O.PROB01, O.PROB0_ONLY])
def test_mixed_level_search_gives_the_oracle_partition(seed, mode):
    rng = np.random.default_rng(seed)
    gens = [lambda: synth.random_chain(n=600, deg=3, goal_frac=0.02, sink_frac=0.05, seed=seed),
            lambda: synth.layered_chain(layers=30, width=20, seed=seed),
            lambda: synth.gamblers_ruin(80, 0.45)]
    for make in gens:
        c = make()
        goal = c.goal.astype(bool)
        cls_o = O.partition(c.n, c.rowptr, c.col, c.val, c.goal, mode)
        none = np.zeros(c.n, bool)
        can_reach_goal = _search(c.n, c.rowptr, c.col, c.val, goal, none, rng)
        s0 = ~can_reach_goal
        assert np.array_equal(s0, cls_o == O.S0)
        if mode == O.PROB01:
            # S=1: states that cannot reach S=0 along a path avoiding the goals
            reach_s0 = _search(c.n, c.rowptr, c.col, c.val, s0, goal & ~s0, rng)
            s1 = ~reach_s0 & ~s0
        else:
            s1 = goal & ~s0
        assert np.array_equal(s1, cls_o == O.S1)


def test_a_mistake_in_the_model_is_caught():
    """Letting a blocked goal count as a marked successor in the S=1 search (the bug the
    kernels avoid by reading the goal mask) changes the partition on a chain where a
    state reaches S=0 only through a goal."""
    # 0 -> 1 (goal) -> 2 (sink); 3 -> 0 or 4 (goal, absorbing); 2 and 4 absorb
    rowptr = np.array([0, 1, 2, 3, 5, 6])
    col = np.array([1, 2, 2, 0, 4, 4], np.int32)
    val = np.array([1.0, 1.0, 1.0, 0.5, 0.5, 1.0])
    goal = np.array([0, 1, 0, 0, 1], np.uint8)
    cls_o = O.partition(5, rowptr, col, val, goal, O.PROB01)
    rng = np.random.default_rng(0)
    g = goal.astype(bool)
    s0 = ~_search(5, rowptr, col, val, g, np.zeros(5, bool), rng)
    right = ~_search(5, rowptr, col, val, s0, g & ~s0, rng) & ~s0
    wrong = ~_search(5, rowptr, col, val, s0 | g, np.zeros(5, bool), rng) & ~s0
    assert np.array_equal(right, cls_o == O.S1)
    assert not np.array_equal(wrong, cls_o == O.S1)
