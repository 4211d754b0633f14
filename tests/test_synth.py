"""The seeded generators produce well-formed chains of the stated shapes (no GPU)."""
import numpy as np
import pytest

import oracle as O
from paper_1210_6412_gb300 import synth


def _well_formed(c, distinct=True):
    O.check_chain(c.n, c.rowptr, c.col, c.val, c.goal, tol=1e-12)
    assert c.rowptr.dtype == np.int64 and c.col.dtype == np.int32 and c.val.dtype == np.float64
    assert c.goal.dtype == np.uint8
    if distinct:
        for i in np.linspace(0, c.n - 1, 50).astype(int):
            row = c.col[c.rowptr[i]:c.rowptr[i + 1]]
            assert np.all(np.diff(row) > 0)


def test_random_chain_shape_and_determinism():
    a = synth.random_chain(n=1000, deg=16, seed=1)
    b = synth.random_chain(n=1000, deg=16, seed=1)
    _well_formed(a)
    assert np.array_equal(a.col, b.col) and np.array_equal(a.val, b.val)
    deg = np.diff(a.rowptr)
    sinks = (deg == 1) & (a.col[a.rowptr[:-1]] == np.arange(1000))
    assert sinks.sum() == 20 and a.goal.sum() == 20
    assert np.all(deg[~sinks] == 16)
    assert a.goal[0] == 0 and not sinks[0]


def test_dense_random_chain_density():
    c = synth.dense_random_chain(n=2048, density=0.1, seed=2)
    _well_formed(c)
    assert abs(c.m / (2048 * 2048) - 0.1) < 0.005
    assert c.goal.sum() == round(0.01 * 2048)


def test_layered_chain_structure():
    layers, width = 50, 200
    c = synth.layered_chain(layers=layers, width=width, seed=3)
    _well_formed(c)
    deg = np.diff(c.rowptr)
    row = np.repeat(np.arange(c.n), deg)
    sink = (deg == 1) & (c.col[c.rowptr[:-1]] == np.arange(c.n)) & (c.val[c.rowptr[:-1]] == 1.0)
    # 5% drawn sinks, plus the odd degree-1 state whose only successor is itself
    assert 0 <= sink.sum() - 0.05 * c.n <= 0.005 * c.n
    live = ~sink[row]
    lay_from, lay_to = row[live] // width, c.col[live] // width
    fwd = (lay_to == lay_from + 1) | ((lay_from == layers - 1) & (lay_to == lay_from))
    assert 0.85 < fwd.mean() < 0.95
    assert np.all(lay_to[~fwd] <= lay_from[~fwd])
    # dyadic probabilities
    assert np.all(np.log2(c.val) == np.round(np.log2(c.val)))
    assert set(np.flatnonzero(c.goal) // width) == {layers - 1}


def test_parametric_chain():
    pc = synth.parametric_chain(n=5000, seed=4)
    deg = np.diff(pc.rowptr)
    assert deg.min() >= 1 and deg.max() <= 8
    assert pc.cls.min() >= 0 and pc.cls.max() < 64 and pc.theta.shape == (64,)
    p = O.softmax_probs(pc.rowptr, pc.cls, pc.offset, pc.theta)
    O.check_chain(pc.n, pc.rowptr, pc.col, p, pc.goal, tol=1e-12)


def test_batched_chains_regenerate_and_concat():
    b = synth.batched_chains(n_chains=6, n_min=100, n_max=3000, k=3, seed=9)
    assert len(b.chains) == 6 and b.k == 3
    for c, g in zip(b.chains, b.goals):
        _well_formed(c)
        assert g.shape == (3, c.n) and np.all(g.sum(axis=1) >= 1)
    n, rowptr, col, val, goal, offs = b.concat()
    O.check_chain(n, rowptr, col, val, goal[0])
    assert offs[-1] == n and goal.shape == (3, n)
    b2 = synth.batched_chains(n_chains=6, n_min=100, n_max=3000, k=3, seed=9)
    assert all(np.array_equal(x.val, y.val) for x, y in zip(b.chains, b2.chains))


def test_diag_dominant_system():
    import scipy.sparse as sp
    s = synth.diag_dominant_system(n=1500, density=0.02, seed=3)
    m = sp.csr_matrix((s.val, s.col, s.rowptr), shape=(s.n, s.n))
    d = m.diagonal()
    assert np.all(d > np.abs(m).sum(axis=1).A1 - np.abs(d))          # strictly dominant
    assert np.all(s.val == np.round(s.val)) and np.all(s.val >= 1)   # positive integers
    assert np.all(s.b == np.round(s.b)) and abs(m.nnz / s.n ** 2 - 0.02) < 0.005


@pytest.mark.parametrize("n,m", synth.TABLE1_QUICKSORT[:3] + synth.TABLE1_BIASED_DIE[:2])
def test_table1_shapes(n, m):
    c = synth.table1_chain(n, m)
    _well_formed(c)
    sinks = int(round(0.02 * n)) or 1
    assert abs(c.m - m) <= 2 * sinks + n // 50 + 2


def test_cascade_chain_structure():
    blocks, width = 12, 300
    c = synth.cascade_chain(blocks=blocks, width=width, seed=9)
    _well_formed(c)
    deg = np.diff(c.rowptr)
    row = np.repeat(np.arange(c.n), deg)
    sink = (deg == 1) & (c.col[c.rowptr[:-1]] == np.arange(c.n)) & (c.val[c.rowptr[:-1]] == 1.0)
    live = ~sink[row]
    b_from, b_to = row[live] // width, c.col[live] // width
    assert np.all((b_to == b_from) | (b_to == b_from + 1))          # same block or the next
    stay = (b_to == b_from)[b_from < blocks - 1]
    assert 0.85 < stay.mean() < 0.95
    assert set(np.flatnonzero(c.goal) // width) == {blocks - 1}


def test_skewed_chain_hubs():
    c = synth.skewed_chain(n=5000, hubs=3, hub_deg=1500, seed=10)
    _well_formed(c)
    deg = np.diff(c.rowptr)
    assert np.sum(deg == 1500) == 3 and np.sort(deg)[-4] <= 64
