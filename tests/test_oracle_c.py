"""The C build of the oracle's Jacobi and BiCGStab loops (the CPU baseline) pinned on the CPU.

It must reproduce the numpy oracle's iterates (same steps, same summation order), the
worked chain's x = (5/8, 1/4) and the gambler's-ruin closed form, and its Jacobi iterates
must not depend on the number of threads (rows are independent in a sweep).
"""
import numpy as np
import pytest

import oracle as O
from oracle import c_oracle as CO
from paper_1210_6412_gb300 import synth
from tests import brute


def _system(c, mode=O.PROB01):
    cls = O.partition(c.n, c.rowptr, c.col, c.val, c.goal, mode)
    q, a, b = O.extract_system(c.n, c.rowptr, c.col, c.val, cls)
    return q, O.system_matrix(a), b


def test_worked_chain():
    q, m, b = _system(synth.worked_chain())
    x, it, d, ok = CO.jacobi(m, b, 1e-15, 1000)
    assert ok and np.max(np.abs(x - [0.625, 0.25])) < 1e-14
    x, it, r, st = CO.bicgstab(m, b, 1e-15, 100)
    assert st == 0 and np.max(np.abs(x - [0.625, 0.25])) < 1e-14


@pytest.mark.parametrize("N,p", [(20, 0.4), (33, 0.5), (15, 0.7)])
def test_gamblers_ruin_closed_form(N, p):
    c = synth.gamblers_ruin(N, p)
    q, m, b = _system(c)
    want = np.array([brute.gambler_closed_form(N, p, i) for i in q])
    x, it, d, ok = CO.jacobi(m, b, 1e-14, 2_000_000)
    assert ok and np.max(np.abs(x - want)) < 1e-9
    x, it, r, st = CO.bicgstab(m, b, 1e-13, 10 * N)
    assert st == 0 and np.max(np.abs(x - want)) < 1e-9


@pytest.mark.parametrize("sweeps", [1, 7, 40])
def test_jacobi_iterates_equal_the_numpy_oracle(sweeps):
    c = synth.random_chain(n=3000, deg=12, goal_frac=0.02, sink_frac=0.02, seed=5)
    q, m, b = _system(c)
    xo, _, do, _ = O.jacobi(m, b, 0.0, sweeps)
    xc, it, dc, ok = CO.jacobi(m, b, 0.0, sweeps)
    assert it == sweeps and not ok
    assert np.max(np.abs(xc - xo)) <= 1e-15
    assert abs(dc - do) <= 1e-15


def test_jacobi_does_not_depend_on_the_thread_count():
    c = synth.random_chain(n=5000, deg=16, goal_frac=0.02, sink_frac=0.02, seed=6)
    q, m, b = _system(c)
    CO.set_threads(1)
    x1, i1, d1, _ = CO.jacobi(m, b, 1e-12, 100_000)
    CO.set_threads(4)
    x4, i4, d4, _ = CO.jacobi(m, b, 1e-12, 100_000)
    CO.set_threads(0)
    assert i1 == i4 and d1 == d4 and np.array_equal(x1, x4)


@pytest.mark.parametrize("threads", [1, 3])
def test_bicgstab_matches_the_numpy_oracle(threads):
    c = synth.random_chain(n=2000, deg=8, goal_frac=0.03, sink_frac=0.03, seed=7)
    q, m, b = _system(c)
    CO.set_threads(threads)
    xc, ic, rc, st = CO.bicgstab(m, b, 1e-13, 1000)
    CO.set_threads(0)
    xo, io, ro, ok = O.bicgstab(m, b, 1e-13, 1000)
    xs = O.dense_solve(m, b)
    assert st == 0 and ok
    assert np.max(np.abs(xc - xs)) < 1e-10 and np.max(np.abs(xo - xs)) < 1e-10
    assert abs(ic - io) <= 2


def test_bicgstab_restart_and_cap():
    """Table-1 sized chain with a sparse b: q . r can vanish, one restart recovers; a cap
    of 3 iterations reports max_iter."""
    c = synth.table1_chain(92, 211)
    q, m, b = _system(c)
    x, it, r, st = CO.bicgstab(m, b, 1e-14, 500)
    assert st == 0 and np.max(np.abs(x - O.dense_solve(m, b))) < 1e-12
    g = synth.gamblers_ruin(200, 0.5)
    qg, mg, bg = _system(g)
    x, it, r, st = CO.bicgstab(mg, bg, 1e-30, 3)
    assert st == 1 and it == 3


def test_jacobi_cap_and_empty_system():
    g = synth.gamblers_ruin(50, 0.5)
    q, m, b = _system(g)
    x, it, d, ok = CO.jacobi(m, b, 1e-30, 25)
    assert it == 25 and not ok
    xo, _, _, _ = O.jacobi(m, b, 1e-30, 25)
    assert np.max(np.abs(x - xo)) <= 1e-15
    import scipy.sparse as sp
    x, it, d, ok = CO.jacobi(sp.csr_matrix((0, 0)), np.zeros(0), 1e-9, 10)
    assert ok and x.size == 0
