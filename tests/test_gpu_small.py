"""The cluster-resident solvers of small systems (one launch, matrix in shared memory)
against the oracle and against the graph-driven solvers (REACH_SMALL=0).

Systems of up to a few thousand unknowns -- the random 4096-state chain, the Table 1
state-space sizes, gambler's ruins, the worked chain of §2 -- take this path by default
for the mixed method, and for FP64 Jacobi up to 10240 stored entries (REACH_SMALL=1 makes
FP64 Jacobi take it whenever it fits, as these tests do).  Both paths must give the oracle's x within the
method's tolerance, the same stopping behaviour (checks every refine_k sweeps), and honour
max_iter and warm starts.
"""
import numpy as np
import pytest

import oracle as O
import paper_1210_6412_gb300 as R
from paper_1210_6412_gb300 import synth
from tests import brute
from tests.gpu_util import TOL_FP64, TOL_MIXED, need_gpu, oracle_solution

pytestmark = pytest.mark.gpu

CASES = {
    "random4096": lambda: synth.random_chain(n=4096, deg=16, goal_frac=0.02, sink_frac=0.02),
    "table1_die": lambda: synth.table1_chain(7647, 15293),
    "table1_qs": lambda: synth.table1_chain(92, 211),
    "dense2000": lambda: synth.dense_random_chain(n=2000, density=0.1, goal_frac=0.01, sink_frac=0.02, seed=5),
    "layered": lambda: synth.layered_chain(layers=20, width=150, seed=3),
    "worked": synth.worked_chain,
    "single": lambda: synth.gamblers_ruin(2, 0.5),
}


def _solve(c, method, eps, monkeypatch, small, **kw):
    monkeypatch.setenv("REACH_SMALL", "1" if small else "0")
    with R.Solver(c.n, c.rowptr, c.col, c.val, c.goal) as s:
        return s.solve(method, eps=eps, **kw)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("method,tol,eps", [("jacobi", TOL_FP64, 1e-13), ("mixed", TOL_MIXED, 1e-10)])
def test_small_solver_matches_oracle_and_graph_solver(name, method, tol, eps, monkeypatch):
    need_gpu()
    c = CASES[name]()
    cls_o, x_o = oracle_solution(c)
    x_s, i_s = _solve(c, method, eps, monkeypatch, True)
    x_g, i_g = _solve(c, method, eps, monkeypatch, False)
    assert i_s["status"] == R.REACH_OK and i_g["status"] == R.REACH_OK
    assert np.max(np.abs(x_s - x_o)) <= tol, name
    assert np.max(np.abs(x_g - x_o)) <= tol, name
    # same rule, same check period: the sweep counts agree up to one period
    k = 16
    assert abs(i_s["iters"] - i_g["iters"]) <= k, (i_s["iters"], i_g["iters"])
    assert i_s["err_bound"] >= 0.0


@pytest.mark.parametrize("N,p", [(20, 0.4), (60, 0.5)])
def test_small_solver_gamblers_ruin_closed_form(N, p, monkeypatch):
    need_gpu()
    c = synth.gamblers_ruin(N, p)
    want = np.array([brute.gambler_closed_form(N, p, i) for i in range(N + 1)])
    x, info = _solve(c, "jacobi", 1e-14, monkeypatch, True, max_iter=5_000_000)
    assert np.max(np.abs(x - want)) <= TOL_FP64
    x, info = _solve(c, "mixed", 1e-12, monkeypatch, True, max_iter=5_000_000)
    assert np.max(np.abs(x - want)) <= TOL_MIXED


@pytest.mark.parametrize("method", ["jacobi", "mixed"])
def test_small_solver_iteration_cap_and_warm_start(method, monkeypatch):
    need_gpu()
    c = CASES["random4096"]()
    cls_o, x_o = oracle_solution(c)
    monkeypatch.setenv("REACH_SMALL", "1")
    with R.Solver(c.n, c.rowptr, c.col, c.val, c.goal) as s:
        x, info = s.solve(method, eps=1e-14, max_iter=20, refine_k=4, check=False)
        assert info["status"] == R.REACH_ENOTCONV and info["iters"] <= 20 + 4
        if method == "jacobi":
            assert info["iters"] == 20
        x2, info2 = s.solve(method, eps=1e-13 if method == "jacobi" else 1e-10, x0=x)
        assert info2["status"] == R.REACH_OK
        assert np.max(np.abs(x2 - x_o)) <= (TOL_FP64 if method == "jacobi" else TOL_MIXED)
        # from the solution: stops at the first check
        x3, info3 = s.solve(method, eps=1e-9, x0=x_o, refine_k=4)
        assert info3["iters"] <= 4 and np.max(np.abs(x3 - x_o)) <= 1e-9


def test_small_solver_fixed_sweeps_equal_the_oracle_iterate(monkeypatch):
    """Sixteen sweeps from 0 with an unreachable eps: the oracle's sixteenth iterate."""
    need_gpu()
    c = CASES["random4096"]()
    cls = O.partition(c.n, c.rowptr, c.col, c.val, c.goal)
    q, a, b = O.extract_system(c.n, c.rowptr, c.col, c.val, cls)
    xo, _, _, _ = O.jacobi(O.system_matrix(a), b, 0.0, 16)
    x, info = _solve(c, "jacobi", 1e-300, monkeypatch, True, max_iter=16, refine_k=16, check=False)
    assert info["iters"] == 16
    assert np.max(np.abs(x[q] - xo)) <= 1e-13
