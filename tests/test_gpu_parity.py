"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Classes (S=0 / S=1 / S?) must match bit for bit; x within 1e-9 absolute for the FP64
methods and 1e-6 for the mixed-precision form.  Sizes span several CTAs and leave
ragged tails; the edge cases of the method (empty S?, empty goal set, single state,
duplicate / unsorted / zero entries, invalid chains) are covered too.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import paper_1210_6412_gb300 as R
from paper_1210_6412_gb300 import synth
from tests import brute
from tests.gpu_util import TOL_FP64, TOL_MIXED, gpu_solve, need_gpu, oracle_solution

pytestmark = pytest.mark.gpu

METHODS = [("jacobi", TOL_FP64), ("mixed", TOL_MIXED), ("bicgstab", TOL_FP64)]
MODES = [O.PROB01, O.PROB0_ONLY]


def _eps(method):
    return 1e-13 if method != "mixed" else 1e-10


@pytest.fixture(scope="module")
def c1():
    return synth.random_chain(n=4096, deg=16, goal_frac=0.02, sink_frac=0.02)


@pytest.mark.parametrize("method,tol", METHODS)
def test_worked_chain(method, tol):
    with open(os.path.join(os.path.dirname(__file__), "golden", "worked_chain.json")) as f:
        g = json.load(f)
    c = synth.worked_chain()
    cls, x, info = gpu_solve(c, O.PROB01, method, _eps(method))
    assert np.flatnonzero(cls == 0).tolist() == g["S0"]
    assert np.flatnonzero(cls == 1).tolist() == g["S1"]
    assert np.flatnonzero(cls == 2).tolist() == g["Sq"]
    np.testing.assert_allclose(x[g["Sq"]], g["x_Sq"], atol=tol, rtol=0)
    assert x[1] == 0.0 and x[3] == 1.0
    assert info["n_q"] == 2 and info["m_q"] == 2


@pytest.mark.parametrize("method,tol", METHODS)
@pytest.mark.parametrize("mode", MODES)
def test_config_small_random_chain(c1, method, tol, mode):
    """4096 states, 16 successors, 2% goals, 2% sinks (the small random-chain workload)."""
    cls_o, x_o = oracle_solution(c1, mode)
    cls, x, info = gpu_solve(c1, mode, method, _eps(method))
    assert np.array_equal(cls, cls_o)
    assert np.max(np.abs(x - x_o)) <= tol
    assert info["status"] == R.REACH_OK and info["iters"] > 0
    assert info["resid_inf"] < 1e-9


@pytest.mark.parametrize("N,p", [(20, 0.4), (60, 0.5), (33, 0.55)])
@pytest.mark.parametrize("method,tol", METHODS)
def test_gamblers_ruin(N, p, method, tol):
    c = synth.gamblers_ruin(N, p)
    want = np.array([brute.gambler_closed_form(N, p, i) for i in range(N + 1)])
    cls, x, info = gpu_solve(c, O.PROB01, method, 1e-14 if method != "mixed" else 1e-12)
    assert cls[0] == 0 and cls[N] == 1 and np.all(cls[1:N] == 2)
    assert np.max(np.abs(x - want)) <= tol


@pytest.mark.parametrize("n,m", synth.TABLE1_QUICKSORT[::4] + synth.TABLE1_BIASED_DIE[::4])
@pytest.mark.parametrize("method,tol", METHODS)
def test_table1_shapes(n, m, method, tol):
    c = synth.table1_chain(n, m)
    cls_o, x_o = oracle_solution(c)
    cls, x, _ = gpu_solve(c, O.PROB01, method, _eps(method))
    assert np.array_equal(cls, cls_o)
    assert np.max(np.abs(x - x_o)) <= tol


@pytest.mark.parametrize("method,tol", METHODS)
def test_layered_chain(method, tol):
    c = synth.layered_chain(layers=60, width=300, seed=11)
    cls_o, x_o = oracle_solution(c)
    cls, x, _ = gpu_solve(c, O.PROB01, method, _eps(method))
    assert np.array_equal(cls, cls_o)
    assert np.max(np.abs(x - x_o)) <= tol


@pytest.mark.parametrize("method,tol", METHODS)
def test_dense_chain_with_sinks(method, tol):
    """Long rows (about 200 entries): the vector-load row kernels."""
    c = synth.dense_random_chain(n=2000, density=0.1, goal_frac=0.01, sink_frac=0.02, seed=5)
    cls_o, x_o = oracle_solution(c)
    cls, x, _ = gpu_solve(c, O.PROB01, method, _eps(method))
    assert np.array_equal(cls, cls_o)
    assert np.max(np.abs(x - x_o)) <= tol


def test_dense_chain_without_sinks_is_degenerate():
    """No sinks: every state reaches GS almost surely, so S=1 = S and x = 1."""
    c = synth.dense_random_chain(n=3000, density=0.1, goal_frac=0.01, seed=6)
    cls, x, info = gpu_solve(c, O.PROB01, "jacobi", 1e-12)
    assert np.all(cls == 1) and np.all(x == 1.0) and info["n_q"] == 0
    cls_o = O.partition(c.n, c.rowptr, c.col, c.val, c.goal)
    assert np.array_equal(cls, cls_o)
    # the same matrix in PROB0_ONLY mode iterates to x -> 1
    for method, tol in METHODS:
        cls0, x0, info0 = gpu_solve(c, O.PROB0_ONLY, method, 1e-13 if method != "mixed" else 1e-11)
        assert info0["n_q"] == c.n - int(c.goal.sum())
        assert np.max(np.abs(x0 - 1.0)) <= tol, method


@pytest.mark.parametrize("method,tol", METHODS)
def test_device_pointers_match_host_pointers(c1, method, tol):
    _, xh, ih = gpu_solve(c1, O.PROB01, method, _eps(method))
    _, xd, idd = gpu_solve(c1, O.PROB01, method, _eps(method), device=True)
    assert np.array_equal(xh, xd) and ih["iters"] == idd["iters"]


def test_host_loops_match_device_loops(c1, monkeypatch):
    _, xa, ia = gpu_solve(c1, O.PROB01, "jacobi", 1e-12)
    monkeypatch.setenv("REACH_HOST_LOOPS", "1")
    for method, tol in METHODS:
        cls_o, x_o = oracle_solution(c1)
        cls, x, info = gpu_solve(c1, O.PROB01, method, _eps(method))
        assert np.array_equal(cls, cls_o) and np.max(np.abs(x - x_o)) <= tol
    _, xb, ib = gpu_solve(c1, O.PROB01, "jacobi", 1e-12)
    assert np.array_equal(xa, xb) and ia["iters"] == ib["iters"]


def test_warm_start_and_iteration_cap(c1):
    cls_o, x_o = oracle_solution(c1)
    torch = need_gpu()
    with R.Solver(c1.n, c1.rowptr, c1.col, c1.val, c1.goal) as s:
        x, info = s.solve("jacobi", eps=1e-12, max_iter=4, refine_k=2, check=False)
        assert info["status"] == R.REACH_ENOTCONV and info["iters"] == 4
        # resuming from the last iterate (the checkpoint) converges to the same answer
        x2, info2 = s.solve("jacobi", eps=1e-13, x0=x)
        assert np.max(np.abs(x2 - x_o)) <= TOL_FP64
        # starting at the solution stops at the first check
        x3, info3 = s.solve("jacobi", eps=1e-10, x0=x_o, refine_k=2)
        assert info3["iters"] == 2 and np.max(np.abs(x3 - x_o)) <= 1e-10
        x4, info4 = s.solve("bicgstab", eps=1e-12, max_iter=1, check=False)
        assert info4["status"] in (R.REACH_ENOTCONV, R.REACH_OK)
    del torch


@pytest.mark.parametrize("name", ["random", "skewed", "dense", "gambler", "table1", "layered"])
def test_segmented_jacobi_matches_oracle(c1, name):
    """The entry-balanced sweep (segmented reduction) gives the FP64 Jacobi answer:
    long rows spanning many tiles, rows without off-diagonal entries, a ragged last tile."""
    c = {"random": lambda: c1,
         "skewed": lambda: synth.skewed_chain(n=20000, hub_deg=9000),
         "dense": lambda: synth.dense_random_chain(n=2000, density=0.1, sink_frac=0.02, seed=5),
         "gambler": lambda: synth.gamblers_ruin(40, 0.45),
         "table1": lambda: synth.table1_chain(1333, 2665),
         "layered": lambda: synth.layered_chain(layers=60, width=300, seed=11)}[name]()
    cls_o, x_o = oracle_solution(c)
    cls, x, info = gpu_solve(c, O.PROB01, "jacobi_seg", 1e-13)
    _, xj, ij = gpu_solve(c, O.PROB01, "jacobi", 1e-13)
    assert np.array_equal(cls, cls_o)
    assert np.max(np.abs(x - x_o)) <= TOL_FP64
    assert abs(info["iters"] - ij["iters"]) <= 16 and info["resid_inf"] < 1e-11


@pytest.mark.parametrize("name", ["skewed", "random"])
@pytest.mark.parametrize("method", ["jacobi", "jacobi_seg"])
def test_fixed_sweep_count_matches_oracle_iterate(c1, name, method):
    """After exactly 32 sweeps from x = 0 (the first solve of a fresh context, so any
    setup done inside that solve is covered) the iterate and the last step size match the
    oracle's Jacobi after 32 sweeps."""
    c = {"random": lambda: c1, "skewed": lambda: synth.skewed_chain(n=20000, hub_deg=9000)}[name]()
    cls = O.partition(c.n, c.rowptr, c.col, c.val, c.goal)
    q, a, b = O.extract_system(c.n, c.rowptr, c.col, c.val, cls)
    xq, it, delta, ok = O.jacobi(O.system_matrix(a), b, 0.0, 32)
    need_gpu()
    with R.Solver(c.n, c.rowptr, c.col, c.val, c.goal) as s:
        x, info = s.solve(method, eps=1e-300, max_iter=32, refine_k=16, check=False)
    assert info["status"] == R.REACH_ENOTCONV and info["iters"] == 32
    assert np.max(np.abs(x[q] - xq)) <= 1e-13
    assert abs(info["last_delta"] - delta) <= 1e-9 * delta + 1e-15


@pytest.mark.parametrize("method,tol", METHODS)
def test_autotune_then_solve(c1, method, tol):
    """The autotuner's pick (timed on a fresh solve state, even after a finished solve)
    is a valid mapping, and solves with it still match the oracle."""
    cls_o, x_o = oracle_solution(c1)
    need_gpu()
    with R.Solver(c1.n, c1.rowptr, c1.col, c1.val, c1.goal) as s:
        s.solve("jacobi", eps=1e-12)                 # leaves the device state 'done'
        t = s.autotune(method)
        assert t["lanes"] in (1, 2, 4, 8, 16, 32, 48, 64, 66, 128) and t["sweep_ms"] > 0
        x, info = s.solve(method, eps=_eps(method))
        assert np.max(np.abs(x - x_o)) <= tol
        for k in ("jacobi64", "sweep32", "resid_mixed", "bicgstab_spmv"):
            assert R.reach_time_kernel(s.ctx, k, 3) > 0.0


def test_jacobi_monotone_from_below(c1):
    """Iterates from x = 0 never decrease and never pass x* (A >= 0, b >= 0)."""
    cls_o, x_o = oracle_solution(c1)
    prev = np.zeros(c1.n)
    with R.Solver(c1.n, c1.rowptr, c1.col, c1.val, c1.goal) as s:
        for it in (2, 4, 8, 16, 32):
            x, _ = s.solve("jacobi", eps=1e-300, max_iter=it, refine_k=2, check=False)
            assert np.all(x >= prev - 1e-15) and np.all(x <= x_o + 1e-12)
            prev = x


# ------------------------------------------------------------------ edge cases

def _chain(rows, goal):
    """Chain from a list of {col: prob} rows (input order kept)."""
    rowptr = [0]
    col, val = [], []
    for r in rows:
        for k, v in r:
            col.append(k)
            val.append(v)
        rowptr.append(len(col))
    return synth.Chain(n=len(rows), rowptr=np.array(rowptr, np.int64), col=np.array(col, np.int32),
                       val=np.array(val, np.float64), goal=np.array(goal, np.uint8))


@pytest.mark.parametrize("method", ["jacobi", "mixed", "bicgstab"])
def test_single_state(method):
    for goal, want in ((1, 1.0), (0, 0.0)):
        c = _chain([[(0, 1.0)]], [goal])
        cls, x, info = gpu_solve(c, O.PROB01, method, 1e-12)
        assert x.tolist() == [want] and info["n_q"] == 0


def test_empty_goal_set(c1):
    c = synth.Chain(c1.n, c1.rowptr, c1.col, c1.val, np.zeros(c1.n, np.uint8))
    cls, x, info = gpu_solve(c, O.PROB01, "bicgstab", 1e-12)
    assert np.all(cls == 0) and np.all(x == 0.0)


def test_all_goal_states(c1):
    c = synth.Chain(c1.n, c1.rowptr, c1.col, c1.val, np.ones(c1.n, np.uint8))
    cls, x, _ = gpu_solve(c, O.PROB0_ONLY, "jacobi", 1e-12)
    assert np.all(cls == 1) and np.all(x == 1.0)


def test_unsorted_duplicate_and_zero_entries():
    # state 0: successors stored out of order, 2 split into two entries, an explicit zero to 1
    c = _chain([[(3, 0.25), (2, 0.125), (1, 0.0), (0, 0.25), (2, 0.375)],
                [(1, 1.0)], [(0, 0.4), (1, 0.6)], [(3, 1.0)]], [0, 0, 0, 1])
    cls_o, x_o = oracle_solution(c)
    for method, tol in METHODS:
        cls, x, _ = gpu_solve(c, O.PROB01, method, 1e-14)
        assert np.array_equal(cls, cls_o) and np.max(np.abs(x - x_o)) <= tol


@pytest.mark.parametrize("bad", ["negative", "nan", "col", "rowsum", "rowptr"])
def test_invalid_chains_are_rejected(bad):
    need_gpu()
    c = synth.worked_chain()
    rowptr, col, val = c.rowptr.copy(), c.col.copy(), c.val.copy()
    if bad == "negative":
        val[0], val[1] = -0.5, 1.5
    elif bad == "nan":
        val[0] = np.nan
    elif bad == "col":
        col[0] = 4
    elif bad == "rowsum":
        val[0] = 0.6
    elif bad == "rowptr":
        rowptr[1], rowptr[2] = 3, 2
    with pytest.raises(R.ReachError) as ei:
        R.reach_create(c.n, rowptr, col, val, c.goal)
    assert ei.value.status == R.REACH_EINVAL


def test_solve_before_precompute_is_a_state_error():
    need_gpu()
    c = synth.worked_chain()
    s = R.Solver(c.n, c.rowptr, c.col, c.val, c.goal, precompute=False)
    with pytest.raises(R.ReachError) as ei:
        s.solve()
    assert ei.value.status == R.REACH_ESTATE
    with pytest.raises(R.ReachError) as ei:
        s.grad(0)
    assert ei.value.status == R.REACH_ESTATE
    s.close()


def test_injected_allocation_failure(monkeypatch):
    need_gpu()
    monkeypatch.setenv("REACH_FAULT_ENOMEM", "1")
    c = synth.worked_chain()
    with pytest.raises(R.ReachError) as ei:
        R.reach_create(c.n, c.rowptr, c.col, c.val, c.goal)
    assert ei.value.status == R.REACH_ENOMEM


@pytest.mark.parametrize("name", ["skewed", "random", "dense", "gambler"])
@pytest.mark.parametrize("method,tol", [("jacobi", TOL_FP64), ("mixed", TOL_MIXED), ("bicgstab", TOL_FP64)])
def test_entry_balanced_layout_matches_oracle(c1, name, method, tol, monkeypatch):
    """REACH_LANES=128: FP64 Jacobi, both kernels of the mixed method (FP64 residual, FP32
    sweep) and the two BiCGStab products on entry-balanced tiles instead of a row mapping."""
    monkeypatch.setenv("REACH_LANES", "128")
    c = {"random": lambda: c1,
         "skewed": lambda: synth.skewed_chain(n=20000, hub_deg=9000),
         "dense": lambda: synth.dense_random_chain(n=2000, density=0.1, sink_frac=0.02, seed=5),
         "gambler": lambda: synth.gamblers_ruin(40, 0.45)}[name]()
    cls_o, x_o = oracle_solution(c)
    cls, x, info = gpu_solve(c, O.PROB01, method, 1e-11 if method == "mixed" else 1e-13)
    assert np.array_equal(cls, cls_o)
    assert info["status"] == R.REACH_OK
    assert np.max(np.abs(x - x_o)) <= tol


@pytest.mark.parametrize("lanes", ["1", "2", "4"])
@pytest.mark.parametrize("name", ["layered", "random", "gambler"])
@pytest.mark.parametrize("method,tol", [("jacobi", TOL_FP64), ("mixed", TOL_MIXED), ("bicgstab", TOL_FP64)])
def test_short_row_mappings_match_oracle(c1, name, lanes, method, tol, monkeypatch):
    """REACH_LANES=1 (one thread per row, as in §5.1), 2 and 4 on short rows: the row
    dots load a batch of entries per lane before using them, with the slots past the row
    end predicated off; rows of 1 to 4 entries and rows longer than one batch both occur."""
    monkeypatch.setenv("REACH_LANES", lanes)
    c = {"random": lambda: c1,
         "layered": lambda: synth.layered_chain(layers=40, width=300, seed=11),
         "gambler": lambda: synth.gamblers_ruin(40, 0.45)}[name]()
    cls_o, x_o = oracle_solution(c)
    cls, x, info = gpu_solve(c, O.PROB01, method, 1e-11 if method == "mixed" else 1e-13)
    assert np.array_equal(cls, cls_o)
    assert info["status"] == R.REACH_OK
    assert np.max(np.abs(x - x_o)) <= tol


@pytest.mark.parametrize("lanes", ["48", "64", "72"])
@pytest.mark.parametrize("name", ["dense", "skewed", "random"])
@pytest.mark.parametrize("method,tol", [("jacobi", TOL_FP64), ("mixed", TOL_MIXED), ("bicgstab", TOL_FP64)])
def test_vector_row_mappings_match_oracle(c1, name, lanes, method, tol, monkeypatch):
    """REACH_LANES=48 (half a warp per row) and 64 (a warp per row), both with 16-byte
    loads of four indices and four values after a scalar head that aligns the row; 72: as
    64, with the mixed method's FP32 sweep reading its vector from shared memory."""
    monkeypatch.setenv("REACH_LANES", lanes)
    c = {"random": lambda: c1,
         "skewed": lambda: synth.skewed_chain(n=20000, hub_deg=9000),
         "dense": lambda: synth.dense_random_chain(n=2000, density=0.1, sink_frac=0.02, seed=5)}[name]()
    cls_o, x_o = oracle_solution(c)
    cls, x, info = gpu_solve(c, O.PROB01, method, 1e-11 if method == "mixed" else 1e-13)
    assert np.array_equal(cls, cls_o)
    assert info["status"] == R.REACH_OK
    assert np.max(np.abs(x - x_o)) <= tol


def test_autotuner_may_pick_entry_balanced_tiles():
    """On a chain with a few very long rows the entry-balanced tiles are a candidate of the
    autotuner for the FP32 sweep and the FP64 sweep; whatever it picks solves correctly."""
    c = synth.skewed_chain(n=200_000, hubs=8, hub_deg=60_000, seed=3)
    cls_o = O.partition(c.n, c.rowptr, c.col, c.val, c.goal)
    need_gpu()
    with R.Solver(c.n, c.rowptr, c.col, c.val, c.goal) as s:
        picks = {m: s.autotune(m)["lanes"] for m in ("jacobi", "mixed", "bicgstab")}
        xj, ij = s.solve("jacobi", eps=1e-12, max_iter=1_000_000)
        xm, im = s.solve("mixed", eps=1e-11, max_iter=1_000_000)
        xb, ib = s.solve("bicgstab", eps=1e-12, max_iter=10_000)
    assert all(p in (1, 2, 4, 8, 16, 32, 48, 64, 66, 72, 128) for p in picks.values())
    assert ij["status"] == R.REACH_OK and im["status"] == R.REACH_OK and ib["status"] == R.REACH_OK
    assert np.max(np.abs(xj - xm)) <= TOL_MIXED and np.max(np.abs(xj - xb)) <= 1e-9


@pytest.mark.parametrize("name", ["dense", "random", "skewed", "gambler"])
def test_bulk_copy_staged_sweep_matches_oracle(c1, name, monkeypatch):
    """REACH_LANES=80: the mixed method's FP32 sweep with each row staged through shared
    memory by bulk copies (segments aligned to 8 entries, neighbour entries masked)."""
    monkeypatch.setenv("REACH_LANES", "80")
    c = {"random": lambda: c1,
         "skewed": lambda: synth.skewed_chain(n=20000, hub_deg=9000),
         "dense": lambda: synth.dense_random_chain(n=3000, density=0.1, sink_frac=0.02, seed=6),
         "gambler": lambda: synth.gamblers_ruin(40, 0.45)}[name]()
    cls_o, x_o = oracle_solution(c)
    cls, x, info = gpu_solve(c, O.PROB01, "mixed", 1e-11)
    assert info["status"] == R.REACH_OK
    assert np.max(np.abs(x - x_o)) <= TOL_MIXED
    with R.Solver(c.n, c.rowptr, c.col, c.val, c.goal) as s:
        ms = R.reach_time_kernel(s.ctx, "sweep32", 3)
    assert ms > 0.0


# the search's level kernels: narrow levels on the cluster with shared-memory queues or with
# global ones, no cluster at all, no bottom-up levels
BFS_VARIANTS = [
    {"REACH_BFS_CLUSTER": "1", "REACH_BFS_LQ": "1", "REACH_BFS_PULL": "1"},
    {"REACH_BFS_CLUSTER": "1", "REACH_BFS_LQ": "0", "REACH_BFS_PULL": "1"},
    {"REACH_BFS_CLUSTER": "0", "REACH_BFS_LQ": "1", "REACH_BFS_PULL": "1"},
    {"REACH_BFS_CLUSTER": "1", "REACH_BFS_LQ": "1", "REACH_BFS_PULL": "0"},
]


@pytest.mark.parametrize("name", ["layered", "dense", "gambler", "random", "dense_layered", "dense_no_sinks"])
def test_partition_with_and_without_the_cluster_search(c1, name, monkeypatch):
    """The backward searches of §2.2 run their narrow levels on one thread-block cluster,
    others top-down on the whole GPU and wide ones bottom-up; with each of these switched
    off in turn they give the oracle's S=0 / S=1 / S? exactly, in both partition modes."""
    c = {"random": lambda: c1,
         "layered": lambda: synth.layered_chain(layers=300, width=200, seed=12),
         "dense": lambda: synth.dense_random_chain(n=3000, density=0.1, sink_frac=0.02, seed=7),
         "gambler": lambda: synth.gamblers_ruin(500, 0.48),
         # 40 successors per state, 30 layers: starts bottom-up and gives up after 8 levels
         # every state reaches a goal: S=0 is empty and the S=1 search has no sources
         "dense_no_sinks": lambda: synth.dense_random_chain(n=2000, density=0.05, sink_frac=0.0, seed=8),
         "dense_layered": lambda: synth.layered_chain(layers=30, width=64, dmin=33, dmax=48, p_forward=1.0,
                                                      goal_frac_last=0.05, seed=13)}[name]()
    need_gpu()
    for mode in MODES:
        cls_o = O.partition(c.n, c.rowptr, c.col, c.val, c.goal, mode)
        for env in BFS_VARIANTS:
            for k, v in env.items():
                monkeypatch.setenv(k, v)
            with R.Solver(c.n, c.rowptr, c.col, c.val, c.goal, mode=mode) as s:
                assert np.array_equal(s.classes(), cls_o), (name, mode, env)


def _fan_chain(fan, depth):
    """State 0 is the goal; states 1..fan step into it (probability 1/2) and otherwise stay
    (the first half) or fall into an absorbing sink (the second half); behind each of them a
    path of `depth` states leads forward to it; the last fan/8 states of the paths lead only
    to the sink instead.  The first backward level finds `fan` states in one go (one state's
    reversed row), the next ones `fan` states per level."""
    n = 2 + fan * (depth + 1)
    sink = n - 1
    rows = [[(0, 1.0)]]
    for i in range(1, fan + 1):
        rows.append([(0, 0.5), (i if i <= fan // 2 else sink, 0.5)])
    for d in range(1, depth + 1):
        for i in range(1, fan + 1):
            s = d * fan + i
            nxt = (d - 1) * fan + i
            rows.append([(nxt, 1.0)] if i <= fan - fan // 8 or d < depth else [(sink, 1.0)])
    rows.append([(sink, 1.0)])
    assert len(rows) == n
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([c for r in rows for c, _ in r], np.int32)
    val = np.array([v for r in rows for _, v in r], np.float64)
    goal = np.zeros(n, np.uint8)
    goal[0] = 1
    return synth.Chain(n=n, rowptr=rp, col=col, val=val, goal=goal)


@pytest.mark.parametrize("fan,depth", [(40_000, 3), (12_000, 40), (200, 300)])
def test_partition_through_full_local_queues(fan, depth, monkeypatch):
    """A level that finds more states than a CTA's shared-memory queue holds (they spill to
    the global queue), frontiers that leave the cluster for the whole GPU, and a long run of
    narrow levels: classes against the oracle in both modes."""
    need_gpu()
    c = _fan_chain(fan, depth)
    for mode in MODES:
        cls_o = O.partition(c.n, c.rowptr, c.col, c.val, c.goal, mode)
        for env in BFS_VARIANTS:
            for k, v in env.items():
                monkeypatch.setenv(k, v)
            with R.Solver(c.n, c.rowptr, c.col, c.val, c.goal, mode=mode) as s:
                assert np.array_equal(s.classes(), cls_o), (fan, depth, mode, env)
