"""Components, levels and the level-by-level Jacobi (§8) of the CUDA path vs the oracle.

Labels and levels are unique (a component is named by its largest row index, and its
level is its height in the condensation), so they are compared bit for bit; x is
compared with the FP64 tolerance.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import paper_1210_6412_gb300 as R
from paper_1210_6412_gb300 import synth
from tests.gpu_util import TOL_FP64, need_gpu, oracle_solution

pytestmark = pytest.mark.gpu


def _oracle_scc(c, mode=O.PROB01):
    cls = O.partition(c.n, c.rowptr, c.col, c.val, c.goal, mode)
    q, a, b = O.extract_system(c.n, c.rowptr, c.col, c.val, cls)
    lab = O.scc_labels(a)
    return a, lab, O.scc_levels(a, lab)


CHAINS = {
    "random": lambda: synth.random_chain(n=3000, deg=3, goal_frac=0.02, sink_frac=0.05, seed=11),
    "random_dense": lambda: synth.random_chain(n=2048, deg=16, seed=12),
    "layered": lambda: synth.layered_chain(layers=40, width=200, seed=13),
    "layered_dag": lambda: synth.layered_chain(layers=60, width=150, p_forward=1.0, seed=14),
    "cascade": lambda: synth.cascade_chain(blocks=24, width=300, seed=15),
    "skewed": lambda: synth.skewed_chain(n=6000, hubs=4, hub_deg=2500, seed=16),
    "gambler": lambda: synth.gamblers_ruin(N=300, p=0.45),
    "worked": synth.worked_chain,
}


@pytest.mark.parametrize("name", sorted(CHAINS))
@pytest.mark.parametrize("driver", ["persistent", "graph", "host"])
def test_labels_and_levels_bit_exact(name, driver, monkeypatch):
    """Three drivers of the same passes: cooperative launches with grid barriers (default),
    conditional-while graphs (REACH_SCC_GRAPH=1), and host-driven loops."""
    need_gpu()
    if driver != "persistent":
        monkeypatch.setenv("REACH_SCC_GRAPH", "1")
    if driver == "host":
        monkeypatch.setenv("REACH_HOST_LOOPS", "1")
    c = CHAINS[name]()
    a, lab_o, lev_o = _oracle_scc(c)
    with R.Solver(c.n, c.rowptr, c.col, c.val, c.goal) as s:
        lab, lev, info = s.scc()
    assert info["exact"] == 1
    assert info["n_q"] == a.shape[0]
    assert np.array_equal(lab, lab_o)
    assert np.array_equal(lev, lev_o)
    assert info["n_scc"] == np.unique(lab_o).size
    assert info["n_levels"] == (int(lev_o.max()) + 1 if lev_o.size else 0)
    sizes = np.unique(lab_o, return_counts=True)[1]
    assert info["n_trivial"] == int(np.sum(sizes == 1))
    assert info["largest"] == (int(sizes.max()) if sizes.size else 0)


@pytest.mark.parametrize("name", sorted(CHAINS))
@pytest.mark.parametrize("driver", ["cluster", "grid", "graph"])
def test_level_by_level_jacobi_matches_oracle(name, driver, monkeypatch):
    """Three drivers of the level loop: small levels on one thread-block cluster and big
    ones on a cooperative grid (default), the cooperative grid for every level
    (REACH_SCC_CLUSTER=0), and the conditional-while graph of sweep + apply
    (REACH_SCC_GRAPH=1)."""
    need_gpu()
    if driver == "graph":
        monkeypatch.setenv("REACH_SCC_GRAPH", "1")
    if driver == "grid":
        monkeypatch.setenv("REACH_SCC_CLUSTER", "0")
    c = CHAINS[name]()
    cls_o, x_o = oracle_solution(c)
    with R.Solver(c.n, c.rowptr, c.col, c.val, c.goal) as s:
        x, info = s.solve("scc_jacobi", eps=1e-14, max_iter=5_000_000)
        x2, info2 = s.solve("scc_jacobi", eps=1e-14, max_iter=5_000_000)   # cached decomposition
    assert info["status"] == R.REACH_OK
    assert np.max(np.abs(x - x_o)) <= TOL_FP64
    assert np.array_equal(x, x2)
    assert info["iters"] == info2["iters"]


@pytest.mark.parametrize("graph", [False, True])
def test_sweep_count_matches_oracle_block_jacobi(graph, monkeypatch):
    """Same levels, same stopping rule per level: the sweep counts agree (the oracle spends
    one extra confirming sweep on each level of single-row components)."""
    need_gpu()
    if graph:
        monkeypatch.setenv("REACH_SCC_GRAPH", "1")
    c = CHAINS["cascade"]()
    cls = O.partition(c.n, c.rowptr, c.col, c.val, c.goal)
    q, a, b = O.extract_system(c.n, c.rowptr, c.col, c.val, cls)
    lab = O.scc_labels(a)
    lev = O.scc_levels(a, lab)
    eps = 1e-11
    xq, sweeps, nl, ok = O.block_jacobi(O.system_matrix(a), b, eps, 1_000_000, lab, lev)
    assert ok
    acyclic = sum(1 for h in range(nl) if np.unique(lab[lev == h]).size == np.count_nonzero(lev == h))
    with R.Solver(c.n, c.rowptr, c.col, c.val, c.goal) as s:
        x, info = s.solve("scc_jacobi", eps=eps, max_iter=1_000_000)
    assert info["status"] == R.REACH_OK
    assert abs(info["iters"] - (sweeps - acyclic)) <= 2 * nl // 10 + 2
    assert np.max(np.abs(x[q] - xq)) <= 1e-9


def _cycle_chain_system(L):
    """L three-row cycles; cycle k feeds cycle k - 1.  The largest indices sit upstream,
    so each colouring round resolves one cycle only: L rounds are needed."""
    rows, cols, vals = [], [], []
    for k in range(L):
        a, b, c = 3 * k, 3 * k + 1, 3 * k + 2
        for r, t in ((a, b), (b, c), (c, a)):
            rows.append(r), cols.append(t), vals.append(-1.0)
        if k > 0:
            rows.append(a), cols.append(3 * (k - 1)), vals.append(-1.0)
    n = 3 * L
    rows += list(range(n))
    cols += list(range(n))
    vals += [4.0] * n
    m = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    m.sort_indices()
    b = np.linspace(1.0, 2.0, n)
    return m, b


@pytest.mark.parametrize("graph", [False, True])
def test_round_cap_merges_the_core_and_still_solves(graph, monkeypatch):
    """Past the round cap the cyclic core is kept as one block: the order stays valid
    (every edge leaves a level for a lower one or stays in its block) and the solve is
    unchanged.  Without the cap every cycle is found, one per round."""
    need_gpu()
    if graph:
        monkeypatch.setenv("REACH_SCC_GRAPH", "1")
    L = 40
    m, b = _cycle_chain_system(L)
    lab_o = O.scc_labels(m)
    lev_o = O.scc_levels(m, lab_o)
    x_o = O.dense_solve(m, b)
    args = (m.shape[0], m.indptr.astype(np.int64), m.indices.astype(np.int32), m.data, b)
    with R.Solver.system(*args) as sol:
        lab, lev, info = sol.scc(max_rounds=3)
        x, sinfo = sol.solve("scc_jacobi", eps=1e-15, max_iter=1_000_000)
    assert info["exact"] == 0 and info["rounds"] == 3
    assert np.unique(lab).size == 1                   # nothing was trimmed: one block
    assert sinfo["status"] == R.REACH_OK
    assert np.max(np.abs(x - x_o)) <= 1e-12
    with R.Solver.system(*args) as sol:
        lab, lev, info = sol.scc()
        x, sinfo = sol.solve("scc_jacobi", eps=1e-15, max_iter=1_000_000)
    assert info["exact"] == 1 and info["rounds"] == L
    assert np.array_equal(lab, lab_o) and np.array_equal(lev, lev_o)
    assert info["n_levels"] == L
    assert np.max(np.abs(x - x_o)) <= 1e-12


def test_merged_core_order_is_valid_on_a_cascade():
    need_gpu()
    c = CHAINS["cascade"]()
    a, lab_o, lev_o = _oracle_scc(c)
    cls_o, x_o = oracle_solution(c)
    with R.Solver(c.n, c.rowptr, c.col, c.val, c.goal) as s:
        lab, lev, info = s.scc(max_rounds=1)
        x, sinfo = s.solve("scc_jacobi", eps=1e-14, max_iter=5_000_000)
    a = sp.coo_matrix(a)
    off = a.row != a.col
    i, j = a.row[off], a.col[off]
    same = lab[i] == lab[j]
    assert np.all(lev[i][same] == lev[j][same])
    assert np.all(lev[i][~same] > lev[j][~same])
    # every block is a union of true components
    for L in np.unique(lab_o):
        assert np.unique(lab[lab_o == L]).size == 1
    if info["exact"]:
        assert np.array_equal(lab, lab_o)
    assert sinfo["status"] == R.REACH_OK
    assert np.max(np.abs(x - x_o)) <= TOL_FP64


def test_general_system_components():
    need_gpu()
    s = synth.diag_dominant_system(n=1500, density=0.002, seed=5)
    m = sp.csr_matrix((s.val, s.col, s.rowptr), shape=(s.n, s.n))
    lab_o = O.scc_labels(m)
    lev_o = O.scc_levels(m, lab_o)
    x_o = O.dense_solve(m, s.b)
    with R.Solver.system(s.n, s.rowptr, s.col, s.val, s.b) as sol:
        lab, lev, info = sol.scc()
        x, sinfo = sol.solve("scc_jacobi", eps=1e-14, max_iter=5_000_000)
    assert np.array_equal(lab, lab_o) and np.array_equal(lev, lev_o)
    assert sinfo["status"] == R.REACH_OK
    assert np.max(np.abs(x - x_o)) <= 1e-9 * max(1.0, float(np.max(np.abs(x_o))))


def test_empty_system_and_device_outputs():
    torch = need_gpu()
    c = synth.worked_chain()
    goal = np.ones(c.n, np.uint8)                    # every state a goal: S? is empty
    with R.Solver(c.n, c.rowptr, c.col, c.val, goal) as s:
        lab, lev, info = s.scc()
        x, sinfo = s.solve("scc_jacobi", eps=1e-12)
    assert info["n_q"] == 0 and lab.size == 0 and lev.size == 0
    assert np.all(x == 1.0)
    c = CHAINS["layered"]()
    a, lab_o, lev_o = _oracle_scc(c)
    with R.Solver(c.n, c.rowptr, c.col, c.val, c.goal) as s:
        lab_d = torch.empty(a.shape[0], dtype=torch.int32, device="cuda")
        lev_d = torch.empty(a.shape[0], dtype=torch.int32, device="cuda")
        R.reach_scc(s.ctx, out_label=lab_d, out_level=lev_d)
    assert np.array_equal(lab_d.cpu().numpy(), lab_o)
    assert np.array_equal(lev_d.cpu().numpy(), lev_o)


@pytest.mark.parametrize("graph", [False, True])
def test_max_iter_bounds_the_level_sweeps(graph, monkeypatch):
    need_gpu()
    if graph:
        monkeypatch.setenv("REACH_SCC_GRAPH", "1")
    c = CHAINS["cascade"]()
    with R.Solver(c.n, c.rowptr, c.col, c.val, c.goal) as s:
        with pytest.raises(R.ReachError) as ei:
            s.solve("scc_jacobi", eps=1e-14, max_iter=10)
    assert ei.value.status == R.REACH_ENOTCONV


def test_scc_argument_and_state_errors():
    need_gpu()
    c = CHAINS["random"]()
    ctx = R.reach_create(c.n, c.rowptr, c.col, c.val, c.goal)
    try:
        with pytest.raises(R.ReachError) as ei:
            R.reach_scc(ctx)
        assert ei.value.status == R.REACH_ESTATE            # before reach_precompute
        R.reach_precompute(ctx)
        with pytest.raises(R.ReachError) as ei:
            R.reach_scc(ctx, max_rounds=-1)
        assert ei.value.status == R.REACH_EINVAL
        lab, lev, info = R.reach_scc(ctx)
        assert info["exact"] == 1 and info["passes"] > 0
        # a new precompute (another partition) drops the decomposition
        R.reach_precompute(ctx, R.REACH_PROB0_ONLY)
        lab2, lev2, info2 = R.reach_scc(ctx)
        a, lab_o, lev_o = _oracle_scc(c, O.PROB0_ONLY)
        assert np.array_equal(lab2, lab_o) and np.array_equal(lev2, lev_o)
    finally:
        R.reach_destroy(ctx)


def test_level_by_level_jacobi_warm_start():
    need_gpu()
    c = CHAINS["cascade"]()
    cls_o, x_o = oracle_solution(c)
    with R.Solver(c.n, c.rowptr, c.col, c.val, c.goal) as s:
        x, info = s.solve("scc_jacobi", eps=1e-14, max_iter=5_000_000)
        x2, info2 = s.solve("scc_jacobi", eps=1e-12, max_iter=5_000_000, x0=x)
    assert info2["status"] == R.REACH_OK
    assert info2["iters"] < info["iters"]
    assert np.max(np.abs(x2 - x_o)) <= TOL_FP64
