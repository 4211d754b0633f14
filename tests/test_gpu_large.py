"""Oracle parity on the code paths that only large systems take.

Above 65536 unknowns the mixed method's kernels read 32-bit column indices instead of
16-bit ones; chains with thousands of BFS levels keep the backward searches on the
thread-block cluster for many levels per launch; a batch whose chains have hundreds of
thousands of states deals rows from chain lists over several windows.  These cases run the
same comparisons as the small parity tests -- classes bit for bit, x within 1e-9 (FP64) or
1e-6 (mixed, batched), gradients against the oracle's adjoint -- at sizes the oracle still
solves in seconds.
"""
import numpy as np
import pytest

import oracle as O
import paper_1210_6412_gb300 as R
from paper_1210_6412_gb300 import synth
from tests.gpu_util import TOL_FP64, TOL_MIXED, need_gpu
from tests.test_gpu_parity import BFS_VARIANTS

pytestmark = pytest.mark.gpu

ALL_METHODS = [("jacobi", TOL_FP64, 1e-13), ("mixed", TOL_MIXED, 1e-10), ("bicgstab", TOL_FP64, 1e-13),
               ("jacobi_seg", TOL_FP64, 1e-13), ("scc_jacobi", TOL_FP64, 1e-13)]


def _oracle(c, mode=O.PROB01, eps=1e-14):
    """Classes and x by the oracle's partition, extraction and Jacobi (§2.2, §2.3, §3.1)."""
    cls = O.partition(c.n, c.rowptr, c.col, c.val, c.goal, mode)
    q, a, b = O.extract_system(c.n, c.rowptr, c.col, c.val, cls)
    m = O.system_matrix(a)
    xq, it, _, ok = O.jacobi(m, b, eps, 1_000_000)
    assert ok
    return cls, O.full_vector(c.n, cls, q, xq), q, m, b


def _dev(torch, *arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


@pytest.fixture(scope="module")
def layered():
    c = synth.layered_chain(layers=400, width=1000)
    return c, _oracle(c)


@pytest.fixture(scope="module")
def wide():
    """100k states with 128 successors each: warp-per-row vector rows with 32-bit indices."""
    c = synth.random_chain(n=100_000, deg=128, goal_frac=0.05, sink_frac=0.05, seed=31)
    return c, _oracle(c, eps=1e-13)


@pytest.mark.parametrize("method,tol,eps", ALL_METHODS)
def test_layered_400k(layered, method, tol, eps):
    torch = need_gpu()
    c, (cls_o, x_o, q, m, b) = layered
    assert q.size > 65536
    with R.Solver(c.n, *_dev(torch, c.rowptr, c.col, c.val, c.goal)) as s:
        assert np.array_equal(s.classes(), cls_o)
        x, info = s.solve(method, eps=eps)
    assert info["status"] == R.REACH_OK
    assert np.max(np.abs(x - x_o)) <= tol, method


@pytest.mark.parametrize("lanes", ["2", "128"])
@pytest.mark.parametrize("method,tol,eps", ALL_METHODS[:3])
def test_layered_400k_other_mappings(layered, lanes, method, tol, eps, monkeypatch):
    torch = need_gpu()
    monkeypatch.setenv("REACH_LANES", lanes)
    c, (cls_o, x_o, q, m, b) = layered
    with R.Solver(c.n, *_dev(torch, c.rowptr, c.col, c.val, c.goal)) as s:
        x, info = s.solve(method, eps=eps)
    assert np.max(np.abs(x - x_o)) <= tol, (lanes, method)


@pytest.mark.parametrize("mode", [O.PROB01, O.PROB0_ONLY])
def test_layered_400k_classes_both_searches(layered, mode, monkeypatch):
    """Hundreds of levels per search, with and without the cluster for narrow levels."""
    torch = need_gpu()
    c, _ = layered
    cls_o = O.partition(c.n, c.rowptr, c.col, c.val, c.goal, mode)
    for env in BFS_VARIANTS:
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        with R.Solver(c.n, *_dev(torch, c.rowptr, c.col, c.val, c.goal), mode=mode) as s:
            assert np.array_equal(s.classes(), cls_o), env


def test_two_thousand_levels_on_the_cluster():
    """2000 layers of 50 states: the backward searches run about 2000 narrow levels."""
    torch = need_gpu()
    c = synth.layered_chain(layers=2000, width=50)
    cls_o, x_o, q, m, b = _oracle(c)
    with R.Solver(c.n, *_dev(torch, c.rowptr, c.col, c.val, c.goal)) as s:
        assert np.array_equal(s.classes(), cls_o)
        for meth, tol, eps in ALL_METHODS[:3]:
            x, info = s.solve(meth, eps=eps)
            assert np.max(np.abs(x - x_o)) <= tol, meth


@pytest.mark.parametrize("lanes", [None, "48", "64", "66", "128"])
@pytest.mark.parametrize("method,tol,eps", ALL_METHODS[:3])
def test_wide_rows_32bit_indices(wide, lanes, method, tol, eps, monkeypatch):
    torch = need_gpu()
    if lanes:
        monkeypatch.setenv("REACH_LANES", lanes)
    c, (cls_o, x_o, q, m, b) = wide
    assert q.size > 65536
    with R.Solver(c.n, *_dev(torch, c.rowptr, c.col, c.val, c.goal)) as s:
        assert np.array_equal(s.classes(), cls_o)
        x, info = s.solve(method, eps=eps)
    assert np.max(np.abs(x - x_o)) <= tol, (lanes, method)


def test_skewed_200k_against_the_oracle():
    """Zipf out-degrees with a few 50,000-entry rows, above 65536 unknowns, every method."""
    torch = need_gpu()
    c = synth.skewed_chain(n=200_000, hubs=8, hub_deg=50_000, seed=9)
    cls_o, x_o, q, m, b = _oracle(c)
    assert q.size > 65536
    with R.Solver(c.n, *_dev(torch, c.rowptr, c.col, c.val, c.goal)) as s:
        assert np.array_equal(s.classes(), cls_o)
        for meth, tol, eps in ALL_METHODS:
            x, info = s.solve(meth, eps=eps)
            assert np.max(np.abs(x - x_o)) <= tol, meth


def test_parametric_300k_gradient_against_the_oracle():
    """Softmax chain of 300k states: x_init and d x_init / d theta against the oracle's
    probabilities, forward solve, adjoint (M^T y = e_init by the oracle's Jacobi) and chain
    rule; then central differences of the GPU forward solve on four classes."""
    torch = need_gpu()
    from paper_1210_6412_gb300.autograd import reach_prob
    pc = synth.parametric_chain(n=300_000, seed=44)
    p = O.softmax_probs(pc.rowptr, pc.cls, pc.offset, pc.theta)
    chain = synth.Chain(n=pc.n, rowptr=pc.rowptr, col=pc.col, val=p, goal=pc.goal, init=pc.init)
    cls, x_o, q, m, b = _oracle(chain, eps=1e-15)
    assert cls[pc.init] == O.SQ and q.size > 65536
    pos = np.searchsorted(q, pc.init)
    y, _, _, ok = O.jacobi(m.T.tocsr(), np.eye(1, q.size, pos).ravel(), 1e-16, 1_000_000)
    assert ok
    row = np.repeat(np.arange(pc.n), np.diff(pc.rowptr))
    g_p = np.zeros(pc.m)
    inq = cls[row] == O.SQ
    qpos = np.full(pc.n, -1)
    qpos[q] = np.arange(q.size)
    g_p[inq] = y[qpos[row[inq]]] * x_o[pc.col[inq]]
    g_o = O.grad_theta(pc.rowptr, p, g_p, pc.cls, pc.theta.size)
    args = _dev(torch, pc.rowptr, pc.col, pc.cls, pc.offset, pc.goal)
    for meth in ("jacobi", "bicgstab"):
        theta = torch.from_numpy(pc.theta).cuda().requires_grad_(True)
        val = reach_prob(theta, *args, pc.init, eps=1e-14, adj_eps=1e-15, method=meth, adj_method=meth)
        val.backward()
        assert abs(float(val) - x_o[pc.init]) <= TOL_FP64
        g = theta.grad.cpu().numpy()
        assert np.max(np.abs(g - g_o)) <= 1e-9 * max(1.0, np.max(np.abs(g_o))), meth
    h = 1e-6
    for j in (0, 9, 33, 63):
        e = np.zeros(pc.theta.size)
        e[j] = h
        with torch.no_grad():
            fp = float(reach_prob(torch.from_numpy(pc.theta + e).cuda(), *args, pc.init, eps=1e-15))
            fm = float(reach_prob(torch.from_numpy(pc.theta - e).cuda(), *args, pc.init, eps=1e-15))
        assert abs((fp - fm) / (2 * h) - g_o[j]) <= 1e-6 * max(abs(g_o[j]), 1e-4), j


def test_batch_with_half_million_state_chains():
    """Three chains of 500k-600k states (8 goal sets each) in one batch, per-chain
    stopping: every class bit for bit; x of two goal sets per chain against the oracle."""
    torch = need_gpu()
    bt = synth.batched_chains(n_chains=3, n_min=500_000, n_max=600_000, sink_frac=0.02, seed=61)
    n, rowptr, col, val, goals, offs = bt.concat()
    with R.BatchSolver(n, *_dev(torch, rowptr, col, val, goals), chains=offs) as bs:
        cls = bs.classes()
        x, info = bs.solve(eps=1e-10)
    assert info["status"] == R.REACH_OK
    for ci, ch in enumerate(bt.chains):
        a, z = int(offs[ci]), int(offs[ci + 1])
        assert ch.n >= 500_000
        for j in range(goals.shape[0]):
            cls_o = O.partition(ch.n, ch.rowptr, ch.col, ch.val, bt.goals[ci][j])
            assert np.array_equal(cls[j, a:z], cls_o), (ci, j)
        for j in (0, goals.shape[0] - 1):
            g = synth.Chain(n=ch.n, rowptr=ch.rowptr, col=ch.col, val=ch.val, goal=bt.goals[ci][j])
            _, x_o, _, _, _ = _oracle(g, eps=1e-12)
            assert np.max(np.abs(x[j, a:z] - x_o)) <= TOL_MIXED, (ci, j)
