"""Parity at the full workload sizes.

The dense random chain (n = 32768, 10% density, about 107M entries) is the benchmark
workload.  The layered 8M-state chain, the 4M-state parametric chain and the 256-chain
batch (67M states, 1.1G entries) are the other full configurations; together they take a
few minutes, most of it generating the batch on the host.

Where the oracle cannot solve the full system in seconds the check uses facts that hold
at any size: the exact solution x* = 1 certified by the S=0/S=1 partition, or the
a-posteriori bound ||x* - x|| <= ||b - M x|| / min_i (M_ii - sum_j |M_ij|) for the strictly
diagonally dominant M = I - A (Varah's bound), with the residual computed by the oracle.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import paper_1210_6412_gb300 as R
from paper_1210_6412_gb300 import synth
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

EPS = {"jacobi": 5e-12, "mixed": 5e-12, "bicgstab": 5e-12}    # the benchmark's thresholds


def _dev(torch, *arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def _certified_error(c, cls, x):
    """Varah bound on max|x* - x| over S? from the oracle's residual of the GPU x."""
    q, a, b = O.extract_system(c.n, c.rowptr, c.col, c.val, cls)
    m = O.system_matrix(a)
    r = b - m @ x[q]
    margin = np.min(1.0 - a @ np.ones(q.size))          # M_ii - sum_j |M_ij| = exit probability
    assert margin > 0
    return float(np.max(np.abs(r)) / margin)


@pytest.fixture(scope="module")
def dense():
    return synth.dense_random_chain(n=32768, density=0.10, goal_frac=0.01)


def test_bench_workload_full(dense):
    """The benchmark system at full size, in the benchmark's launch configuration."""
    torch = need_gpu()
    c = dense
    cls01_o = O.partition(c.n, c.rowptr, c.col, c.val, c.goal, O.PROB01)
    cls0_o = O.partition(c.n, c.rowptr, c.col, c.val, c.goal, O.PROB0_ONLY)
    assert np.all(cls01_o == O.S1)                      # x* = 1 everywhere
    d_in = _dev(torch, c.rowptr, c.col, c.val, c.goal)
    with R.Solver(c.n, *d_in, mode=R.REACH_PROB01) as s:
        assert np.array_equal(s.classes(), cls01_o)
    with R.Solver(c.n, *d_in, mode=R.REACH_PROB0_ONLY) as s:
        assert np.array_equal(s.classes(), cls0_o)
        kinv, _ = s.norm_bound("bicgstab", eps=1e-8)
        assert np.isfinite(kinv)
        for meth in ("jacobi", "mixed", "bicgstab"):
            s.autotune(meth)
            x, info = s.solve(meth, eps=EPS[meth], max_iter=200_000, refine_k=16,
                              out=torch.empty(c.n, dtype=torch.float64, device="cuda"))
            err = float(torch.max(torch.abs(x - 1.0)))
            assert info["status"] == R.REACH_OK and err <= 1e-9, (meth, err)
            # the certified bound covers the true error and certifies the target accuracy
            assert err <= info["err_bound"] <= 1e-9, (meth, err, info["err_bound"])


def test_dense_with_sinks_full():
    """Same shape with 2% absorbing states: non-trivial x, certified from the residual."""
    torch = need_gpu()
    c = synth.dense_random_chain(n=32768, density=0.10, goal_frac=0.01, sink_frac=0.02, seed=91)
    cls_o = O.partition(c.n, c.rowptr, c.col, c.val, c.goal)
    with R.Solver(c.n, *_dev(torch, c.rowptr, c.col, c.val, c.goal)) as s:
        assert np.array_equal(s.classes(), cls_o)
        for meth, tol in (("jacobi", 1e-9), ("mixed", 1e-6), ("bicgstab", 1e-9)):
            x, info = s.solve(meth, eps=1e-12 if meth != "mixed" else 1e-10)
            assert _certified_error(c, cls_o, x) <= tol, meth
            assert np.all((x >= 0) & (x <= 1))


def test_layered_full():
    torch = need_gpu()
    c = synth.layered_chain()
    cls_o = O.partition(c.n, c.rowptr, c.col, c.val, c.goal)
    q, a, b = O.extract_system(c.n, c.rowptr, c.col, c.val, cls_o)
    xq, it, _, ok = O.jacobi(O.system_matrix(a), b, 1e-14, 200_000)
    x_o = O.full_vector(c.n, cls_o, q, xq)
    with R.Solver(c.n, *_dev(torch, c.rowptr, c.col, c.val, c.goal)) as s:
        assert np.array_equal(s.classes(), cls_o)
        kinv, _ = s.norm_bound("bicgstab", eps=1e-8)
        for meth, tol in (("jacobi", 1e-9), ("mixed", 1e-6), ("bicgstab", 1e-9)):
            x, info = s.solve(meth, eps=1e-13 if meth != "mixed" else 1e-11)
            err = np.max(np.abs(x - x_o))
            assert err <= tol, meth
            # certified against the exact solution, which the oracle's x approximates to 1e-12
            assert err <= info["err_bound"] + 1e-12 and info["err_bound"] <= tol, (meth, info["err_bound"])


def test_parametric_full():
    torch = need_gpu()
    from paper_1210_6412_gb300.autograd import reach_prob
    pc = synth.parametric_chain()
    args = _dev(torch, pc.rowptr, pc.col, pc.cls, pc.offset, pc.goal)
    theta = torch.from_numpy(pc.theta).cuda().requires_grad_(True)
    y = reach_prob(theta, *args, pc.init, eps=1e-14, adj_eps=1e-15)
    y.backward()
    g = theta.grad.cpu().numpy()
    h = 1e-6
    for j in (0, 17, 40, 63):
        e = np.zeros(64)
        e[j] = h
        with torch.no_grad():
            fp = float(reach_prob(torch.from_numpy(pc.theta + e).cuda(), *args, pc.init, eps=1e-14))
            fm = float(reach_prob(torch.from_numpy(pc.theta - e).cuda(), *args, pc.init, eps=1e-14))
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g[j]) <= 1e-5 * max(abs(fd), 1e-6) + 1e-9, (j, fd, g[j])


def test_batched_full():
    torch = need_gpu()
    bt = synth.batched_chains(sink_frac=0.02)
    n, rowptr, col, val, goals, offs = bt.concat()
    d_in = _dev(torch, rowptr, col, val, goals)
    with R.BatchSolver(n, *d_in, chains=offs) as bs:     # per-chain stopping, as the benchmark
        cls = bs.classes()
        x, info = bs.solve(eps=1e-8)
    assert info["status"] == R.REACH_OK
    sizes = np.diff(offs)
    picks = list(np.argsort(sizes)[:3]) + [int(np.argsort(sizes)[len(sizes) // 2])]
    for ci in picks:
        c, g = bt.chains[ci], bt.goals[ci]
        a, b = int(offs[ci]), int(offs[ci + 1])
        for j in range(g.shape[0]):
            x_o, cls_o, _ = O.reach_probabilities(c.n, c.rowptr, c.col, c.val, g[j], method="jacobi",
                                                  eps=1e-13, max_iter=1_000_000)
            assert np.array_equal(cls[j, a:b], cls_o)
            assert np.max(np.abs(x[j, a:b] - x_o)) <= 1e-6
