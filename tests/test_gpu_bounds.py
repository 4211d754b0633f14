"""The certified error bound of every solve (reach_info.err_bound) against the oracle.

For M = I - A on S? (§2.3), ||x* - x|| <= ||M^-1|| ||b - M x||.  The library bounds ||M^-1||
by Varah's row-dominance margin (at precompute) or by an approximate tau = M^-1 1
(reach_norm_bound), and the residual by its computed value plus a rounding allowance.
Checks: the bound holds against the oracle's exact solution for every method; it agrees
with the oracle's own bounds evaluated at the GPU's x (varah_bound, error_bound); the
norm bound from tau matches the closed form max_i i (N - i) of the fair gambler's ruin and
the oracle's dense ||M^-1||; it is infinite exactly when no bound is available.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import paper_1210_6412_gb300 as R
from paper_1210_6412_gb300 import synth
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

METHODS = (("jacobi", 1e-12), ("mixed", 1e-10), ("bicgstab", 1e-12), ("jacobi_seg", 1e-12),
           ("scc_jacobi", 1e-12))


def _system(c, mode=O.PROB01):
    cls = O.partition(c.n, c.rowptr, c.col, c.val, c.goal, mode)
    q, a, b = O.extract_system(c.n, c.rowptr, c.col, c.val, cls)
    return cls, q, O.system_matrix(a), b


def test_varah_bound_on_a_chain_where_every_state_exits():
    """Dense chain, PROB0_ONLY: every S? row has goal successors, so the margin is positive
    and every solve comes with a finite bound that covers its true error."""
    need_gpu()
    c = synth.dense_random_chain(n=2048, density=0.10, goal_frac=0.10, seed=5)
    cls, q, m, b = _system(c, O.PROB0_ONLY)
    margin = O.varah_margin(m)
    assert margin > 0
    xs = O.dense_solve(m, b)
    with R.Solver(c.n, c.rowptr, c.col, c.val, c.goal, mode=R.REACH_PROB0_ONLY) as s:
        for meth, eps in METHODS:
            x, info = s.solve(meth, eps=eps)
            err = float(np.max(np.abs(x[q] - xs)))
            bound = info["err_bound"]
            assert np.isfinite(bound) and err <= bound, (meth, err, bound)
            want = O.varah_bound(m, b, x[q])             # the oracle's bound at the GPU's x
            # the library adds only the rounding allowance of its residual (tiny here)
            assert want * (1 - 1e-9) <= bound <= want * (1 + 1e-6) + 1e-13 / margin, (meth, bound, want)


def test_bound_is_infinite_without_a_margin_until_norm_bound():
    """Sinks and goals reached only through other states: some rows cannot leave S? in one
    step, Varah's margin is 0 and no bound exists -- until reach_norm_bound certifies
    ||M^-1|| from tau, after which every solve's bound holds and is close to the oracle's
    exact-tau bound."""
    need_gpu()
    c = synth.random_chain(n=1500, deg=8, goal_frac=0.03, sink_frac=0.03, seed=12)
    cls, q, m, b = _system(c)
    assert O.varah_margin(m) <= 0
    xs = O.dense_solve(m, b)
    tau = O.dense_solve(m, np.ones(q.size))
    with R.Solver(c.n, c.rowptr, c.col, c.val, c.goal) as s:
        x, info = s.solve("jacobi", eps=1e-12)
        assert info["err_bound"] == np.inf
        k, tinfo = s.norm_bound("bicgstab", eps=1e-10)
        assert tinfo["status"] == R.REACH_OK
        assert tau.max() * (1 - 1e-12) <= k <= tau.max() * (1 + 1e-6), (k, tau.max())
        for meth, eps in METHODS:
            x, info = s.solve(meth, eps=eps)
            err = float(np.max(np.abs(x[q] - xs)))
            bound = info["err_bound"]
            assert err <= bound, (meth, err, bound)
            want = O.error_bound(m, b, x[q])             # exact ||M^-1|| times the residual
            assert want * (1 - 1e-9) <= bound <= want * (1 + 1e-5) + 1e-13 * tau.max(), (meth, bound, want)


@pytest.mark.parametrize("method", ["jacobi", "mixed", "bicgstab"])
def test_norm_bound_of_the_fair_gamblers_ruin(method):
    """Fair walk on 0..N: ||M^-1||_inf = max_i i (N - i) exactly (the expected duration)."""
    need_gpu()
    N = 64
    c = synth.gamblers_ruin(N, 0.5)
    exact = (N // 2) * ((N + 1) // 2)
    with R.Solver(c.n, c.rowptr, c.col, c.val, c.goal) as s:
        k, info = s.norm_bound(method, eps=1e-9)
        assert exact <= k <= exact * (1 + 1e-6), (k, exact)
        x, sinfo = s.solve("bicgstab", eps=1e-13)
        want = np.arange(N + 1) / N
        err = float(np.max(np.abs(x - want)))
        assert err <= sinfo["err_bound"] <= 1e-8


def test_norm_bound_keeps_the_system_and_the_last_solution():
    """The tau solve borrows the right-hand side: b is restored (a later solve gives the
    same x) and the last solution stays available to reach_grad."""
    need_gpu()
    c = synth.random_chain(n=800, deg=6, goal_frac=0.04, sink_frac=0.04, seed=3)
    with R.Solver(c.n, c.rowptr, c.col, c.val, c.goal) as s:
        x1, _ = s.solve("jacobi", eps=1e-13)
        g1, _ = s.grad(c.init)
        s.norm_bound("jacobi", eps=1e-9)
        g2, _ = s.grad(c.init)
        x2, _ = s.solve("jacobi", eps=1e-13)
    assert np.array_equal(x1, x2)
    assert np.array_equal(g1, g2)


def test_norm_bound_cap_still_certifies():
    """A tau solve stopped by max_iter returns a looser but still valid bound."""
    need_gpu()
    c = synth.random_chain(n=1000, deg=8, goal_frac=0.03, sink_frac=0.03, seed=8)
    cls, q, m, b = _system(c)
    tau = O.dense_solve(m, np.ones(q.size))
    with R.Solver(c.n, c.rowptr, c.col, c.val, c.goal) as s:
        k, info = s.norm_bound("jacobi", eps=1e-12, max_iter=40)
        assert info["status"] == R.REACH_ENOTCONV
        assert k >= tau.max() * (1 - 1e-12)


def test_general_system_varah_bound():
    """The diagonally dominant random systems of §6: Varah's bound covers every solve; the
    tau bound is refused (M^-1 >= 0 does not hold there)."""
    need_gpu()
    sysm = synth.diag_dominant_system(n=1200, density=0.01, seed=4)
    m = sp.csr_matrix((sysm.val, sysm.col, sysm.rowptr), shape=(sysm.n, sysm.n))
    xs = O.dense_solve(m, sysm.b)
    with R.Solver.system(sysm.n, sysm.rowptr, sysm.col, sysm.val, sysm.b) as s:
        for meth, eps in (("jacobi", 1e-12), ("bicgstab", 1e-12)):
            x, info = s.solve(meth, eps=eps)
            err = float(np.max(np.abs(x - xs)))
            assert np.isfinite(info["err_bound"]) and err <= info["err_bound"], meth
            want = O.varah_bound(m, sysm.b, x)
            assert want * (1 - 1e-9) <= info["err_bound"] <= want * (1 + 1e-6) + 1e-12
        with pytest.raises(R.ReachError) as ei:
            s.norm_bound()
        assert ei.value.status == R.REACH_ESTATE


def test_adjoint_bound_on_the_worked_chain():
    """Worked chain of §2: A = [[0, .5], [.4, 0]] has column margins 0.6 and 0.5, so the
    adjoint y of (I - A)^T y = e_0 gets a finite bound that covers its error."""
    need_gpu()
    c = synth.worked_chain()
    cls, q, m, b = _system(c)
    y = O.dense_solve(m.T.tocsr(), np.array([1.0, 0.0]))
    g_o, _, _ = O.grad_p(c.n, c.rowptr, c.col, c.val, c.goal, 0)
    with R.Solver(c.n, c.rowptr, c.col, c.val, c.goal) as s:
        s.solve("jacobi", eps=1e-15)
        g, info = s.grad(0, eps=1e-6)
    assert np.isfinite(info["err_bound"]) and info["err_bound"] <= 1e-5
    # gradient entries are y_s x_s' with x exact to ~1e-15 and x <= 1
    assert np.max(np.abs(g - g_o)) <= info["err_bound"] + 1e-14
    assert info["err_bound"] >= 0.0 and y.size == 2
