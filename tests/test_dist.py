"""The row-split (multi-GPU) Jacobi and BiCGStab loops on the CPU, against the oracle.

Partition and halo plan are checked structurally; the loops run with host arithmetic
(tests/dist_host.py) in one process (LockstepComm, 1 to 4 ranks) and on two gloo CPU
processes (TorchComm).  Jacobi checked every sweep must reproduce the oracle's Jacobi
iterates sweep for sweep; BiCGStab must reach the oracle's solution.
"""
import socket

import numpy as np
import pytest

import oracle as O
from paper_1210_6412_gb300 import dist as D
from paper_1210_6412_gb300 import synth
from tests.dist_host import HostBlockOps, gloo_worker, system_of


def test_partition_rows_balances_work():
    rng = np.random.default_rng(1)
    deg = rng.integers(0, 300, size=1000)
    deg[17] = 20000                                   # one long row
    rowptr = np.concatenate([[0], np.cumsum(deg)])
    cost = deg + 2
    for parts in (1, 2, 3, 7, 16):
        b = D.partition_rows(rowptr, parts)
        assert b[0] == 0 and b[-1] == 1000 and np.all(np.diff(b) >= 1)
        loads = [cost[b[i]:b[i + 1]].sum() for i in range(parts)]
        assert max(loads) <= cost.sum() / parts + cost.max()
    with pytest.raises(ValueError):
        D.partition_rows(rowptr[:3], 3)


@pytest.mark.parametrize("parts", [1, 2, 3, 5])
def test_block_plan_renumbers_columns_and_halo(parts):
    c = synth.random_chain(n=700, deg=9, goal_frac=0.03, sink_frac=0.03, seed=2)
    rp, ci, v, d, b, q, _ = system_of(c)
    nq = rp.size - 1
    bounds = D.partition_rows(rp, parts)
    x = np.random.default_rng(3).random(nq)
    gathered = np.full(parts * int(np.max(np.diff(bounds))), np.nan)
    mr = int(np.max(np.diff(bounds)))
    for r in range(parts):
        gathered[r * mr: r * mr + bounds[r + 1] - bounds[r]] = x[bounds[r]:bounds[r + 1]]
    seen = 0
    for r in range(parts):
        p = D.block_plan(rp, ci, v, d, b, bounds, r)
        # own columns first, then the halo; mapping back gives the original entries
        ids = np.concatenate([p.halo_ids, [-1]])           # (a block without a halo)
        glob = np.where(p.col < p.n_rows, p.col + p.r0, ids[np.maximum(p.col - p.n_rows, 0)])
        lo, hi = rp[p.r0], rp[p.r1]
        assert np.array_equal(glob, ci[lo:hi]) and np.array_equal(p.val, v[lo:hi])
        assert np.all((p.halo_ids < p.r0) | (p.halo_ids >= p.r1))
        # the halo sources pick the right entries of the all-gathered vector
        assert np.array_equal(gathered[p.halo_src], x[p.halo_ids])
        assert np.array_equal(p.d, d[p.r0:p.r1]) and np.array_equal(p.b, b[p.r0:p.r1])
        seen += p.n_rows
    assert seen == nq


def _lockstep(c, ranks, method, eps, max_iter, check_every=1):
    rp, ci, v, d, b, q, m = system_of(c)
    bounds = D.partition_rows(rp, ranks)
    plans = [D.block_plan(rp, ci, v, d, b, bounds, r) for r in range(ranks)]
    ops = [HostBlockOps(p) for p in plans]
    if method == "jacobi":
        gens = [D.jacobi(o, p, eps, max_iter, check_every) for o, p in zip(ops, plans)]
    else:
        gens = [D.bicgstab(o, p, eps, max_iter) for o, p in zip(ops, plans)]
    res = D.LockstepComm.run_all(gens, np.concatenate)
    xq = D.LockstepComm.run_all([D.collect(o, p, r[0]) for o, p, r in zip(ops, plans, res)], np.concatenate)
    assert all(np.array_equal(xq[0], xr) for xr in xq)
    return xq[0], res[0], m, b


@pytest.mark.parametrize("ranks", [1, 2, 3, 4])
@pytest.mark.parametrize("sweeps", [1, 9, 60])
def test_lockstep_jacobi_equals_the_oracle_sweep_for_sweep(ranks, sweeps):
    c = synth.random_chain(n=900, deg=10, goal_frac=0.03, sink_frac=0.03, seed=4)
    x, (_, it, delta, ok), m, b = _lockstep(c, ranks, "jacobi", 0.0, sweeps)
    xo, ito, do, oko = O.jacobi(m, b, 0.0, sweeps)
    assert it == ito == sweeps and not ok
    assert np.max(np.abs(x - xo)) <= 1e-15 and abs(delta - do) <= 1e-15


@pytest.mark.parametrize("ranks", [2, 3])
def test_lockstep_jacobi_stopping_rule(ranks):
    """Checked every sweep, the split loop stops at the oracle's sweep; checked every 16, at
    the next multiple of 16."""
    c = synth.random_chain(n=1200, deg=8, goal_frac=0.04, sink_frac=0.04, seed=5)
    x, (_, it, delta, ok), m, b = _lockstep(c, ranks, "jacobi", 1e-12, 100_000, check_every=1)
    xo, ito, do, oko = O.jacobi(m, b, 1e-12, 100_000)
    assert ok and oko and it == ito and np.max(np.abs(x - xo)) <= 1e-15
    x16, (_, it16, _, ok16), _, _ = _lockstep(c, ranks, "jacobi", 1e-12, 100_000, check_every=16)
    assert ok16 and it16 == -(-ito // 16) * 16
    assert np.max(np.abs(x16 - O.dense_solve(m, b))) <= 1e-9


@pytest.mark.parametrize("ranks", [1, 2, 3])
def test_lockstep_bicgstab_reaches_the_oracle_solution(ranks):
    c = synth.random_chain(n=1500, deg=8, goal_frac=0.03, sink_frac=0.03, seed=6)
    x, (_, it, res, status), m, b = _lockstep(c, ranks, "bicgstab", 1e-13, 1000)
    xo, ito, ro, oko = O.bicgstab(m, b, 1e-13, 1000)
    assert status == "ok" and oko
    assert np.max(np.abs(x - O.dense_solve(m, b))) <= 1e-10
    assert abs(it - ito) <= 2


def test_lockstep_bicgstab_restart_and_gamblers_ruin():
    """Sparse b (q . r = 0 reachable): the restart path; and the closed form of the
    gambler's ruin on 3 ranks."""
    from tests import brute
    c = synth.table1_chain(92, 211)
    x, (_, it, res, status), m, b = _lockstep(c, 2, "bicgstab", 1e-14, 500)
    assert status == "ok" and np.max(np.abs(x - O.dense_solve(m, b))) <= 1e-12
    g = synth.gamblers_ruin(40, 0.45)
    x, (_, it, res, status), m, b = _lockstep(g, 3, "bicgstab", 1e-13, 400)
    want = np.array([brute.gambler_closed_form(40, 0.45, i) for i in range(1, 40)])
    assert status == "ok" and np.max(np.abs(x - want)) <= 1e-9


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("method", ["jacobi", "bicgstab"])
def test_two_gloo_ranks_match_the_oracle(method):
    import torch.multiprocessing as mp
    c = synth.random_chain(n=1000, deg=8, goal_frac=0.04, sink_frac=0.04, seed=7)
    _, _, _, _, _, q, m = system_of(c)
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    eps = 1e-13
    procs = [ctx.Process(target=gloo_worker, args=(r, 2, port, c, method, eps, 100_000, 1, out))
             for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((out.get(timeout=180) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    x0, x1 = res[0][1], res[1][1]
    assert np.array_equal(x0, x1) and res[0][2] == res[1][2]
    assert res[0][5] > 0 and res[1][5] > 0                    # both blocks have a halo
    xs = O.dense_solve(m, np.asarray(system_of(c)[4]))
    assert np.max(np.abs(x0 - xs)) <= 1e-10
    if method == "jacobi":
        xo, ito, _, _ = O.jacobi(m, system_of(c)[4], eps, 100_000)
        assert res[0][2] == ito and np.max(np.abs(x0 - xo)) <= 1e-15
