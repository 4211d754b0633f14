"""Batched multi-RHS solves (K goal sets over many chains) vs the oracle, chain by chain."""
import numpy as np
import pytest

import oracle as O
import paper_1210_6412_gb300 as R
from paper_1210_6412_gb300 import synth
from tests.gpu_util import TOL_MIXED, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    # a scaled-down batch: 6 chains of 100..3000 states, out-degree 2..32, 8 goal sets,
    # 2% sinks so that every goal set leaves a non-trivial S?
    return synth.batched_chains(n_chains=6, n_min=100, n_max=3000, k=8, sink_frac=0.02, seed=31)


def _oracle(batch, mode):
    cls_all, x_all = [], []
    for c, goals in zip(batch.chains, batch.goals):
        cl, xs = [], []
        for j in range(goals.shape[0]):
            x, cls, _ = O.reach_probabilities(c.n, c.rowptr, c.col, c.val, goals[j], mode, method="dense")
            cl.append(cls)
            xs.append(x)
        cls_all.append(np.stack(cl))
        x_all.append(np.stack(xs))
    return np.concatenate(cls_all, axis=1), np.concatenate(x_all, axis=1)


@pytest.mark.parametrize("mode", [O.PROB01, O.PROB0_ONLY])
@pytest.mark.parametrize("device", [False, True])
def test_batch_matches_oracle(batch, mode, device):
    torch = need_gpu()
    n, rowptr, col, val, goals, offs = batch.concat()
    cls_o, x_o = _oracle(batch, mode)
    args = (rowptr, col, val, goals)
    if device:
        args = tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in args)
    with R.BatchSolver(n, *args, mode=mode) as bs:
        cls = bs.classes()
        x, info = bs.solve(eps=1e-9)
    assert np.array_equal(cls, cls_o)
    assert np.max(np.abs(x - x_o)) <= TOL_MIXED
    assert info["status"] == R.REACH_OK and info["refinements"] >= 1
    assert info["resid_inf"] < 1e-8


def test_batch_fewer_goal_sets_and_repeat_solve(batch):
    need_gpu()
    n, rowptr, col, val, goals, offs = batch.concat()
    g3 = np.ascontiguousarray(goals[:3])
    cls_o, x_o = _oracle(synth.Batch(batch.chains, [g[:3] for g in batch.goals]), O.PROB01)
    with R.BatchSolver(n, rowptr, col, val, g3) as bs:
        x1, i1 = bs.solve(eps=1e-9)
        x2, i2 = bs.solve(eps=1e-9)
        assert np.array_equal(bs.classes(), cls_o)
    assert np.max(np.abs(x1 - x_o)) <= TOL_MIXED
    assert np.array_equal(x1, x2) and i1["iters"] == i2["iters"]


def test_batch_host_loops(batch, monkeypatch):
    need_gpu()
    monkeypatch.setenv("REACH_HOST_LOOPS", "1")
    n, rowptr, col, val, goals, offs = batch.concat()
    cls_o, x_o = _oracle(batch, O.PROB01)
    with R.BatchSolver(n, rowptr, col, val, goals) as bs:
        assert np.array_equal(bs.classes(), cls_o)
        x, info = bs.solve(eps=1e-9)
    assert np.max(np.abs(x - x_o)) <= TOL_MIXED


def test_batch_rejects_bad_k():
    need_gpu()
    c = synth.worked_chain()
    goals = np.zeros((9, c.n), np.uint8)
    with pytest.raises(R.ReachError) as ei:
        R.reach_batch_create(c.n, c.rowptr, c.col, c.val, goals)
    assert ei.value.status == R.REACH_EINVAL
