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


# ---------------------------------------------------------------- per-chain stopping

@pytest.fixture(scope="module")
def mixed_speed():
    # chains that converge at different rates: few absorbing states (slow) and many (fast)
    slow = synth.batched_chains(n_chains=3, n_min=200, n_max=4000, k=8, sink_frac=0.01, seed=41)
    fast = synth.batched_chains(n_chains=3, n_min=200, n_max=4000, k=8, sink_frac=0.25, seed=42)
    return synth.Batch(slow.chains[:2] + fast.chains + slow.chains[2:], slow.goals[:2] + fast.goals + slow.goals[2:])


def _solo(bt, i, eps, refine_k=0):
    c = bt.chains[i]
    with R.BatchSolver(c.n, c.rowptr, c.col, c.val, np.ascontiguousarray(bt.goals[i])) as bs:
        x, info = bs.solve(eps=eps, refine_k=refine_k)
        iters, last = bs.chain_info()
    assert iters[0] == info["iters"]
    return x, info


def test_chains_stop_on_their_own_and_match_solo_solves(mixed_speed):
    need_gpu()
    n, rowptr, col, val, goals, offs = mixed_speed.concat()
    with R.BatchSolver(n, rowptr, col, val, goals, chains=offs) as bs:
        x, info = bs.solve(eps=1e-9)
        iters, last = bs.chain_info()
    assert info["status"] == R.REACH_OK
    assert len(set(iters.tolist())) > 1          # the chains really stopped at different sweeps
    assert info["iters"] == iters.max()
    assert np.all(last < 1e-9)
    for i in range(len(mixed_speed.chains)):
        xs, inf_s = _solo(mixed_speed, i, 1e-9)
        a, b = int(offs[i]), int(offs[i + 1])
        # identical per-row arithmetic and the same stopping point: bit-identical
        assert iters[i] == inf_s["iters"]
        assert np.array_equal(x[:, a:b], xs)


def test_chains_match_oracle(batch):
    need_gpu()
    n, rowptr, col, val, goals, offs = batch.concat()
    cls_o, x_o = _oracle(batch, O.PROB01)
    with R.BatchSolver(n, rowptr, col, val, goals, chains=offs) as bs:
        assert np.array_equal(bs.classes(), cls_o)
        x, info = bs.solve(eps=1e-9)
    assert np.max(np.abs(x - x_o)) <= TOL_MIXED
    assert info["resid_inf"] < 1e-8


def test_chains_save_work_against_one_stopping_rule(mixed_speed):
    need_gpu()
    n, rowptr, col, val, goals, offs = mixed_speed.concat()
    with R.BatchSolver(n, rowptr, col, val, goals) as bs:
        x1, i1 = bs.solve(eps=1e-9)
        bs.set_chains(offs)
        x2, i2 = bs.solve(eps=1e-9)
        it2, _ = bs.chain_info()
    assert i1["iters"] == i2["iters"]                 # the slowest chain sets both
    assert i2["bytes_moved"] < i1["bytes_moved"]      # converged chains were skipped
    slowest = int(np.argmax(it2))
    a, b = int(offs[slowest]), int(offs[slowest + 1])
    assert np.array_equal(x1[:, a:b], x2[:, a:b])


def test_chains_host_loops_and_refine_k(mixed_speed, monkeypatch):
    need_gpu()
    n, rowptr, col, val, goals, offs = mixed_speed.concat()
    with R.BatchSolver(n, rowptr, col, val, goals, chains=offs) as bs:
        xd, idev = bs.solve(eps=1e-9, refine_k=8)
    monkeypatch.setenv("REACH_HOST_LOOPS", "1")
    with R.BatchSolver(n, rowptr, col, val, goals, chains=offs) as bs:
        xh, ihost = bs.solve(eps=1e-9, refine_k=8)
        ith, _ = bs.chain_info()
    assert np.array_equal(xd, xh) and idev["iters"] == ihost["iters"]
    xs, inf_s = _solo(mixed_speed, 0, 1e-9, refine_k=8)
    assert ith[0] == inf_s["iters"] and np.array_equal(xh[:, int(offs[0]):int(offs[1])], xs)


def test_chains_max_iter_and_empty_chains(mixed_speed):
    need_gpu()
    n, rowptr, col, val, goals, offs = mixed_speed.concat()
    # an empty chain at the front, between two chains and at the back
    offs2 = np.concatenate([[0], offs[:3], offs[2:], [n]]).astype(np.int64)
    with R.BatchSolver(n, rowptr, col, val, goals, chains=offs2) as bs:
        x, info = bs.solve(eps=1e-300, max_iter=48, check=False)
        iters, last = bs.chain_info()
        assert info["status"] == R.REACH_ENOTCONV
        nonempty = np.diff(offs2) > 0
        assert np.all(iters[nonempty] == -1)
        x2, info2 = bs.solve(eps=1e-9)
        iters2, _ = bs.chain_info()
    assert info2["status"] == R.REACH_OK
    assert np.all(iters2[~nonempty] == 1)             # nothing to solve: stops at the first check
    with R.BatchSolver(n, rowptr, col, val, goals, chains=offs) as bs:
        x3, _ = bs.solve(eps=1e-9)
    assert np.array_equal(x2, x3)


def test_set_chains_rejects_bad_offsets(mixed_speed):
    need_gpu()
    n, rowptr, col, val, goals, offs = mixed_speed.concat()
    with R.BatchSolver(n, rowptr, col, val, goals) as bs:
        x0, i0 = bs.solve(eps=1e-9)
        for bad in ([1, n], [0, n - 1], [0, 5, 3, n], [0]):
            with pytest.raises((R.ReachError, ValueError)) as ei:
                bs.set_chains(np.array(bad, np.int64))
            if isinstance(ei.value, R.ReachError):
                assert ei.value.status == R.REACH_EINVAL
        # a boundary that cuts through a chain: its entries cross it
        cut = np.array([0, int(offs[1]) // 2, n], np.int64)
        with pytest.raises(R.ReachError) as ei:
            bs.set_chains(cut)
        assert ei.value.status == R.REACH_EINVAL and "outside its chain" in R.reach_last_error(None)
        # the batch is unchanged: still one chain
        x1, i1 = bs.solve(eps=1e-9)
    assert np.array_equal(x0, x1) and i0["iters"] == i1["iters"]


@pytest.mark.parametrize("variant", ["0", "1", "2", "3", "4"])
def test_every_sweep_variant_matches_oracle(batch, variant, monkeypatch):
    """The five FP32 sweep variants (autotuner candidates); 0, 2, 3 and 4 run the same FMAs
    in the same order, so their x is bit-identical."""
    need_gpu()
    n, rowptr, col, val, goals, offs = batch.concat()
    cls_o, x_o = _oracle(batch, O.PROB01)
    monkeypatch.setenv("REACH_BSWEEP_VARIANT", variant)
    with R.BatchSolver(n, rowptr, col, val, goals, chains=offs) as bs:
        x, info = bs.solve(eps=1e-9)
    monkeypatch.setenv("REACH_BSWEEP_VARIANT", "0")
    with R.BatchSolver(n, rowptr, col, val, goals, chains=offs) as bs:
        x0, _ = bs.solve(eps=1e-9)
    assert np.max(np.abs(x - x_o)) <= TOL_MIXED
    if variant != "1":
        assert np.array_equal(x, x0)


def test_batch_autotune_picks_a_variant_and_period(batch):
    need_gpu()
    n, rowptr, col, val, goals, offs = batch.concat()
    cls_o, x_o = _oracle(batch, O.PROB01)
    with R.BatchSolver(n, rowptr, col, val, goals, chains=offs) as bs:
        t = bs.autotune()
        assert t["variant"] in range(5) and t["sweep_ms"] > 0
        assert 8 <= t["refine_k"] <= 62 and t["refine_k"] % 2 == 0
        x, info = bs.solve(eps=1e-9)
    assert info["status"] == R.REACH_OK
    assert np.max(np.abs(x - x_o)) <= TOL_MIXED
