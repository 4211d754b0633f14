"""The row-split Jacobi and BiCGStab on the GPU's row-block kernels, against the oracle.

One GPU holds every rank's block; LockstepComm advances the ranks in turn and performs
their all-gathers and all-reduces on the host side, so no kernel waits for another.  The
single-rank NCCL group runs the whole user-level path (partition and extraction on the
GPU, reach_get_system, the block, TorchComm over NCCL, the final collect).
"""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_1210_6412_gb300 import dist as D
from paper_1210_6412_gb300 import synth
from tests.dist_host import system_of
from tests.gpu_util import TOL_FP64, need_gpu

pytestmark = pytest.mark.gpu


def _run(torch, c, ranks, method, eps, max_iter, check_every=1):
    rp, ci, v, d, b, q, m = system_of(c)
    bounds = D.partition_rows(rp, ranks)
    plans = [D.block_plan(rp, ci, v, d, b, bounds, r) for r in range(ranks)]
    ops = [D.CudaBlockOps(p) for p in plans]
    try:
        if method == "jacobi":
            gens = [D.jacobi(o, p, eps, max_iter, check_every) for o, p in zip(ops, plans)]
        else:
            gens = [D.bicgstab(o, p, eps, max_iter) for o, p in zip(ops, plans)]
        res = D.LockstepComm.run_all(gens, torch.cat)
        xq = D.LockstepComm.run_all([D.collect(o, p, r[0]) for o, p, r in zip(ops, plans, res)], torch.cat)
    finally:
        for o in ops:
            o.close()
    return xq[0], res[0], m, b


@pytest.mark.parametrize("ranks", [1, 2, 3])
@pytest.mark.parametrize("sweeps", [1, 25])
def test_block_jacobi_iterates_match_the_oracle(ranks, sweeps):
    torch = need_gpu()
    c = synth.random_chain(n=3000, deg=12, goal_frac=0.03, sink_frac=0.03, seed=14)
    x, (_, it, delta, ok), m, b = _run(torch, c, ranks, "jacobi", 0.0, sweeps)
    xo, ito, do, _ = O.jacobi(m, b, 0.0, sweeps)
    assert it == sweeps
    assert np.max(np.abs(x - xo)) <= 1e-13 and abs(delta - do) <= 1e-13


@pytest.mark.parametrize("ranks", [2, 4])
@pytest.mark.parametrize("method", ["jacobi", "bicgstab"])
def test_block_solves_reach_the_oracle_solution(ranks, method):
    torch = need_gpu()
    c = synth.random_chain(n=5000, deg=10, goal_frac=0.03, sink_frac=0.03, seed=15)
    x, (_, it, last, st), m, b = _run(torch, c, ranks, method, 1e-13, 200_000, check_every=16)
    assert st in (True, "ok")
    assert np.max(np.abs(x - O.dense_solve(m, b))) <= TOL_FP64


def test_block_bicgstab_on_the_layered_chain():
    """A model-checker-shaped system: halos from forward and back edges across blocks."""
    torch = need_gpu()
    c = synth.layered_chain(layers=60, width=300)
    x, (_, it, last, st), m, b = _run(torch, c, 3, "bicgstab", 1e-13, 5000)
    xo, _, _, ok = O.jacobi(m, b, 1e-15, 1_000_000)
    assert st == "ok" and ok and np.max(np.abs(x - xo)) <= TOL_FP64


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("method", ["jacobi", "bicgstab"])
def test_solve_distributed_single_nccl_rank(method):
    torch = need_gpu()
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(_free_port())
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        c = synth.random_chain(n=4000, deg=12, goal_frac=0.02, sink_frac=0.02, seed=16)
        x_o, cls_o, _ = O.reach_probabilities(c.n, c.rowptr, c.col, c.val, c.goal, method="dense")
        comm = D.TorchComm("cuda")
        x, info = D.solve_distributed(c.n, c.rowptr, c.col, c.val, c.goal, comm, method=method, eps=1e-13)
        assert info["status"] == "ok"
        assert np.max(np.abs(x - x_o)) <= TOL_FP64
    finally:
        dist.destroy_process_group()
