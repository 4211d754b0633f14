"""Shared helpers of the GPU parity tests: run the CUDA path and the oracle on one chain."""
import numpy as np
import pytest

import oracle as O
import paper_1210_6412_gb300 as R

TOL_FP64 = 1e-9      # x within 1e-9 absolute of the FP64 oracle
TOL_MIXED = 1e-6     # mixed-precision form


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def oracle_solution(c, mode=O.PROB01):
    """Classes and x of the oracle: dense LU when S? is small, else Jacobi to 1e-14."""
    cls = O.partition(c.n, c.rowptr, c.col, c.val, c.goal, mode)
    q, a, b = O.extract_system(c.n, c.rowptr, c.col, c.val, cls)
    m = O.system_matrix(a)
    if q.size <= 3000:
        xq = O.dense_solve(m, b)
    else:
        xq, it, _, ok = O.jacobi(m, b, 1e-14, 2_000_000)
        assert ok
    return cls, O.full_vector(c.n, cls, q, xq)


def gpu_solve(c, mode, method, eps, max_iter=2_000_000, refine_k=0, device=False):
    torch = need_gpu()
    args = (c.rowptr, c.col, c.val, c.goal)
    if device:
        args = tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in args)
    with R.Solver(c.n, *args, mode=mode) as s:
        cls = s.classes()
        x, info = s.solve(method, eps=eps, max_iter=max_iter, refine_k=refine_k)
    return cls, x, info
