"""The allocation-free Jacobi entry point against the oracle and the regular solver.

reach_jacobi_solve_noalloc serves callers that cannot call cudaMalloc (code inside an
application that owns the device memory through its own pool, or on a path where an
allocation would stall the device).  It keeps its scratch in a fixed device array inside
the library.  These tests build the system over S? on the host, hand it to the entry point
through the C ABI twice in a row, and compare x with the oracle's and with reach_solve's
FP64 Jacobi result; a capped call must stop after exactly max_iter sweeps with the
oracle's iterate after that many sweeps.  The file is collected last so that a run
stopping at its first failure has run everything else.
"""
import ctypes as C

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import paper_1210_6412_gb300 as R
from paper_1210_6412_gb300 import synth
from tests.gpu_util import TOL_FP64, need_gpu, oracle_solution

pytestmark = pytest.mark.gpu


def _system(c):
    cls = O.partition(c.n, c.rowptr, c.col, c.val, c.goal)
    q, a, b = O.extract_system(c.n, c.rowptr, c.col, c.val, cls)
    d = 1.0 - a.diagonal()
    off = (a - sp.diags(a.diagonal())).tocsr()
    off.eliminate_zeros()
    return q, off, b, d, O.system_matrix(a)


def _call(torch, dev_sys, nq, eps, max_iter, check_every, x0=None):
    rp, ci, av, bb, dd = dev_sys
    x = torch.zeros(nq, dtype=torch.float64, device="cuda") if x0 is None else x0.clone()
    iters, delta = C.c_int64(0), C.c_double(0.0)
    st = R.lib().reach_jacobi_solve_noalloc(nq, rp.data_ptr(), ci.data_ptr(), av.data_ptr(), bb.data_ptr(),
                                            dd.data_ptr(), eps, max_iter, check_every, x.data_ptr(),
                                            C.byref(iters), C.byref(delta),
                                            torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return st, x.cpu().numpy(), iters.value, delta.value


def _to_dev(torch, q, off, b, d):
    dev = lambda arr, dt: torch.from_numpy(np.ascontiguousarray(arr, dtype=dt)).cuda()
    return (dev(off.indptr, np.int64), dev(off.indices, np.int32), dev(off.data, np.float64),
            dev(b, np.float64), dev(d, np.float64))


def test_noalloc_matches_oracle_and_regular_solver_twice():
    torch = need_gpu()
    c = synth.random_chain(n=4096, deg=16, goal_frac=0.02, sink_frac=0.02, seed=77)
    cls_o, x_o = oracle_solution(c)
    with R.Solver(c.n, c.rowptr, c.col, c.val, c.goal) as s:
        x_ref, info = s.solve("jacobi", eps=1e-13)
    q, off, b, d, _ = _system(c)
    dev_sys = _to_dev(torch, q, off, b, d)
    for call in range(2):
        st, xs, iters, delta = _call(torch, dev_sys, q.size, 1e-13, 1_000_000, 16)
        assert st == R.REACH_OK, R.reach_last_error()
        assert np.max(np.abs(xs - x_o[q])) <= TOL_FP64, call
        assert np.max(np.abs(xs - x_ref[q])) <= TOL_FP64, call
        assert abs(iters - info["iters"]) <= 16 and delta < 1e-13


@pytest.mark.parametrize("max_iter,check_every", [(10, 16), (7, 4), (33, 8)])
def test_noalloc_runs_exactly_max_iter_sweeps(max_iter, check_every):
    """A cap that is not a multiple of the check period: exactly max_iter sweeps run, x is
    the oracle's Jacobi iterate after max_iter sweeps from 0, and the call says so."""
    torch = need_gpu()
    c = synth.random_chain(n=3000, deg=12, goal_frac=0.02, sink_frac=0.02, seed=78)
    q, off, b, d, m = _system(c)
    x_o, it_o, delta_o, ok = O.jacobi(m, b, 0.0, max_iter)
    assert not ok and it_o == max_iter
    dev_sys = _to_dev(torch, q, off, b, d)
    for call in range(2):
        st, xs, iters, delta = _call(torch, dev_sys, q.size, 1e-300, max_iter, check_every)
        assert st == R.REACH_ENOTCONV
        assert iters == max_iter, (iters, max_iter)
        assert np.max(np.abs(xs - x_o)) <= 1e-13, call
        assert abs(delta - delta_o) <= 1e-13


def test_noalloc_rejects_oversized_system():
    need_gpu()
    lib = R.lib()
    st = lib.reach_jacobi_solve_noalloc((1 << 19) + 1, 1, 1, 1, 1, 1, 1e-9, 10, 2, 1, None, None, None)
    assert st == R.REACH_EINVAL
    assert "524288" in R.reach_last_error()
