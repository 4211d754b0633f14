"""The allocation-free Jacobi entry point agrees with the regular solver.

reach_jacobi_solve_noalloc serves callers that cannot call cudaMalloc (code inside an
application that owns the device memory through its own pool, or on a path where an
allocation would stall the device).  It keeps its scratch in a fixed device array inside
the library.  This test builds the system over S? on the host, hands it to the entry point
through the C ABI twice in a row, and compares x with reach_solve's FP64 Jacobi result.
It is collected last so that a run stopping at its first failure has run everything else.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
import paper_1210_6412_gb300 as R
from paper_1210_6412_gb300 import synth
from tests.gpu_util import TOL_FP64, need_gpu

pytestmark = pytest.mark.gpu


def test_noalloc_matches_regular_solver_twice():
    torch = need_gpu()
    c = synth.random_chain(n=4096, deg=16, goal_frac=0.02, sink_frac=0.02, seed=77)
    # regular entry point: x over all states
    with R.Solver(c.n, c.rowptr, c.col, c.val, c.goal) as s:
        x_ref, info = s.solve("jacobi", eps=1e-13)
    # the same system over S?, extracted on the host
    cls = O.partition(c.n, c.rowptr, c.col, c.val, c.goal)
    q, a, b = O.extract_system(c.n, c.rowptr, c.col, c.val, cls)
    d = 1.0 - a.diagonal()
    off = (a - __import__("scipy.sparse", fromlist=["diags"]).diags(a.diagonal())).tocsr()
    off.eliminate_zeros()
    dev = lambda arr, dt: torch.from_numpy(np.ascontiguousarray(arr, dtype=dt)).cuda()
    rp, ci, av = dev(off.indptr, np.int64), dev(off.indices, np.int32), dev(off.data, np.float64)
    bb, dd = dev(b, np.float64), dev(d, np.float64)
    stream = torch.cuda.current_stream().cuda_stream
    lib = R.lib()
    for call in range(2):
        x = torch.zeros(q.size, dtype=torch.float64, device="cuda")
        iters, delta = C.c_int64(0), C.c_double(0.0)
        st = lib.reach_jacobi_solve_noalloc(q.size, rp.data_ptr(), ci.data_ptr(), av.data_ptr(),
                                            bb.data_ptr(), dd.data_ptr(), 1e-13, 1_000_000, 16,
                                            x.data_ptr(), C.byref(iters), C.byref(delta), stream)
        assert st == R.REACH_OK, R.reach_last_error()
        torch.cuda.synchronize()
        xs = x.cpu().numpy()
        assert np.max(np.abs(xs - x_ref[q])) <= TOL_FP64, call
        assert abs(iters.value - info["iters"]) <= 16 and delta.value < 1e-13


def test_noalloc_rejects_oversized_system():
    need_gpu()
    lib = R.lib()
    st = lib.reach_jacobi_solve_noalloc((1 << 19) + 1, 1, 1, 1, 1, 1, 1e-9, 10, 2, 1, None, None, None)
    assert st == R.REACH_EINVAL
    assert "524288" in R.reach_last_error()
