"""General systems M x = b (the random diagonally dominant matrices of §6) vs the oracle."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import paper_1210_6412_gb300 as R
from paper_1210_6412_gb300 import synth
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _oracle(s):
    m = sp.csr_matrix((s.val, s.col, s.rowptr), shape=(s.n, s.n))
    return O.dense_solve(m, s.b)


@pytest.mark.parametrize("n,density", [(500, 0.05), (3000, 0.01), (1200, 0.2)])
@pytest.mark.parametrize("method,tol", [("jacobi", 1e-9), ("mixed", 1e-6), ("bicgstab", 1e-9)])
def test_general_system_matches_oracle(n, density, method, tol):
    need_gpu()
    s = synth.diag_dominant_system(n=n, density=density, seed=n)
    x_o = _oracle(s)
    scale = max(1.0, float(np.max(np.abs(x_o))))
    with R.Solver.system(s.n, s.rowptr, s.col, s.val, s.b) as sol:
        x, info = sol.solve(method, eps=1e-14 if method != "mixed" else 1e-12, max_iter=2_000_000)
        with pytest.raises(R.ReachError) as ei:
            sol.precompute()
        assert ei.value.status == R.REACH_ESTATE
    assert info["status"] == R.REACH_OK
    assert np.max(np.abs(x - x_o)) <= tol * scale


def test_general_system_signs_and_zero_diagonal():
    need_gpu()
    # mixed signs: M = [[4, -1, 0], [2, 5, -1], [0, -3, 6]]
    rowptr = np.array([0, 2, 5, 7], np.int64)
    col = np.array([0, 1, 0, 1, 2, 1, 2], np.int32)
    val = np.array([4.0, -1, 2, 5, -1, -3, 6])
    b = np.array([1.0, -2.0, 3.0])
    want = np.linalg.solve(np.array([[4, -1, 0], [2, 5, -1], [0, -3, 6.0]]), b)
    for method in ("jacobi", "bicgstab"):
        with R.Solver.system(3, rowptr, col, val, b) as sol:
            x, _ = sol.solve(method, eps=1e-15)
        np.testing.assert_allclose(x, want, atol=1e-13)
    bad = val.copy()
    bad[3] = 0.0                       # M_11 = 0
    with pytest.raises(R.ReachError) as ei:
        R.reach_system_create(3, rowptr, col, bad, b)
    assert ei.value.status == R.REACH_EINVAL and "zero diagonal" in str(ei.value)
