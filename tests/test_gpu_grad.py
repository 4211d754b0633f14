"""Adjoint solve and parameter gradients on the GPU vs the FP64 oracle and central differences."""
import numpy as np
import pytest

import oracle as O
import paper_1210_6412_gb300 as R
from paper_1210_6412_gb300 import synth
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    return synth.parametric_chain(n=3000, n_classes=16, goal_frac=0.01, sink_frac=0.02, seed=21)


def _t(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_softmax_probs_match_oracle(pc):
    torch = need_gpu()
    p = torch.empty(pc.m, dtype=torch.float64, device="cuda")
    R.reach_param_probs(_t(torch, pc.rowptr), _t(torch, pc.cls), _t(torch, pc.offset),
                        _t(torch, pc.theta), p)
    torch.cuda.synchronize()
    want = O.softmax_probs(pc.rowptr, pc.cls, pc.offset, pc.theta)
    np.testing.assert_allclose(p.cpu().numpy(), want, rtol=1e-14, atol=1e-16)


def test_grad_p_matches_oracle_adjoint(pc):
    need_gpu()
    p = O.softmax_probs(pc.rowptr, pc.cls, pc.offset, pc.theta)
    g_o, x_o, cls_o = O.grad_p(pc.n, pc.rowptr, pc.col, p, pc.goal, pc.init)
    assert cls_o[pc.init] == O.SQ
    with R.Solver(pc.n, pc.rowptr, pc.col, p, pc.goal) as s:
        x, _ = s.solve("jacobi", eps=1e-14)
        g, info = s.grad(pc.init, eps=1e-15)
    np.testing.assert_allclose(x, x_o, atol=1e-12, rtol=0)
    assert info["status"] == R.REACH_OK
    scale = np.max(np.abs(g_o))
    np.testing.assert_allclose(g, g_o, atol=1e-10 * scale, rtol=1e-9)


@pytest.mark.parametrize("method", ["jacobi", "bicgstab"])
def test_grad_p_adjoint_methods_match_oracle(pc, method):
    """The adjoint system (I - A)^T y = e_init solved by FP64 Jacobi or by BiCGStab (§3.2 on
    the transpose): the same d x_init / d P, after a forward solve by the other method too."""
    need_gpu()
    p = O.softmax_probs(pc.rowptr, pc.cls, pc.offset, pc.theta)
    g_o, x_o, cls_o = O.grad_p(pc.n, pc.rowptr, pc.col, p, pc.goal, pc.init)
    with R.Solver(pc.n, pc.rowptr, pc.col, p, pc.goal) as s:
        x, _ = s.solve("bicgstab" if method == "jacobi" else "jacobi", eps=1e-14)
        g, info = s.grad(pc.init, eps=1e-15, method=method)
        g2, info2 = s.grad(pc.init, eps=1e-15, method=method)   # the cached loop graph again
    np.testing.assert_allclose(x, x_o, atol=1e-12, rtol=0)
    assert info["status"] == R.REACH_OK and info["iters"] > 0
    scale = np.max(np.abs(g_o))
    np.testing.assert_allclose(g, g_o, atol=1e-10 * scale, rtol=1e-9)
    assert np.array_equal(g, g2) and info["iters"] == info2["iters"]


def test_grad_rejects_other_adjoint_methods(pc):
    need_gpu()
    p = O.softmax_probs(pc.rowptr, pc.cls, pc.offset, pc.theta)
    with R.Solver(pc.n, pc.rowptr, pc.col, p, pc.goal) as s:
        s.solve("jacobi", eps=1e-12)
        for m in ("mixed", "scc_jacobi"):
            with pytest.raises(R.ReachError) as ei:
                s.grad(pc.init, method=m)
            assert ei.value.status == R.REACH_EINVAL


def test_grad_theta_kernel_matches_oracle(pc):
    torch = need_gpu()
    p = O.softmax_probs(pc.rowptr, pc.cls, pc.offset, pc.theta)
    g_p = np.random.default_rng(0).standard_normal(pc.m)
    out = torch.empty(16, dtype=torch.float64, device="cuda")
    R.reach_param_grad_theta(_t(torch, pc.rowptr), _t(torch, pc.cls), _t(torch, p), _t(torch, g_p), 16, out)
    torch.cuda.synchronize()
    want = O.grad_theta(pc.rowptr, p, g_p, pc.cls, 16)
    np.testing.assert_allclose(out.cpu().numpy(), want, rtol=1e-10, atol=1e-12)


def test_autograd_matches_central_differences(pc):
    torch = need_gpu()
    from paper_1210_6412_gb300.autograd import reach_prob
    args = [_t(torch, a) for a in (pc.rowptr, pc.col, pc.cls, pc.offset, pc.goal)]
    theta = _t(torch, pc.theta).clone().requires_grad_(True)
    y = reach_prob(theta, *args, pc.init)
    y.backward()
    g = theta.grad.cpu().numpy()
    # BiCGStab forward and adjoint: the same value and gradient (each solver's own stopping
    # rule at 1e-13 / 1e-14 leaves differences of about 1e-12)
    theta_b = _t(torch, pc.theta).clone().requires_grad_(True)
    yb = reach_prob(theta_b, *args, pc.init, method="bicgstab", adj_method="bicgstab")
    yb.backward()
    assert abs(float(yb) - float(y)) <= 1e-10
    gb = theta_b.grad.cpu().numpy()

    def f(th):
        with torch.no_grad():
            return float(reach_prob(_t(torch, th), *args, pc.init))

    h = 1e-6
    for j in range(0, 16, 3):
        e = np.zeros(16)
        e[j] = h
        fd = (f(pc.theta + e) - f(pc.theta - e)) / (2 * h)
        assert abs(fd - g[j]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (j, fd, g[j])
    # oracle gradient of the same chain
    p = O.softmax_probs(pc.rowptr, pc.cls, pc.offset, pc.theta)
    g_p, _, _ = O.grad_p(pc.n, pc.rowptr, pc.col, p, pc.goal, pc.init)
    g_want = O.grad_theta(pc.rowptr, p, g_p, pc.cls, 16)
    np.testing.assert_allclose(g, g_want, rtol=1e-8, atol=1e-12)
    np.testing.assert_allclose(gb, g_want, rtol=1e-8, atol=1e-12)


def test_grad_outside_sq_is_zero(pc):
    need_gpu()
    p = O.softmax_probs(pc.rowptr, pc.cls, pc.offset, pc.theta)
    goal_state = int(np.flatnonzero(pc.goal)[0])
    with R.Solver(pc.n, pc.rowptr, pc.col, p, pc.goal) as s:
        s.solve("bicgstab", eps=1e-13)
        g, _ = s.grad(goal_state)
    assert np.all(g == 0.0)
