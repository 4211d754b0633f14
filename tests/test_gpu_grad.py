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
    np.testing.assert_allclose(g, O.grad_theta(pc.rowptr, p, g_p, pc.cls, 16), rtol=1e-8, atol=1e-12)


def test_grad_outside_sq_is_zero(pc):
    need_gpu()
    p = O.softmax_probs(pc.rowptr, pc.cls, pc.offset, pc.theta)
    goal_state = int(np.flatnonzero(pc.goal)[0])
    with R.Solver(pc.n, pc.rowptr, pc.col, p, pc.goal) as s:
        s.solve("bicgstab", eps=1e-13)
        g, _ = s.grad(goal_state)
    assert np.all(g == 0.0)
