"""Planted mistakes in the oracle (on the CPU) are caught by the pins.

Each test swaps one oracle step for a plausible wrong version (a transposed operand, a
dropped term, a flipped sign, a wrong index) and checks that a pin of
test_oracle_pins fails.  This shows the pins constrain every step they cover.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from oracle import reach_oracle as R
from tests import test_oracle_pins as pins


def _patch(monkeypatch, name, fn):
    monkeypatch.setattr(R, name, fn)
    monkeypatch.setattr(O, name, fn)


def test_transposed_a_is_caught(monkeypatch):
    orig = R.extract_system

    def bad(*a):
        q, A, b = orig(*a)
        return q, A.T.tocsr(), b
    _patch(monkeypatch, "extract_system", bad)
    with pytest.raises(AssertionError):
        pins.test_worked_chain_partition_and_system()


def test_dropped_b_term_is_caught(monkeypatch):
    orig = R.extract_system

    def bad(n, rowptr, col, val, cls):
        q, A, b = orig(n, rowptr, col, val, cls)
        return q, A, b * (np.arange(b.size) != b.size - 1)
    _patch(monkeypatch, "extract_system", bad)
    with pytest.raises(AssertionError):
        pins.test_gamblers_ruin_closed_form(20, 0.4)


def test_jacobi_sign_is_caught(monkeypatch):
    def bad(m, b, eps, max_iter, x0=None, history=None):
        m = sp.csr_matrix(m)
        d = m.diagonal()
        off = (m - sp.diags(d)).tocsr()
        x = np.zeros(m.shape[0])
        for it in range(1, max_iter + 1):
            xp = x
            x = (b + off @ xp) / d
            if np.max(np.abs(x - xp)) < eps:
                return x, it, 0.0, True
        return x, max_iter, 1.0, False
    _patch(monkeypatch, "jacobi", bad)
    with pytest.raises(AssertionError):
        pins.test_worked_chain_solution("jacobi")


def test_bicgstab_beta_is_caught(monkeypatch):
    orig_dot = np.ndarray.__matmul__

    def bad(m, b, eps, max_iter, x0=None):
        m = sp.csr_matrix(m)
        x = np.zeros(m.shape[0]); r = b.copy(); q = r.copy()
        y = a = w = 1.0; v = np.zeros_like(x); p = np.zeros_like(x)
        for it in range(1, min(max_iter, 500) + 1):
            yp, y = y, q @ r
            p = r + y / yp * (p - w * v)      # drops the a / w factor of beta
            v = m @ p
            a = y / (q @ v)
            s = r - a * v
            t = m @ s
            w = (t @ s) / (t @ t)
            x = x + a * p + w * s
            r = s - w * t
            if np.max(np.abs(r)) < eps:
                return x, it, 0.0, True
        return x, max_iter, 1.0, False
    del orig_dot
    _patch(monkeypatch, "bicgstab", bad)
    with pytest.raises(AssertionError):
        pins.test_bicgstab_finite_termination(20, 0.45)


def test_prob1_without_goal_barrier_is_caught(monkeypatch):
    def bad(n, rowptr, col, val, goal, s0=None):
        p = R.canonical_csr(n, rowptr, col, val)
        if s0 is None:
            s0 = R.prob0(n, rowptr, col, val, goal)
        return ~R._backward_reach(p, s0, np.ones(n, bool))
    _patch(monkeypatch, "prob1", bad)
    with pytest.raises(AssertionError):
        pins.test_prob1_literal_reading_differs_from_definition()


def test_grad_wrong_index_is_caught(monkeypatch):
    orig = R.grad_p

    def bad(n, rowptr, col, val, goal, init, mode=O.PROB01, method="dense"):
        g, x, cls = orig(n, rowptr, col, val, goal, init, mode, method)
        row = np.repeat(np.arange(n), np.diff(rowptr))
        scale = np.where(x[np.asarray(col)] > 0, x[row] / np.maximum(x[np.asarray(col)], 1e-300), 0)
        return g * scale, x, cls
    _patch(monkeypatch, "grad_p", bad)
    with pytest.raises(AssertionError):
        pins.test_grad_p_matches_central_differences()


def test_scc_label_by_smallest_row_is_caught(monkeypatch):
    orig = R.scc_labels

    def bad(a):
        lab = orig(a)
        out = lab.copy()
        for c in np.unique(lab):
            out[lab == c] = np.flatnonzero(lab == c).min()
        return out
    _patch(monkeypatch, "scc_labels", bad)
    with pytest.raises(AssertionError):
        for seed in range(25):
            pins.test_scc_labels_and_levels_match_brute_force(seed)


def test_scc_levels_counting_vertices_not_components_is_caught(monkeypatch):
    """Heights over the vertex digraph (edges inside a component counted) are wrong."""
    def bad(a, labels):
        import scipy.sparse.csgraph as csg
        a = sp.csr_matrix(a)
        nq = a.shape[0]
        h = np.zeros(nq, np.int64)
        for _ in range(nq):
            row = np.repeat(np.arange(nq), np.diff(a.indptr))
            nh = np.zeros(nq, np.int64)
            np.maximum.at(nh, row, h[a.indices] + 1)
            nh = np.minimum(nh, nq)
            if np.array_equal(nh, h):
                break
            h = nh
        return h
    _patch(monkeypatch, "scc_levels", bad)
    with pytest.raises(AssertionError):
        for seed in range(25):
            pins.test_scc_labels_and_levels_match_brute_force(seed)


def test_block_jacobi_highest_level_first_is_caught(monkeypatch):
    def bad(m, b, eps, max_iter, labels=None, levels=None):
        m = sp.csr_matrix(m)
        nq = m.shape[0]
        diag = m.diagonal()
        off = (m - sp.diags(diag)).tocsr()
        lab = R.scc_labels(-off)
        lev = R.scc_levels(-off, lab)
        x = np.zeros(nq)
        nl = int(lev.max()) + 1 if nq else 0
        sweeps = 0
        for h in reversed(range(nl)):
            rows = np.flatnonzero(lev == h)
            for _ in range(max_iter):
                new = (b[rows] - off[rows] @ x) / diag[rows]
                d = float(np.max(np.abs(new - x[rows])))
                x[rows] = new
                sweeps += 1
                if d < eps:
                    break
        return x, sweeps, nl, True
    _patch(monkeypatch, "block_jacobi", bad)
    with pytest.raises(AssertionError):
        for seed in range(10):
            pins.test_block_jacobi_matches_lu(seed)


def _softmax_variant(index_by_row=False, offset_sign=1.0, shift_from_first_row=False):
    def bad(rowptr, cls_e, offset, theta):
        rowptr = np.asarray(rowptr)
        deg = np.diff(rowptr)
        row = np.repeat(np.arange(deg.size), deg)
        idx = np.minimum(row, len(theta) - 1) if index_by_row else np.asarray(cls_e)
        logit = np.asarray(theta, float)[idx] + offset_sign * np.asarray(offset, float)
        mx = np.maximum.reduceat(logit, rowptr[:-1])
        shift = np.full(logit.size, mx[0]) if shift_from_first_row else np.repeat(mx, deg)
        e = np.exp(logit - shift)
        return e / np.repeat(np.add.reduceat(e, rowptr[:-1]), deg)
    return bad


def test_softmax_theta_indexed_by_row_is_caught(monkeypatch):
    _patch(monkeypatch, "softmax_probs", _softmax_variant(index_by_row=True))
    with pytest.raises(AssertionError):
        pins.test_softmax_class_parameters_set_edge_ratios()


def test_softmax_offset_sign_is_caught(monkeypatch):
    _patch(monkeypatch, "softmax_probs", _softmax_variant(offset_sign=-1.0))
    with pytest.raises(AssertionError):
        pins.test_softmax_offsets_of_one_class_give_exact_shares()


def test_softmax_shift_from_another_row_is_caught(monkeypatch):
    _patch(monkeypatch, "softmax_probs", _softmax_variant(shift_from_first_row=True))
    with pytest.raises(AssertionError), np.errstate(all="ignore"):
        pins.test_softmax_large_logits_per_row()


def test_error_bound_with_the_smallest_tau_is_caught(monkeypatch):
    def bad(m, b, x):
        tau = R.dense_solve(m, np.ones(m.shape[0]))
        return float(np.min(tau) * np.max(np.abs(b - m @ x)))
    _patch(monkeypatch, "error_bound", bad)
    with pytest.raises(AssertionError):
        pins.test_error_bound_exact_on_fair_gamblers_ruin(10)


def test_error_bound_with_the_mean_tau_is_caught(monkeypatch):
    def bad(m, b, x):
        tau = R.dense_solve(m, np.ones(m.shape[0]))
        return float(np.mean(tau) * np.max(np.abs(b - m @ x)))
    _patch(monkeypatch, "error_bound", bad)
    with pytest.raises(AssertionError):
        pins.test_error_bound_exact_on_fair_gamblers_ruin(10)


def test_varah_margin_without_absolute_values_is_caught(monkeypatch):
    def bad(m):
        m = sp.csr_matrix(m)
        off = (m - sp.diags(m.diagonal())) @ np.ones(m.shape[0])
        return float(np.min(m.diagonal() - off))
    _patch(monkeypatch, "varah_margin", bad)
    with pytest.raises(AssertionError):
        pins.test_varah_margin_of_chains_is_the_smallest_exit_probability()


def test_varah_margin_with_the_diagonal_in_the_sum_is_caught(monkeypatch):
    def bad(m):
        m = sp.csr_matrix(m)
        return float(np.min(np.abs(m.diagonal()) - abs(m) @ np.ones(m.shape[0])))
    _patch(monkeypatch, "varah_margin", bad)
    with pytest.raises(AssertionError):
        pins.test_varah_bound_attained_on_constant_exit_rows()


def test_supersolution_bound_with_max_over_min_swapped_is_caught(monkeypatch):
    def bad(m, t):
        t = np.asarray(t, float)
        c = float(np.max(sp.csr_matrix(m) @ t))
        return float(np.max(t) / c) if c > 0 else np.inf
    _patch(monkeypatch, "supersolution_norm_bound", bad)
    with pytest.raises(AssertionError):
        pins.test_supersolution_bound_from_an_approximate_tau()
