"""The oracle against what the paper and the mathematics fix (no GPU).

Pins: the worked chain of §2 (partition §2.2, A and b §2.3), the CSR example of §4,
the gambler's-ruin closed form, path sums on tiny acyclic chains (§2 cylinder sets),
set parity against a boolean closure, and the invariants of the method (x in [0,1],
monotone Jacobi from 0 and from 1, agreement of Jacobi / BiCGStab / LU, PROB01 vs
PROB0_ONLY).
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_1210_6412_gb300 import synth
from tests import brute

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def chain_arrays(c):
    return c.n, c.rowptr, c.col, c.val, c.goal


# ------------------------------------------------------------------ §4 CSR example

def test_csr_example_section4():
    g = load("csr_example.json")
    rstart, col, nz = O.csr_from_dense(g["matrix"])
    assert rstart.tolist() == g["rstart"]
    assert col.tolist() == g["col"]
    assert nz.tolist() == g["nonzero"]


def test_canonical_csr_sorts_and_merges():
    # row 0 stored out of order with a duplicate and a stored zero
    rowptr = np.array([0, 4, 5])
    col = np.array([1, 0, 1, 0, 1])
    val = np.array([0.25, 0.5, 0.25, 0.0, 1.0])
    p = O.canonical_csr(2, rowptr, col, val)
    assert p.indptr.tolist() == [0, 2, 3]
    assert p.indices.tolist() == [0, 1, 1]
    assert p.data.tolist() == [0.5, 0.5, 1.0]


# ------------------------------------------------------------------ §2 worked chain

def test_worked_chain_partition_and_system():
    g = load("worked_chain.json")
    c = synth.worked_chain()
    assert np.array_equal(sp.csr_matrix((c.val, c.col, c.rowptr)).toarray(), np.array(g["P"]))
    cls = O.partition(*chain_arrays(c))
    assert np.flatnonzero(cls == O.S0).tolist() == g["S0"]
    assert np.flatnonzero(cls == O.S1).tolist() == g["S1"]
    assert np.flatnonzero(cls == O.SQ).tolist() == g["Sq"]
    q, a, b = O.extract_system(c.n, c.rowptr, c.col, c.val, cls)
    assert q.tolist() == g["Sq"]
    assert np.array_equal(a.toarray(), np.array(g["A"]))
    assert np.array_equal(b, np.array(g["b"], float))


@pytest.mark.parametrize("method", ["dense", "jacobi", "bicgstab"])
def test_worked_chain_solution(method):
    g = load("worked_chain.json")
    c = synth.worked_chain()
    x, cls, _ = O.reach_probabilities(*chain_arrays(c), method=method, eps=1e-15)
    np.testing.assert_allclose(x[g["Sq"]], g["x_Sq"], rtol=0, atol=1e-14)
    assert x[1] == 0.0 and x[3] == 1.0


def test_worked_chain_path_sum_and_cylinder():
    g = load("worked_chain.json")
    p = np.array(g["P"], float)
    # Pr(Cyl(0 3)) = P(0,3) (§2)
    assert p[0, 3] == g["Pr_cyl_03"]
    # path sum over (02)^n 0 3 truncated at depth 2k+1 equals 0.5 * sum_{j<=k} 0.2^j
    tot = sum(0.5 * 0.2 ** j for j in range(60))
    assert abs(tot - g["x_Sq"][0]) < 1e-15


# ------------------------------------------------------------------ closed form

@pytest.mark.parametrize("N,p", [(10, 0.5), (20, 0.4), (20, 0.6), (50, 0.49), (7, 0.9)])
def test_gamblers_ruin_closed_form(N, p):
    c = synth.gamblers_ruin(N, p)
    want = np.array([brute.gambler_closed_form(N, p, i) for i in range(N + 1)])
    for method, tol in (("dense", 1e-12), ("bicgstab", 1e-9), ("jacobi", 1e-8)):
        x, cls, info = O.reach_probabilities(*chain_arrays(c), method=method, eps=1e-13,
                                             max_iter=2_000_000)
        np.testing.assert_allclose(x, want, rtol=0, atol=tol, err_msg=method)
    assert cls[0] == O.S0 and cls[N] == O.S1 and np.all(cls[1:N] == O.SQ)


# ------------------------------------------------------------------ brute force

@pytest.mark.parametrize("seed", range(12))
def test_path_sum_on_acyclic_chains(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 12))
    p, goal = brute.random_dag_chain(rng, n)
    rowptr, col, val = brute.dense_to_csr(p)
    x, cls, _ = O.reach_probabilities(n, rowptr, col, val, goal, method="dense")
    for s in range(n):
        assert abs(x[s] - brute.path_sum(p, goal, s)) < 1e-13


@pytest.mark.parametrize("seed", range(20))
def test_sets_match_boolean_closure(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 60))
    dens = rng.uniform(0.02, 0.3)
    p = (rng.random((n, n)) < dens) * rng.random((n, n))
    for i in range(n):
        if p[i].sum() == 0 or rng.random() < 0.1:
            p[i] = 0
            p[i, i] = 1.0
    p = p / p.sum(axis=1, keepdims=True)
    goal = (rng.random(n) < 0.1).astype(np.uint8)
    rowptr, col, val = brute.dense_to_csr(p)
    s0_ref, s1_ref = brute.sets_by_closure(p, goal)
    cls = O.partition(n, rowptr, col, val, goal)
    assert np.array_equal(cls == O.S0, s0_ref)
    assert np.array_equal(cls == O.S1, s1_ref & ~s0_ref)
    # S=1 and S=0 agree with the values themselves, computed on the PROB0_ONLY system
    x, _, _ = O.reach_probabilities(n, rowptr, col, val, goal, mode=O.PROB0_ONLY, method="dense")
    assert np.all(np.abs(x[cls == O.S1] - 1.0) < 1e-9)
    assert np.all(x[cls == O.S0] == 0.0)
    sq = cls == O.SQ
    assert np.all((x[sq] > 1e-12) & (x[sq] < 1 - 1e-9))


def test_prob1_literal_reading_differs_from_definition():
    """A non-goal state whose only way to S=0 runs through a goal is in S=1 (definition)."""
    # 0 -> 1 (goal) ; goal 1 -> 2 (sink) ; so state 0 reaches S=0 only through GS.
    p = np.array([[0, 1.0, 0], [0, 0, 1.0], [0, 0, 1.0]])
    goal = np.array([0, 1, 0], np.uint8)
    rowptr, col, val = brute.dense_to_csr(p)
    cls = O.partition(3, rowptr, col, val, goal)
    assert cls.tolist() == [O.S1, O.S1, O.S0]


# ------------------------------------------------------------------ invariants

@pytest.fixture(scope="module")
def c1_small():
    return synth.random_chain(n=512, deg=8, goal_frac=0.03, sink_frac=0.03, seed=7)


def test_methods_agree_and_invariants(c1_small):
    c = c1_small
    xd, cls, _ = O.reach_probabilities(*chain_arrays(c), method="dense")
    xj, _, ij = O.reach_probabilities(*chain_arrays(c), method="jacobi", eps=1e-14)
    xb, _, ib = O.reach_probabilities(*chain_arrays(c), method="bicgstab", eps=1e-14)
    assert ij["converged"] and ib["converged"]
    np.testing.assert_allclose(xj, xd, atol=1e-11, rtol=0)
    np.testing.assert_allclose(xb, xd, atol=1e-11, rtol=0)
    assert np.all((xd >= 0) & (xd <= 1))
    assert np.all(xd[cls == O.S1] == 1) and np.all(xd[cls == O.S0] == 0)
    sq = cls == O.SQ
    assert np.all((xd[sq] > 0) & (xd[sq] < 1))
    # PROB0_ONLY gives the same probabilities
    x0, _, _ = O.reach_probabilities(*chain_arrays(c), mode=O.PROB0_ONLY, method="dense")
    np.testing.assert_allclose(x0, xd, atol=1e-12, rtol=0)


def test_jacobi_monotone_sandwich(c1_small):
    c = c1_small
    cls = O.partition(*chain_arrays(c))
    q, a, b = O.extract_system(c.n, c.rowptr, c.col, c.val, cls)
    m = O.system_matrix(a)
    xs = O.dense_solve(m, b)
    lo, hi = [], []
    O.jacobi(m, b, 0.0, 60, history=lo)
    O.jacobi(m, b, 0.0, 60, x0=np.ones(q.size), history=hi)
    prev = np.zeros(q.size)
    for x in lo:
        assert np.all(x >= prev - 1e-15) and np.all(x <= xs + 1e-12)
        prev = x
    prev = np.ones(q.size)
    for x in hi:
        assert np.all(x <= prev + 1e-15) and np.all(x >= xs - 1e-12)
        prev = x


def test_error_bound_certifies(c1_small):
    c = c1_small
    cls = O.partition(*chain_arrays(c))
    q, a, b = O.extract_system(c.n, c.rowptr, c.col, c.val, cls)
    m = O.system_matrix(a)
    xs = O.dense_solve(m, b)
    xj, _, _, _ = O.jacobi(m, b, 1e-6, 100000)
    bound = O.error_bound(m, b, xj)
    assert np.max(np.abs(xj - xs)) <= bound * (1 + 1e-9) + 1e-15


def test_check_chain_rejects_bad_inputs():
    c = synth.worked_chain()
    O.check_chain(*chain_arrays(c))
    bad = c.val.copy(); bad[0] = -0.5
    with pytest.raises(O.OracleInputError):
        O.check_chain(c.n, c.rowptr, c.col, bad, c.goal)
    bad = c.val.copy(); bad[0] = 0.6
    with pytest.raises(O.OracleInputError):
        O.check_chain(c.n, c.rowptr, c.col, bad, c.goal)
    badc = c.col.copy(); badc[0] = 4
    with pytest.raises(O.OracleInputError):
        O.check_chain(c.n, c.rowptr, badc, c.val, c.goal)
    bad = c.val.copy(); bad[0] = np.nan
    with pytest.raises(O.OracleInputError):
        O.check_chain(c.n, c.rowptr, c.col, bad, c.goal)


def test_empty_goal_set_gives_zero():
    c = synth.random_chain(n=64, deg=4, seed=3)
    goal = np.zeros(c.n, np.uint8)
    x, cls, _ = O.reach_probabilities(c.n, c.rowptr, c.col, c.val, goal)
    assert np.all(cls == O.S0) and np.all(x == 0)


@pytest.mark.parametrize("N,p", [(3, 0.5), (12, 0.4), (20, 0.45)])
def test_bicgstab_finite_termination(N, p):
    """§3: in exact arithmetic BiCGStab ends within n iterations for an n x n system."""
    c = synth.gamblers_ruin(N, p)
    cls = O.partition(*chain_arrays(c))
    q, a, b = O.extract_system(c.n, c.rowptr, c.col, c.val, cls)
    x, it, res, ok = O.bicgstab(O.system_matrix(a), b, 1e-11, q.size + 2)
    assert ok and it <= q.size + 2
    want = np.array([brute.gambler_closed_form(N, p, i) for i in q])
    np.testing.assert_allclose(x, want, atol=1e-9, rtol=0)


def test_bicgstab_restart_after_breakdown():
    """With the shadow vector q = b sparse, q . r can vanish exactly; one restart with
    q = r recovers and the answer matches the direct solve."""
    c = synth.table1_chain(92, 211)
    cls = O.partition(*chain_arrays(c))
    q, a, b = O.extract_system(c.n, c.rowptr, c.col, c.val, cls)
    m = O.system_matrix(a)
    x, it, res, ok = O.bicgstab(m, b, 1e-14, 500)
    assert ok
    np.testing.assert_allclose(x, O.dense_solve(m, b), atol=1e-12, rtol=0)


def test_bicgstab_iteration_cap():
    c = synth.gamblers_ruin(200, 0.5)
    cls = O.partition(*chain_arrays(c))
    q, a, b = O.extract_system(c.n, c.rowptr, c.col, c.val, cls)
    x, it, res, ok = O.bicgstab(O.system_matrix(a), b, 1e-30, 3)
    assert not ok and it == 3


# ------------------------------------------------------------------ gradients

def _fd_on_sq_rows(c, init, entries, h=1e-6):
    """Central differences of x_init in P entries of S? rows (linear system kept fixed)."""
    cls = O.partition(*chain_arrays(c))
    out = []
    for k in entries:
        vals = []
        for sgn in (+1, -1):
            v = c.val.copy()
            v[k] += sgn * h
            q, a, b = O.extract_system(c.n, c.rowptr, c.col, v, cls)
            xq = O.dense_solve(O.system_matrix(a), b)
            vals.append(O.full_vector(c.n, cls, q, xq)[init])
        out.append((vals[0] - vals[1]) / (2 * h))
    return np.array(out)


def test_grad_p_matches_central_differences():
    c = synth.random_chain(n=200, deg=5, goal_frac=0.05, sink_frac=0.05, seed=11)
    g, x, cls = O.grad_p(*chain_arrays(c), init=c.init)
    assert cls[c.init] == O.SQ
    row = np.repeat(np.arange(c.n), np.diff(c.rowptr))
    rng = np.random.default_rng(0)
    cand = np.flatnonzero(cls[row] == O.SQ)
    ks = rng.choice(cand, size=25, replace=False)
    fd = _fd_on_sq_rows(c, c.init, ks)
    np.testing.assert_allclose(g[ks], fd, rtol=1e-6, atol=1e-9)
    assert np.all(g[cls[row] != O.SQ] == 0)


def test_grad_theta_matches_central_differences():
    pc = synth.parametric_chain(n=300, n_classes=8, goal_frac=0.03, sink_frac=0.03, seed=5)

    def x_init(theta):
        p = O.softmax_probs(pc.rowptr, pc.cls, pc.offset, theta)
        x, _, _ = O.reach_probabilities(pc.n, pc.rowptr, pc.col, p, pc.goal, method="dense")
        return x[pc.init]

    p = O.softmax_probs(pc.rowptr, pc.cls, pc.offset, pc.theta)
    np.testing.assert_allclose(np.add.reduceat(p, pc.rowptr[:-1]), 1.0, atol=1e-14)
    g_p, x, cls = O.grad_p(pc.n, pc.rowptr, pc.col, p, pc.goal, pc.init)
    assert cls[pc.init] == O.SQ
    g_t = O.grad_theta(pc.rowptr, p, g_p, pc.cls, 8)
    h = 1e-6
    fd = np.array([(x_init(pc.theta + h * np.eye(8)[j]) - x_init(pc.theta - h * np.eye(8)[j])) / (2 * h)
                   for j in range(8)])
    np.testing.assert_allclose(g_t, fd, rtol=1e-5, atol=1e-9)


# ---------------------------------------------------------------- §8: SCCs, reverse topological order

def _random_digraph_system(seed, n_max=60):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(1, n_max))
    dens = rng.uniform(0.01, 0.15)
    adj = (rng.random((n, n)) < dens) & ~np.eye(n, dtype=bool)
    w = adj * rng.uniform(0.05, 1.0, (n, n))
    # substochastic rows that leak to S=1 / S=0: (I - A) is an M-matrix
    a = w / (w.sum(axis=1, keepdims=True) + rng.uniform(0.1, 1.0, (n, 1)))
    b = rng.uniform(0.0, 1.0, n) * (1.0 - a.sum(axis=1))
    return adj, sp.csr_matrix(a), b


@pytest.mark.parametrize("seed", range(25))
def test_scc_labels_and_levels_match_brute_force(seed):
    adj, a, _ = _random_digraph_system(seed)
    lab = O.scc_labels(a)
    assert np.array_equal(lab, brute.scc_by_closure(adj))
    lev = O.scc_levels(a, lab)
    assert np.array_equal(lev, brute.condensation_height(adj, lab))


@pytest.mark.parametrize("seed", range(10))
def test_scc_levels_order_every_edge(seed):
    """Every edge goes to the same component at the same level or to a lower level."""
    adj, a, _ = _random_digraph_system(seed, n_max=200)
    lab = O.scc_labels(a)
    lev = O.scc_levels(a, lab)
    i, j = np.nonzero(adj)
    same = lab[i] == lab[j]
    assert np.all(lev[i][same] == lev[j][same])
    assert np.all(lev[i][~same] > lev[j][~same])


@pytest.mark.parametrize("seed", range(10))
def test_block_jacobi_matches_lu(seed):
    _, a, b = _random_digraph_system(seed, n_max=200)
    m = sp.identity(a.shape[0], format="csr") - a
    x, sweeps, nl, ok = O.block_jacobi(m, b, 1e-14, 100_000)
    assert ok
    assert np.max(np.abs(x - O.dense_solve(m, b))) < 1e-12
    assert nl == (O.scc_levels(a, O.scc_labels(a)).max() + 1 if a.shape[0] else 0)


def test_block_jacobi_on_a_dag_takes_two_sweeps_per_level():
    """Acyclic system: every level is exact after one sweep and the second sees no change."""
    rng = np.random.default_rng(77)
    n = 300
    adj = np.triu(rng.random((n, n)) < 0.02, k=1)          # edges only to higher rows
    perm = rng.permutation(n)
    adj = adj[np.ix_(perm, perm)]
    w = adj * rng.uniform(0.1, 1.0, (n, n))
    a = sp.csr_matrix(w / (w.sum(axis=1, keepdims=True) + 0.5))
    b = rng.uniform(0.0, 1.0, n) * (1.0 - np.asarray(a.sum(axis=1)).ravel())
    lab = O.scc_labels(a)
    assert np.array_equal(lab, np.arange(n))                  # every row its own component
    m = sp.identity(n, format="csr") - a
    x, sweeps, nl, ok = O.block_jacobi(m, b, 1e-300, 10)
    assert ok and sweeps == 2 * nl
    assert np.max(np.abs(x - O.dense_solve(m, b))) < 1e-14
    assert nl == brute.condensation_height(adj, lab).max() + 1


def test_scc_of_the_worked_chain():
    """S? = {s0, s2} of the worked chain form one cycle (s0 -> s2 -> s0): one component."""
    c = synth.worked_chain()
    cls = O.partition(*chain_arrays(c))
    q, a, b = O.extract_system(c.n, c.rowptr, c.col, c.val, cls)
    lab = O.scc_labels(a)
    assert lab.tolist() == [1, 1]
    assert O.scc_levels(a, lab).tolist() == [0, 0]
    x, sweeps, nl, ok = O.block_jacobi(O.system_matrix(a), b, 1e-15, 10_000)
    assert ok and nl == 1
    assert np.max(np.abs(x - np.array([0.625, 0.25]))) < 1e-14


def test_scc_labels_leaves_its_input_alone():
    _, a, _ = _random_digraph_system(3, n_max=80)
    a = a + sp.identity(a.shape[0], format="csr") * 0.25        # stored diagonal
    before = (a.indptr.copy(), a.indices.copy(), a.data.copy())
    O.scc_labels(a)
    assert all(np.array_equal(x, y) for x, y in zip(before, (a.indptr, a.indices, a.data)))


# ---------------------------------------------------------------- softmax parametrisation (exact values)
# P_e = exp(theta[class_e] + offset_e) / sum over the row's out-edges: pinned by values the
# definition fixes, independently of how the oracle evaluates it.

def _one_row(cls_e, offset, theta):
    rowptr = np.array([0, len(cls_e)], np.int64)
    return O.softmax_probs(rowptr, np.asarray(cls_e, np.int32), np.asarray(offset, float),
                           np.asarray(theta, float))


def test_softmax_offsets_of_one_class_give_exact_shares():
    """Three edges of one class with offsets (0, ln 2, ln 3): weights 1 : 2 : 3."""
    p = _one_row([0, 0, 0], [0.0, np.log(2.0), np.log(3.0)], [0.7])
    np.testing.assert_allclose(p, [1 / 6, 1 / 3, 1 / 2], rtol=1e-15, atol=0)


def test_softmax_class_parameters_set_edge_ratios():
    """Equal offsets, classes 1 and 0 with theta differing by ln 4: the edge ratio is 4."""
    theta = np.array([0.3, 0.3 + np.log(4.0)])
    p = _one_row([1, 0], [0.5, 0.5], theta)
    np.testing.assert_allclose(p, [0.8, 0.2], rtol=1e-15, atol=0)
    # class and offset both enter: logits ln 3 + 0 and 0 + ln 2 -> 3 : 2
    p = _one_row([0, 1], [np.log(3.0), 0.0], [0.0, np.log(2.0)])
    np.testing.assert_allclose(p, [0.6, 0.4], rtol=1e-15, atol=0)


def test_softmax_single_edge_and_shift_invariance():
    pc = synth.parametric_chain(n=400, n_classes=8, seed=21)
    p = O.softmax_probs(pc.rowptr, pc.cls, pc.offset, pc.theta)
    np.testing.assert_allclose(np.add.reduceat(p, pc.rowptr[:-1]), 1.0, rtol=0, atol=1e-15)
    single = np.flatnonzero(np.diff(pc.rowptr) == 1)
    assert single.size and np.all(p[pc.rowptr[single]] == 1.0)
    # a constant added to every theta cancels in every row
    p2 = O.softmax_probs(pc.rowptr, pc.cls, pc.offset, pc.theta + 5.25)
    np.testing.assert_allclose(p2, p, rtol=1e-13, atol=0)


def test_softmax_theta_of_a_class_moves_only_its_rows():
    pc = synth.parametric_chain(n=400, n_classes=8, seed=22)
    p = O.softmax_probs(pc.rowptr, pc.cls, pc.offset, pc.theta)
    row = np.repeat(np.arange(pc.n), np.diff(pc.rowptr))
    for c in (0, 5):
        th = pc.theta.copy()
        th[c] += 0.5
        q = O.softmax_probs(pc.rowptr, pc.cls, pc.offset, th)
        rows_c = np.zeros(pc.n, bool)
        rows_c[row[pc.cls == c]] = True
        moved = np.abs(q - p) > 0
        assert np.all(~moved[~rows_c[row]])                       # other rows untouched
        # rows that mix class c with other classes change; class-c edges gain weight
        mixed = rows_c & np.bincount(row, weights=(pc.cls != c), minlength=pc.n).astype(bool)
        assert np.all(moved[mixed[row]])
        assert np.all(q[(pc.cls == c) & mixed[row]] > p[(pc.cls == c) & mixed[row]])


def test_softmax_large_logits_per_row():
    """Rows with logits near +-700: each row is computed from its own logits (exp would
    overflow or underflow if the row's shift came from another row)."""
    rowptr = np.array([0, 2, 4], np.int64)
    cls_e = np.array([0, 1, 2, 3], np.int32)
    theta = np.array([700.0, 700.0 + np.log(3.0), -700.0, -700.0 + np.log(7.0)])
    p = O.softmax_probs(rowptr, cls_e, np.zeros(4), theta)
    np.testing.assert_allclose(p, [0.25, 0.75, 0.125, 0.875], rtol=1e-13, atol=0)


# ---------------------------------------------------------------- error bounds (exact values)

def _fair_gambler_system(N):
    c = synth.gamblers_ruin(N, 0.5)
    cls = O.partition(*chain_arrays(c))
    q, a, b = O.extract_system(c.n, c.rowptr, c.col, c.val, cls)
    return q, O.system_matrix(a), b


@pytest.mark.parametrize("N", [2, 9, 10, 31])
def test_error_bound_exact_on_fair_gamblers_ruin(N):
    """Fair walk on 0..N: tau_i = i (N - i), the expected duration, so ||M^-1||_inf is
    max_i i (N - i) = floor(N/2) ceil(N/2).  At x = x* + c tau the residual is -c 1, the
    error is c max tau and the bound is attained: error_bound = c floor(N/2) ceil(N/2)."""
    q, m, b = _fair_gambler_system(N)
    tau = q * (N - q)                                  # rows of S? are the states 1..N-1
    xs = q / N
    c = 1e-3
    bound = O.error_bound(m, b, xs + c * tau)
    want = c * (N // 2) * ((N + 1) // 2)
    assert abs(bound - want) <= 1e-11 * want
    # one entry perturbed by c: residual max is c (the entry's own row), bound c max tau
    k = len(q) // 2
    x = xs.copy()
    x[k] += c
    assert abs(O.error_bound(m, b, x) - c * (N // 2) * ((N + 1) // 2)) <= 1e-11 * c * N * N
    # the supersolution bound from the exact tau is the same norm
    assert abs(O.supersolution_norm_bound(m, tau) - (N // 2) * ((N + 1) // 2)) <= 1e-12 * N * N


def test_supersolution_bound_from_an_approximate_tau():
    """Any tau' with M tau' >= c 1 bounds the norm from above; it tightens as tau' -> tau."""
    N = 24
    q, m, _ = _fair_gambler_system(N)
    exact = (N // 2) * ((N + 1) // 2)
    tau = (q * (N - q)).astype(float)
    for scale in (1.5, 1.01, 1.0 + 1e-9):
        assert exact <= O.supersolution_norm_bound(m, scale * tau) <= scale * exact * (1 + 1e-12)
    assert O.supersolution_norm_bound(m, 0.5 * tau) >= exact * (1 - 1e-12)
    # a vector with M t <= 0 somewhere certifies nothing
    t = tau.copy()
    t[3] += 5.0
    assert O.supersolution_norm_bound(m, t) == np.inf


def test_varah_bound_attained_on_constant_exit_rows():
    """Rows that all leave S? with the same probability e: M 1 = e 1, so ||M^-1|| = 1/e,
    the margin is e, and at x = x* + c 1 both bounds equal the true error c."""
    rng = np.random.default_rng(4)
    n, e = 40, 0.125
    w = rng.uniform(0.1, 1.0, (n, n)) * (rng.random((n, n)) < 0.3)
    np.fill_diagonal(w, 0.0)
    w[np.arange(n), (np.arange(n) + 1) % n] += 0.1                  # no empty row
    a = sp.csr_matrix((1.0 - e) * w / w.sum(axis=1, keepdims=True))
    m = sp.identity(n, format="csr") - a
    b = np.full(n, e * 0.25)
    xs = O.dense_solve(m, b)
    c = 1e-3
    assert abs(O.varah_margin(m) - e) <= 1e-15
    assert abs(O.varah_bound(m, b, xs + c) - c) <= 1e-11 * c
    assert abs(O.error_bound(m, b, xs + c) - c) <= 1e-11 * c
    # a bound that ignores the exit margin (residual alone) is e times too small
    assert O.varah_bound(m, b, xs + c) >= 0.99 * c > 1.01 * e * c


def test_varah_margin_of_chains_is_the_smallest_exit_probability():
    """On the worked chain's system A = [[0, .5], [.4, 0]]: exits 0.5 and 0.6, margin 0.5;
    on the fair gambler's ruin interior rows never leave S? in one step: margin 0, no bound."""
    c = synth.worked_chain()
    cls = O.partition(*chain_arrays(c))
    q, a, b = O.extract_system(c.n, c.rowptr, c.col, c.val, cls)
    m = O.system_matrix(a)
    assert O.varah_margin(m) == 0.5
    assert O.varah_bound(m, b, np.array([0.625, 0.25]) + 1e-3) == pytest.approx(
        max(abs(b - m @ (np.array([0.625, 0.25]) + 1e-3))) / 0.5, rel=1e-15)
    _, mg, bg = _fair_gambler_system(10)
    assert O.varah_margin(mg) == 0.0
    assert O.varah_bound(mg, bg, np.zeros(9)) == np.inf
    # for a general diagonally dominant system the margin is |M_ii| - sum |M_ij|
    md = sp.csr_matrix(np.array([[4.0, -1.0, 2.0], [1.0, -5.0, 1.0], [0.0, 3.0, 3.5]]))
    assert O.varah_margin(md) == pytest.approx(0.5, abs=1e-15)
