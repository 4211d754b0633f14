"""CPU FP64 oracle for reachability probabilities in a discrete-time Markov chain.

TEST INFRASTRUCTURE, not part of the product.  Only the test-suite, the smoke check in
``__graft_entry__`` and the CPU-baseline / reference leg of ``bench.py`` may import it.
It shares no code with the CUDA library and never calls it; the library never calls it.

Plain numpy / scipy.sparse in float64, one function per step of the paper, in the
paper's order and notation:

  §2, §4     Markov chain (S, P, s0) with row-stochastic P, compressed row storage
             -> csr_from_dense, canonical_csr, check_chain
  §2.2       S=0 / S=1 / S? by backward graph search            -> prob0, prob1, partition
  §2.3       A = P restricted to S?, b_s = Pr(s |= X GS),
             (I - A) x = b                                        -> extract_system, system_matrix
  §3.1       Jacobi                                               -> jacobi
  §3.2       BiCGStab (van der Vorst, unpreconditioned)           -> bicgstab
  §1, §2.3   the direct O(n^3) route (LU with partial pivoting)   -> dense_solve
  (none)     adjoint solve and parameter gradients                -> adjoint, grad_p,
                                                                     softmax_probs, grad_theta
  (none)     a-posteriori error bounds: exact ||M^-1|| from tau = M^-1 1, Varah's
             row-dominance bound, and the bound from an approximate tau -> error_bound,
                                                                     varah_margin, varah_bound,
                                                                     supersolution_norm_bound
  §8         strongly connected components of the digraph of A, solved in reverse
             topological order (the future-work idea of §8)      -> scc_labels, scc_levels,
                                                                     block_jacobi

Where the paper is silent or ambiguous the oracle takes these readings:
  * initial vector x = 0 for both methods (the listings draw it at random);
  * BiCGStab shadow vector q = r0 = b - M x0 (the listing asks only q . r != 0);
  * S=1 follows the definition of §2.2 (states that reach S=0 along a path that avoids
    GS are not in S=1), and b_s sums P(s, s') over all of S=1, which is the paper's
    Pr(s |= X GS) whenever S=1 = GS;
  * Jacobi stops when max|x' - x| < eps; BiCGStab stops when max|s| < eps after the
    a-step (then x += a p) or max|r| < eps after the w-step; at most max_iter iterations;
  * a BiCGStab breakdown (q.r = 0, q.v = 0 or w = 0) restarts once with q = r, p = v = 0.

Large-case oracles: the level-synchronous BFS and the scipy matrix-vector products are
O(m) per level / sweep, so the oracle finishes n = 8M chains in seconds per step.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

S0, S1, SQ = 0, 1, 2          # state classes: S=0, S=1, S?
PROB01, PROB0_ONLY = 0, 1     # partition modes


class OracleInputError(ValueError):
    pass


class BreakdownError(RuntimeError):
    pass


# ---------------------------------------------------------------- §2, §4: the chain

def csr_from_dense(a):
    """Compressed row storage of a dense matrix (§4): rstart, col, nonzero."""
    a = np.asarray(a, np.float64)
    rstart, col, nonzero = [0], [], []
    for i in range(a.shape[0]):
        for j in range(a.shape[1]):
            if a[i, j] != 0.0:
                col.append(j)
                nonzero.append(a[i, j])
        rstart.append(len(col))
    return (np.asarray(rstart, np.int64), np.asarray(col, np.int32), np.asarray(nonzero, np.float64))


def as_matrix(n, rowptr, col, val):
    return sp.csr_matrix((np.asarray(val, np.float64), np.asarray(col, np.int64),
                          np.asarray(rowptr, np.int64)), shape=(n, n))


def canonical_csr(n, rowptr, col, val):
    """Sort columns within each row, sum duplicates and drop stored zeros.

    An edge s -> s' exists iff P(s, s') > 0 (§2.2), so a stored zero is no edge.
    """
    p = as_matrix(n, rowptr, col, val).copy()
    p.sum_duplicates()
    p.eliminate_zeros()
    p.sort_indices()
    return p


def check_chain(n, rowptr, col, val, goal, tol=1e-9):
    """Reject inputs that are not a Markov chain with a goal set (§2).

    P(s, s') must lie in [0, 1], every row must sum to 1 within ``tol``, columns must be
    states, and the goal mask must have one byte per state.
    """
    rowptr = np.asarray(rowptr)
    col = np.asarray(col)
    val = np.asarray(val, np.float64)
    if n < 1:
        raise OracleInputError("a chain needs at least one state")
    if rowptr.shape != (n + 1,) or rowptr[0] != 0 or np.any(np.diff(rowptr) < 0):
        raise OracleInputError("rowptr must be non-decreasing from 0 with n+1 entries")
    m = int(rowptr[-1])
    if col.shape != (m,) or val.shape != (m,):
        raise OracleInputError("col and val need rowptr[n] entries")
    if m and (col.min() < 0 or col.max() >= n):
        raise OracleInputError("column index outside [0, n)")
    if not np.all(np.isfinite(val)) or np.any(val < 0) or np.any(val > 1):
        raise OracleInputError("transition probabilities must be finite and in [0, 1]")
    rowsum = as_matrix(n, rowptr, col, val) @ np.ones(n)
    if np.any(np.abs(rowsum - 1.0) > tol):
        raise OracleInputError("every row of P must sum to 1")
    if np.asarray(goal).shape != (n,):
        raise OracleInputError("goal mask needs n entries")


# ---------------------------------------------------------------- §2.2: partition

def _backward_reach(p, sources, allowed):
    """States from which a state of ``sources`` is reachable in the underlying digraph.

    Level-synchronous search over reversed edges: a predecessor u of a reached state is
    added when u is ``allowed``.  Sources themselves count as reached.
    """
    n = p.shape[0]
    pred = p.T.tocsr()                      # row v lists every u with P(u, v) > 0
    reached = np.asarray(sources, bool).copy()
    frontier = np.flatnonzero(reached)
    while frontier.size:
        lo = pred.indptr[frontier]
        hi = pred.indptr[frontier + 1]
        cnt = hi - lo
        if cnt.sum() == 0:
            break
        first = np.repeat(lo - np.concatenate(([0], np.cumsum(cnt)[:-1])), cnt)
        u = pred.indices[first + np.arange(cnt.sum())]
        u = np.unique(u[allowed[u] & ~reached[u]])
        reached[u] = True
        frontier = u
    assert reached.shape == (n,)
    return reached


def prob0(n, rowptr, col, val, goal):
    """S=0: the complement of the states that can reach GS (GS included) (§2.2)."""
    p = canonical_csr(n, rowptr, col, val)
    can_reach = _backward_reach(p, np.asarray(goal) != 0, np.ones(n, bool))
    return ~can_reach


def prob1(n, rowptr, col, val, goal, s0=None):
    """S=1: the states that cannot reach S=0 along a path avoiding GS (§2.2, definition).

    A state that reaches S=0 with positive probability without first meeting a goal has
    Pr(s |= <> GS) < 1; every other state reaches GS almost surely.
    """
    p = canonical_csr(n, rowptr, col, val)
    g = np.asarray(goal) != 0
    if s0 is None:
        s0 = prob0(n, rowptr, col, val, goal)
    bad = _backward_reach(p, s0, ~g)
    return ~bad


def partition(n, rowptr, col, val, goal, mode=PROB01):
    """Class per state: 0 for S=0, 1 for S=1, 2 for S? (§2.2).

    PROB0_ONLY takes S=1 = GS, so S? = S \\ (S=0 u GS): the system the paper writes in §2.3.
    """
    s0 = prob0(n, rowptr, col, val, goal)
    if mode == PROB01:
        s1 = prob1(n, rowptr, col, val, goal, s0)
    elif mode == PROB0_ONLY:
        s1 = np.asarray(goal) != 0
    else:
        raise OracleInputError("unknown partition mode")
    cls = np.full(n, SQ, np.uint8)
    cls[s1] = S1
    cls[s0] = S0
    return cls


# ---------------------------------------------------------------- §2.3: the system

def extract_system(n, rowptr, col, val, cls):
    """A = P restricted to S? x S?, b_s = sum of P(s, s') over s' in S=1 (§2.3).

    Returns (q, a, b): q = S? states in ascending order (row i of the system is state
    q[i]), ``a`` the n? x n? CSR matrix A (diagonal included), ``b`` float64[n?].
    """
    p = canonical_csr(n, rowptr, col, val)
    q = np.flatnonzero(cls == SQ)
    rows = p[q]
    a = rows[:, q].tocsr()
    b = rows[:, np.flatnonzero(cls == S1)] @ np.ones(int(np.count_nonzero(cls == S1)))
    a.sort_indices()
    return q, a, np.asarray(b, np.float64)


def system_matrix(a):
    """M = I - A (§2.3)."""
    nq = a.shape[0]
    m = (sp.identity(nq, format="csr") - a).tocsr()
    m.sort_indices()
    return m


# ---------------------------------------------------------------- §3.1: Jacobi

def jacobi(m, b, eps, max_iter, x0=None, history=None):
    """Jacobi for M x = b (§3.1): x_i <- (b_i - sum_{j != i} M_ij x'_j) / M_ii.

    ``x'`` is the previous iterate (double buffer).  Stops when max|x - x'| < eps.
    Returns (x, iterations, last max|x - x'|, converged).  When ``history`` is a list,
    every iterate is appended to it.
    """
    m = sp.csr_matrix(m)
    diag = m.diagonal()
    off = (m - sp.diags(diag)).tocsr()
    off.sort_indices()
    x = np.zeros(m.shape[0]) if x0 is None else np.array(x0, np.float64)
    delta = np.inf
    for it in range(1, max_iter + 1):
        x_prev = x
        x = (b - off @ x_prev) / diag
        delta = float(np.max(np.abs(x - x_prev))) if x.size else 0.0
        if history is not None:
            history.append(x.copy())
        if delta < eps:
            return x, it, delta, True
    return x, max_iter, delta, False


# ---------------------------------------------------------------- §3.2: BiCGStab

def bicgstab(m, b, eps, max_iter, x0=None):
    """Unpreconditioned BiCGStab for M x = b, steps as in §3.2.

    Scalars keep the paper's names: y (rho), a (alpha), w (omega).  Returns
    (x, iterations, final max-norm residual estimate, converged).
    """
    m = sp.csr_matrix(m)
    x = np.zeros(m.shape[0]) if x0 is None else np.array(x0, np.float64)
    r = b - m @ x
    if x.size == 0 or np.max(np.abs(r)) < eps:
        return x, 0, float(np.max(np.abs(r))) if r.size else 0.0, True
    q = r.copy()
    y = a = w = 1.0
    v = np.zeros_like(x)
    p = np.zeros_like(x)
    restarted = False
    r_norm = float(np.max(np.abs(r)))
    for it in range(1, max_iter + 1):
        y_prev = y
        y = float(q @ r)
        if y == 0.0:
            if restarted:
                raise BreakdownError("q . r = 0 after restart")
            restarted = True
            q, p, v = r.copy(), np.zeros_like(x), np.zeros_like(x)
            y_prev, a, w = 1.0, 1.0, 1.0
            y = float(q @ r)
        p = r + (y * a) / (y_prev * w) * (p - w * v)
        v = m @ p
        qv = float(q @ v)
        if qv == 0.0:
            if restarted:
                raise BreakdownError("q . v = 0 after restart")
            restarted = True
            q, p, v = r.copy(), r.copy(), m @ r
            y = float(q @ r)
            qv = float(q @ v)
            if qv == 0.0:
                raise BreakdownError("q . v = 0")
        a = y / qv
        s = r - a * v
        s_norm = float(np.max(np.abs(s)))
        if s_norm < eps:
            x = x + a * p
            return x, it, s_norm, True
        t = m @ s
        tt = float(t @ t)
        w = float(t @ s) / tt
        x = x + a * p + w * s
        r = s - w * t
        r_norm = float(np.max(np.abs(r)))
        if r_norm < eps:
            return x, it, r_norm, True
        if w == 0.0:
            if restarted:
                raise BreakdownError("w = 0 after restart")
            restarted = True
            q, p, v = r.copy(), np.zeros_like(x), np.zeros_like(x)
            y, a, w = 1.0, 1.0, 1.0
    return x, max_iter, r_norm, False


# ---------------------------------------------------------------- direct route

def dense_solve(m, b):
    """x = M^-1 b by LU with partial pivoting (LAPACK gesv); small systems only."""
    md = m.toarray() if sp.issparse(m) else np.asarray(m, np.float64)
    if md.shape[0] == 0:
        return np.zeros(0)
    return np.linalg.solve(md, b)


# ---------------------------------------------------------------- whole pipeline

def full_vector(n, cls, q, xq):
    """x over all states: 1 on S=1, 0 on S=0, the solved values on S? (§2.3)."""
    x = np.zeros(n)
    x[cls == S1] = 1.0
    x[q] = xq
    return x


def reach_probabilities(n, rowptr, col, val, goal, mode=PROB01, method="dense", eps=1e-12,
                        max_iter=1_000_000):
    """Pr(s |= <> GS) for every state s (§2.1): partition, extract, solve, assemble."""
    check_chain(n, rowptr, col, val, goal)
    cls = partition(n, rowptr, col, val, goal, mode)
    q, a, b = extract_system(n, rowptr, col, val, cls)
    mm = system_matrix(a)
    if method == "dense":
        xq = dense_solve(mm, b)
        info = {"iters": 0}
    elif method == "jacobi":
        xq, it, delta, ok = jacobi(mm, b, eps, max_iter)
        info = {"iters": it, "delta": delta, "converged": ok}
    elif method == "bicgstab":
        xq, it, res, ok = bicgstab(mm, b, eps, max_iter)
        info = {"iters": it, "resid": res, "converged": ok}
    else:
        raise OracleInputError("unknown method")
    return full_vector(n, cls, q, xq), cls, info


def error_bound(m, b, x):
    """Certified max-norm error of x for M x = b when M = I - A is an M-matrix.

    ||x* - x|| <= ||M^-1|| ||b - M x||, and ||M^-1||_inf = max_i tau_i where M tau = 1
    (tau = expected number of steps spent in S?).  Dense route: small systems only.
    """
    tau = dense_solve(m, np.ones(m.shape[0]))
    r = b - m @ x
    return float(np.max(tau) * np.max(np.abs(r))) if r.size else 0.0


def varah_margin(m):
    """min_i (|M_ii| - sum_{j != i} |M_ij|): the row-dominance margin of M.

    For a chain's M = I - A this is the smallest one-step probability of leaving S?
    (into S=0 or S=1).  When it is positive, ||M^-1||_inf <= 1 / margin (Varah 1975).
    """
    m = sp.csr_matrix(m)
    if m.shape[0] == 0:
        return np.inf
    diag = np.abs(m.diagonal())
    off = abs(m - sp.diags(m.diagonal())) @ np.ones(m.shape[0])
    return float(np.min(diag - off))


def varah_bound(m, b, x):
    """Certified max-norm error of x for M x = b from Varah's bound: ||b - M x|| / margin.

    Valid for any strictly row-diagonally-dominant M; +inf when the margin is not positive.
    """
    r = b - sp.csr_matrix(m) @ x
    if r.size == 0:
        return 0.0
    c = varah_margin(m)
    return float(np.max(np.abs(r)) / c) if c > 0 else np.inf


def supersolution_norm_bound(m, tau_tilde):
    """Upper bound of ||M^-1||_inf from any vector with M tau_tilde >= c 1, c > 0.

    For an M-matrix M = I - A (A >= 0, spectral radius of A below 1) the inverse is
    entrywise non-negative, so M (tau_tilde - c tau) >= 0 gives tau <= tau_tilde / c for the
    exact tau = M^-1 1, and ||M^-1||_inf = max_i tau_i <= max_i tau_tilde_i / c.  An
    approximate tau (from any solver) thus certifies the norm; +inf when c <= 0.
    """
    t = np.asarray(tau_tilde, np.float64)
    if t.size == 0:
        return 0.0
    c = float(np.min(sp.csr_matrix(m) @ t))
    return float(np.max(t) / c) if c > 0 else np.inf


# ---------------------------------------------------------------- §8: SCCs in reverse topological order

def scc_labels(a):
    """Strongly connected component of every row of the digraph of A (§8).

    The digraph has an edge i -> j for every off-diagonal A_ij != 0 (the diagonal sits
    in d and links a state only to itself).  Rows i and j share a component exactly when
    each reaches the other.  The components come from scipy's strong-connectivity
    routine (a library step); each is labelled by its largest row index, a name that
    does not depend on how the components were found.
    """
    import scipy.sparse.csgraph as csg
    a = sp.csr_matrix(a)
    nq = a.shape[0]
    if nq == 0:
        return np.zeros(0, np.int64)
    pat = sp.csr_matrix((np.ones(a.nnz), a.indices.copy(), a.indptr.copy()), shape=a.shape)
    pat.setdiag(0)
    pat.eliminate_zeros()
    _, comp = csg.connected_components(pat, directed=True, connection="strong")
    top = np.full(comp.max() + 1, -1, np.int64)
    np.maximum.at(top, comp, np.arange(nq))
    return top[comp]


def scc_levels(a, labels):
    """Level of every row: its component's height in the condensation DAG (§8).

    A component without edges to other components has level 0; any other component
    sits one above the highest component it has an edge to.  Components of one level
    never link to each other, and every edge leaves a level for a lower one, so solving
    level 0, 1, 2, ... in turn is the reverse topological order of §8.  Computed by
    peeling the condensation from its sinks, one level per pass.
    """
    a = sp.csr_matrix(a)
    nq = a.shape[0]
    labels = np.asarray(labels, np.int64)
    row = np.repeat(np.arange(nq), np.diff(a.indptr))
    src, dst = labels[row], labels[a.indices]
    keep = src != dst
    pairs = np.unique(np.stack([src[keep], dst[keep]], 1), axis=0) if keep.any() else np.zeros((0, 2), np.int64)
    comps = np.unique(labels)
    out_deg = dict.fromkeys(comps.tolist(), 0)
    preds = {c: [] for c in comps.tolist()}
    for u, v in pairs.tolist():
        out_deg[u] += 1
        preds[v].append(u)
    level = {}
    frontier = [c for c in comps.tolist() if out_deg[c] == 0]
    h = 0
    while frontier:
        nxt = []
        for c in frontier:
            level[c] = h
        for c in frontier:
            for u in preds[c]:
                out_deg[u] -= 1
                if out_deg[u] == 0:
                    nxt.append(u)
        frontier = nxt
        h += 1
    if len(level) != comps.size:
        raise OracleInputError("condensation has a cycle")   # impossible for true SCCs
    return np.array([level[c] for c in labels.tolist()], np.int64)


def block_jacobi(m, b, eps, max_iter, labels=None, levels=None):
    """Jacobi for M x = b one level of SCCs at a time, lowest level first (§8, §3.1).

    Rows of level h depend only on rows of their own components and of lower levels,
    which are already solved; so each level runs the Jacobi sweep of §3.1 on its own
    rows, with every other row held fixed, until max|x - x'| < eps over those rows.
    Returns (x, total sweeps, number of levels, converged).  ``max_iter`` bounds the
    sweeps of each level.
    """
    m = sp.csr_matrix(m)
    nq = m.shape[0]
    diag = m.diagonal()
    off = (m - sp.diags(diag)).tocsr()
    off.sort_indices()
    a = -off
    if labels is None:
        labels = scc_labels(a)
    if levels is None:
        levels = scc_levels(a, labels)
    x = np.zeros(nq)
    sweeps = 0
    n_levels = int(levels.max()) + 1 if nq else 0
    for h in range(n_levels):
        rows = np.flatnonzero(levels == h)
        sub = off[rows]
        ok = False
        for _ in range(max_iter):
            new = (b[rows] - sub @ x) / diag[rows]
            delta = float(np.max(np.abs(new - x[rows])))
            x[rows] = new
            sweeps += 1
            if delta < eps:
                ok = True
                break
        if not ok:
            return x, sweeps, n_levels, False
    return x, sweeps, n_levels, True


# ---------------------------------------------------------------- gradients (not in the paper)

def adjoint(m, init_row, eps=1e-14, max_iter=1_000_000, method="dense"):
    """y with M^T y = e_init: the sensitivity of x_init to the right-hand side."""
    e = np.zeros(m.shape[0])
    e[init_row] = 1.0
    mt = sp.csr_matrix(m).T.tocsr()
    if method == "dense":
        return dense_solve(mt, e)
    y, _, _, _ = jacobi(mt, e, eps, max_iter)
    return y


def grad_p(n, rowptr, col, val, goal, init, mode=PROB01, method="dense"):
    """d x_init / d P(s, s') for every stored entry, in input order.

    With F_s(x, P) = x_s - sum_s' P(s, s') xfull_s' = 0 on S?, the entry (s, s') of an S?
    row moves x_init by y_s * xfull_s' where M^T y = e_init; rows outside S? do not enter
    the system and get 0.
    """
    x, cls, _ = reach_probabilities(n, rowptr, col, val, goal, mode, method="dense")
    q, a, b = extract_system(n, rowptr, col, val, cls)
    g = np.zeros(int(np.asarray(rowptr)[-1]))
    if cls[init] != SQ:
        return g, x, cls
    pos = np.full(n, -1, np.int64)
    pos[q] = np.arange(q.size)
    y = adjoint(system_matrix(a), pos[init], method=method)
    row = np.repeat(np.arange(n), np.diff(np.asarray(rowptr)))
    inq = cls[row] == SQ
    g[inq] = y[pos[row[inq]]] * x[np.asarray(col)[inq]]
    return g, x, cls


def softmax_probs(rowptr, cls_e, offset, theta):
    """P_e = exp(l_e) / sum_{f in out(s)} exp(l_f), l_e = theta[class_e] + offset_e."""
    rowptr = np.asarray(rowptr)
    logit = np.asarray(theta, np.float64)[np.asarray(cls_e)] + np.asarray(offset, np.float64)
    deg = np.diff(rowptr)
    mx = np.repeat(np.maximum.reduceat(logit, rowptr[:-1]), deg)
    e = np.exp(logit - mx)
    return e / np.repeat(np.add.reduceat(e, rowptr[:-1]), deg)


def grad_theta(rowptr, p, g_p, cls_e, n_classes):
    """Chain rule through the row softmax: dl_f = P_f (g_f - sum_e P_e g_e), summed per class."""
    rowptr = np.asarray(rowptr)
    deg = np.diff(rowptr)
    inner = np.repeat(np.add.reduceat(p * g_p, rowptr[:-1]), deg)
    g_l = p * (g_p - inner)
    return np.bincount(np.asarray(cls_e), weights=g_l, minlength=n_classes)
