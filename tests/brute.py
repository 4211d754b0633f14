"""Independent references that pin the oracle: brute force on tiny inputs.

None of these shares code with the oracle: they work on dense matrices with plain Python
loops and follow the definitions of §2 (paths, cylinder sets, reachability) directly.
"""
import numpy as np


def closure(adj):
    """Boolean reflexive-transitive closure (Floyd-Warshall / Warshall's algorithm)."""
    n = adj.shape[0]
    r = adj.astype(bool) | np.eye(n, dtype=bool)
    for k in range(n):
        r = r | (r[:, k:k + 1] & r[k:k + 1, :])
    return r


def sets_by_closure(p_dense, goal):
    """S=0 and S=1 of §2.2 from the closure of the underlying digraph.

    S=0: no path to GS.  S=1: no path to S=0 that avoids GS (goal states keep no
    outgoing edges in that second graph, so a path through a goal stops there).
    """
    adj = p_dense > 0
    g = np.asarray(goal, bool)
    reach = closure(adj)
    s0 = ~reach[:, g].any(axis=1)
    adj2 = adj.copy()
    adj2[g, :] = False
    reach2 = closure(adj2)
    hits_s0 = reach2[:, s0].any(axis=1) & ~g
    s1 = ~hits_s0
    return s0, s1


def path_sum(p_dense, goal, s, depth=64):
    """Pr(s |= <> GS) as the sum over finite paths s ... g that first meet GS at g (§2).

    Pr(Cyl(s1..sk)) = prod P(s_i, s_i+1) (§2).  Depth-first enumeration; only for chains
    whose non-absorbing part is acyclic, so every path is finite.
    """
    g = np.asarray(goal, bool)
    total = 0.0
    stack = [(s, 1.0, 0)]
    while stack:
        u, pr, d = stack.pop()
        if g[u]:
            total += pr
            continue
        if d >= depth:
            continue
        for v in np.flatnonzero(p_dense[u] > 0):
            if v == u and p_dense[u, u] == 1.0:
                continue          # absorbing, not a goal: contributes nothing
            stack.append((int(v), pr * p_dense[u, v], d + 1))
    return total


def gambler_closed_form(N, p, i):
    """Ruin probabilities: Pr(reach N from i) = (1 - (q/p)^i) / (1 - (q/p)^N), i/N at p = 1/2."""
    q = 1.0 - p
    if abs(p - 0.5) < 1e-15:
        return i / N
    r = q / p
    return (1.0 - r ** i) / (1.0 - r ** N)


def random_dag_chain(rng, n, max_out=3, goal_frac=0.25, sink_frac=0.2):
    """Tiny chain whose transient part is acyclic: edges only go to higher-numbered states;
    goals and sinks are absorbing (self-loop 1)."""
    p = np.zeros((n, n))
    goal = np.zeros(n, np.uint8)
    order = rng.permutation(np.arange(1, n))
    ng = max(1, int(goal_frac * n))
    ns = int(sink_frac * n)
    goal[order[:ng]] = 1
    sink = np.zeros(n, bool)
    sink[order[ng:ng + ns]] = True
    sink[n - 1] = not goal[n - 1]
    for i in range(n):
        if goal[i] or sink[i] or i == n - 1:
            p[i, i] = 1.0
            continue
        k = rng.integers(1, min(max_out, n - 1 - i) + 1)
        succ = rng.choice(np.arange(i + 1, n), size=k, replace=False)
        w = rng.random(k) + 0.05
        p[i, succ] = w / w.sum()
    return p, goal


def dense_to_csr(p):
    rows, cols = np.nonzero(p)
    rowptr = np.zeros(p.shape[0] + 1, np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, cols.astype(np.int32), p[rows, cols].astype(np.float64)


def scc_by_closure(adj):
    """Label of every vertex's strongly connected component: the largest vertex that
    both reaches it and is reached from it (mutual reachability, by the closure)."""
    r = closure(adj)
    mutual = r & r.T
    n = adj.shape[0]
    return np.array([max(j for j in range(n) if mutual[i, j]) for i in range(n)], np.int64)


def condensation_height(adj, labels):
    """Longest path, counted in edges between components, from each vertex's component
    to a component with no edge out, by memoised depth-first recursion."""
    n = adj.shape[0]
    succ = {}
    for i in range(n):
        for j in range(n):
            if adj[i, j] and labels[i] != labels[j]:
                succ.setdefault(int(labels[i]), set()).add(int(labels[j]))
    memo = {}

    def height(c):
        if c not in memo:
            memo[c] = 1 + max((height(s) for s in succ.get(c, ())), default=-1)
        return memo[c]
    return np.array([height(int(labels[i])) for i in range(n)], np.int64)
