"""Seeded synthetic Markov chains shaped like the paper's workloads.

The paper measures on random matrices of several sizes and densities (§6) and on
sparse state spaces written out by a model checker (§7, Table 1).  Neither its data
nor its generator ships, so these functions stand in for them.  Each returns a
row-stochastic transition matrix P in compressed row storage (§4):

    rowptr  int64[n+1]   rowptr[i] = number of stored entries in rows 0..i-1
    col     int32[m]     column (successor state) of each entry, ascending in a row
    val     float64[m]   P(s, s') > 0
    goal    uint8[n]     1 for the goal states GS

This module only draws random numbers and arranges them.  It holds none of the
method's arithmetic (no partition, no linear system, no iteration), so the CPU
oracle and the CUDA library can both consume its output without sharing code.
Every generator is deterministic in its ``seed`` (numpy PCG64).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Chain", "ParamChain", "Batch",
    "random_chain", "dense_random_chain", "layered_chain", "parametric_chain",
    "batched_chains", "gamblers_ruin", "table1_chain", "worked_chain",
    "TABLE1_QUICKSORT", "TABLE1_BIASED_DIE",
]


@dataclass
class Chain:
    """A discrete-time Markov chain (S, P, s0) with a goal set (§2, §2.1)."""

    n: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    goal: np.ndarray
    init: int = 0
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.rowptr[-1])


@dataclass
class ParamChain:
    """A chain whose out-edge probabilities are a softmax of theta[class] + offset."""

    n: int
    rowptr: np.ndarray
    col: np.ndarray
    cls: np.ndarray        # int32[m], edge class in [0, n_classes)
    offset: np.ndarray     # float64[m]
    theta: np.ndarray      # float64[n_classes]
    goal: np.ndarray
    init: int = 0
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.rowptr[-1])


@dataclass
class Batch:
    """Independent chains, each with K goal sets (uint8[K, n_c] per chain)."""

    chains: list = field(default_factory=list)
    goals: list = field(default_factory=list)
    name: str = ""

    @property
    def k(self) -> int:
        return int(self.goals[0].shape[0]) if self.goals else 0

    def concat(self):
        """Block-diagonal union of all chains: (n, rowptr, col, val, goal uint8[K, n], offsets)."""
        offs = np.zeros(len(self.chains) + 1, np.int64)
        for i, c in enumerate(self.chains):
            offs[i + 1] = offs[i] + c.n
        n = int(offs[-1])
        m = sum(c.m for c in self.chains)
        rowptr = np.zeros(n + 1, np.int64)
        col = np.empty(m, np.int32)
        val = np.empty(m, np.float64)
        goal = np.zeros((self.k, n), np.uint8)
        e = 0
        for i, c in enumerate(self.chains):
            a, b = int(offs[i]), int(offs[i + 1])
            rowptr[a + 1:b + 1] = c.rowptr[1:] + e
            col[e:e + c.m] = c.col + a
            val[e:e + c.m] = c.val
            goal[:, a:b] = self.goals[i]
            e += c.m
        return n, rowptr, col, val, goal, offs


def _rowptr(deg: np.ndarray) -> np.ndarray:
    rowptr = np.zeros(deg.size + 1, np.int64)
    np.cumsum(deg, out=rowptr[1:])
    return rowptr


def _distinct_columns(rng, deg: np.ndarray, draw):
    """Per row i, deg[i] distinct columns; ``draw(rows, slots)`` proposes candidates.

    Candidates that repeat an earlier column of the same row are redrawn until every
    row is duplicate-free.  Rows come back sorted ascending.
    """
    rows = deg.size
    dmax = int(deg.max()) if rows else 0
    slot = np.arange(dmax, dtype=np.int64)
    unused = slot[None, :] >= deg[:, None]
    big = np.int64(1) << np.int64(40)
    cols = draw(np.repeat(np.arange(rows, dtype=np.int64), dmax).reshape(rows, dmax), slot)
    cols[unused] = big + np.broadcast_to(slot, cols.shape)[unused]
    while True:
        order = np.argsort(cols, axis=1, kind="stable")
        cols = np.take_along_axis(cols, order, axis=1)
        dup = np.zeros(cols.shape, bool)
        dup[:, 1:] = cols[:, 1:] == cols[:, :-1]
        if not dup.any():
            break
        r, s = np.nonzero(dup)
        cols[r, s] = draw(r, s)
    valid = cols < big
    return cols[valid].astype(np.int32)


def _finish(n, rowptr, col, w, rng, goal_idx, sink_idx, name, init=0):
    """Normalise weights per row, turn sinks into self-loops, build the Chain."""
    deg = np.diff(rowptr)
    sink = np.zeros(n, bool)
    sink[sink_idx] = True
    if sink.any():
        keep = ~np.repeat(sink, deg)
        deg = np.where(sink, 1, deg)
        new_col = np.empty(int(deg.sum()), np.int32)
        new_w = np.empty(new_col.size, np.float64)
        new_rowptr = _rowptr(deg)
        row_of = np.repeat(np.arange(n), deg)
        is_sink_slot = sink[row_of]
        new_col[~is_sink_slot] = col[keep]
        new_w[~is_sink_slot] = w[keep]
        new_col[is_sink_slot] = np.flatnonzero(sink).astype(np.int32)
        new_w[is_sink_slot] = 1.0
        rowptr, col, w = new_rowptr, new_col, new_w
    rowsum = np.add.reduceat(w, rowptr[:-1]) if n else np.zeros(0)
    val = w / np.repeat(rowsum, np.diff(rowptr))
    goal = np.zeros(n, np.uint8)
    goal[goal_idx] = 1
    return Chain(n=n, rowptr=rowptr, col=col, val=val, goal=goal, init=init, name=name)


def _goals_and_sinks(rng, n, n_goal, n_sink, candidates=None):
    """Disjoint goal / sink index sets, never containing the initial state 0."""
    pool = np.arange(1, n) if candidates is None else candidates[candidates != 0]
    pick = rng.permutation(pool)
    return np.sort(pick[:n_goal]), np.sort(pick[n_goal:n_goal + n_sink])


def random_chain(n=4096, deg=16, goal_frac=0.02, sink_frac=0.02, seed=1210_6412_1):
    """Each row: ``deg`` distinct successors drawn uniformly, weights U(0,1] normalised.

    ``goal_frac`` of the states are goals and ``sink_frac`` are absorbing (self-loop 1.0);
    the initial state is 0 and is neither.  Default: 4096 states, 16 successors, 2% / 2%.
    """
    rng = np.random.default_rng(seed)
    d = np.full(n, min(deg, n), np.int64)
    col = _distinct_columns(rng, d, lambda r, s: rng.integers(0, n, size=np.shape(r), dtype=np.int64))
    w = 1.0 - rng.random(col.size)
    g, s = _goals_and_sinks(rng, n, max(1, int(round(goal_frac * n))), int(round(sink_frac * n)))
    return _finish(n, _rowptr(d), col, w, rng, g, s, f"random n={n} deg={deg}")


def dense_random_chain(n=32768, density=0.10, goal_frac=0.01, sink_frac=0.0, seed=1210_6412_2,
                       chunk_rows=1024):
    """Random pattern with each entry present independently with probability ``density``.

    Positions come from geometric gaps (a Bernoulli process along the row), so an n=32768
    matrix at 10% density (about 107M entries) is drawn without an n x n temporary.
    Weights are U(0,1] normalised per row; ``sink_frac`` of the states become absorbing.
    """
    rng = np.random.default_rng(seed)
    mean = n * density
    kmax = int(np.ceil(mean + 10.0 * np.sqrt(mean * (1 - density) + 1.0) + 16))
    cols, degs = [], []
    for r0 in range(0, n, chunk_rows):
        rows = min(chunk_rows, n - r0)
        pos = np.cumsum(rng.geometric(density, size=(rows, kmax)), axis=1) - 1
        short = np.flatnonzero(pos[:, -1] < n)
        while short.size:       # a row ran out of draws before reaching column n: redraw it
            pos[short] = np.cumsum(rng.geometric(density, size=(short.size, kmax)), axis=1) - 1
            short = short[pos[short, -1] < n]
        mask = pos < n
        d = mask.sum(axis=1)
        empty = np.flatnonzero(d == 0)
        if empty.size:          # keep every row stochastic: an empty row gets a self-loop
            pos[empty, 0] = r0 + empty
            mask[empty, 0] = True
            d[empty] = 1
        cols.append(pos[mask].astype(np.int32))
        degs.append(d)
    col = np.concatenate(cols)
    d = np.concatenate(degs).astype(np.int64)
    w = 1.0 - rng.random(col.size)
    g, s = _goals_and_sinks(rng, n, max(1, int(round(goal_frac * n))), int(round(sink_frac * n)))
    return _finish(n, _rowptr(d), col, w, rng, g, s, f"dense n={n} density={density}")


def layered_chain(layers=2000, width=4000, dmin=1, dmax=4, p_forward=0.9, goal_frac_last=0.01,
                  sink_frac=0.05, seed=1210_6412_3):
    """Model-checker-like layered state space.

    States are numbered layer by layer.  Out-degree is uniform in dmin..dmax; each
    successor is, with probability ``p_forward``, a uniform state of the next layer (the
    last layer: its own layer), else a uniform state of a uniform earlier layer (layer 0:
    its own layer).  Successors of a state are distinct.  Probabilities are dyadic:
    1/2, 1/4, ..., 1/2^(d-1), 1/2^(d-1) (a single successor gets 1), randomly permuted
    over the successors.  ``goal_frac_last`` of the last layer are goals; ``sink_frac`` of
    all states are absorbing.
    """
    rng = np.random.default_rng(seed)
    n = layers * width
    d = rng.integers(dmin, dmax + 1, size=n).astype(np.int64)

    def draw(r, s):
        r = np.asarray(r, np.int64)
        lay = r // width
        fwd = rng.random(r.shape) < p_forward
        nxt = np.minimum(lay + 1, layers - 1)
        back = np.where(lay > 0, (rng.random(r.shape) * np.maximum(lay, 1)).astype(np.int64), 0)
        tl = np.where(fwd, nxt, back)
        return tl * width + rng.integers(0, width, size=r.shape, dtype=np.int64)

    col = _distinct_columns(rng, d, draw)
    # dyadic weights: rank k (0-based) of a random order over the d successors gets 2^-(k+1),
    # the last rank gets 2^-(d-1)
    rowptr = _rowptr(d)
    row_of = np.repeat(np.arange(n, dtype=np.int64), d)
    key = rng.random(col.size) + row_of.astype(np.float64) * 2.0
    order = np.argsort(key, kind="stable")
    rank = np.empty(col.size, np.int64)
    rank[order] = np.arange(col.size, dtype=np.int64) - rowptr[row_of[order]]
    dd = d[row_of]
    w = np.ldexp(1.0, -(np.minimum(rank, dd - 2) + 1).astype(np.int32))
    w[dd == 1] = 1.0
    last = np.arange((layers - 1) * width, n)
    n_goal = max(1, int(round(goal_frac_last * width)))
    goal_idx = np.sort(rng.choice(last, size=n_goal, replace=False))
    pool = np.setdiff1d(np.arange(1, n), goal_idx)
    sink_idx = np.sort(rng.choice(pool, size=int(round(sink_frac * n)), replace=False))
    return _finish(n, rowptr, col, w, rng, goal_idx, sink_idx,
                   f"layered {layers}x{width} deg {dmin}..{dmax}")


def parametric_chain(n=4_000_000, dmin=2, dmax=8, n_classes=64, theta_sd=0.5, goal_frac=0.01,
                     sink_frac=0.02, seed=1210_6412_5):
    """Chain whose out-edge probabilities are softmax(theta[class(e)] + offset_e) per row.

    Out-degree uniform in dmin..dmax with distinct uniform successors, classes uniform in
    [0, n_classes), theta ~ N(0, theta_sd^2), offset ~ N(0, 1).  Absorbing states keep a
    single self-loop edge (softmax of one edge is 1).  Only parameters are returned; the
    probabilities themselves are the method's to compute.
    """
    rng = np.random.default_rng(seed)
    d = rng.integers(dmin, dmax + 1, size=n).astype(np.int64)
    g, s = _goals_and_sinks(rng, n, max(1, int(round(goal_frac * n))), int(round(sink_frac * n)))
    d[s] = 1
    col = _distinct_columns(rng, d, lambda r, sl: rng.integers(0, n, size=np.shape(r), dtype=np.int64))
    rowptr = _rowptr(d)
    col[rowptr[s]] = s.astype(np.int32)
    cls = rng.integers(0, n_classes, size=col.size).astype(np.int32)
    offset = rng.standard_normal(col.size)
    theta = theta_sd * rng.standard_normal(n_classes)
    goal = np.zeros(n, np.uint8)
    goal[g] = 1
    return ParamChain(n=n, rowptr=rowptr, col=col, cls=cls, offset=offset, theta=theta, goal=goal,
                      name=f"parametric n={n} deg {dmin}..{dmax} classes={n_classes}")


def batched_chains(n_chains=256, n_min=1_000, n_max=2_000_000, dmin=2, dmax=32, k=8,
                   goal_lo=0.005, goal_hi=0.05, sink_frac=0.0, seed=1210_6412_4):
    """Independent random chains with sizes log-uniform in [n_min, n_max].

    Out-degree uniform in dmin..dmax (distinct uniform successors, weights U(0,1]
    normalised).  Each chain gets ``k`` goal sets, each a uniform random fraction
    U(goal_lo, goal_hi) of its states (state 0 excluded).  ``sink_frac`` of the states of
    each chain are absorbing.  Every chain has its own seed, so chain c alone can be
    regenerated by ``batched_chains(...)`` with the same arguments.
    """
    root = np.random.SeedSequence(seed)
    rng0 = np.random.default_rng(root.spawn(1)[0])
    sizes = np.exp(rng0.uniform(np.log(n_min), np.log(n_max), size=n_chains)).astype(np.int64)
    out = Batch(name=f"batched {n_chains} chains n in [{n_min},{n_max}] deg {dmin}..{dmax} k={k}")
    for c, ss in enumerate(root.spawn(n_chains + 1)[1:]):
        rng = np.random.default_rng(ss)
        n = int(sizes[c])
        d = rng.integers(dmin, min(dmax, n) + 1, size=n).astype(np.int64)
        col = _distinct_columns(rng, d, lambda r, s: rng.integers(0, n, size=np.shape(r), dtype=np.int64))
        w = 1.0 - rng.random(col.size)
        _, sinks = _goals_and_sinks(rng, n, 0, int(round(sink_frac * n)))
        ch = _finish(n, _rowptr(d), col, w, rng, np.zeros(0, np.int64), sinks, f"chain {c}")
        goals = np.zeros((k, n), np.uint8)
        for j in range(k):
            frac = rng.uniform(goal_lo, goal_hi)
            gi = rng.choice(np.arange(1, n), size=max(1, int(round(frac * n))), replace=False)
            goals[j, gi] = 1
        out.chains.append(ch)
        out.goals.append(goals)
    return out


@dataclass
class System:
    """A general sparse system M x = b in CSR (diagonal included)."""

    n: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    b: np.ndarray
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.rowptr[-1])


def diag_dominant_system(n=4096, density=0.01, max_int=10, margin=(1, 10), seed=1210_6412_7):
    """The random systems of §6: random positive integers at random positions, made
    diagonally dominant with a non-zero diagonal, and a random integer right-hand side.

    Off-diagonal entries: each present with probability ``density``, value U{1..max_int}.
    Diagonal: the row's off-diagonal sum plus U{margin}, so every row is strictly
    dominant.  b: U{1..max_int}.  The integer ranges are not stated in the paper.
    """
    rng = np.random.default_rng(seed)
    cols, degs = [], []
    mean = max(density * n, 1e-9)
    kmax = int(np.ceil(mean + 10.0 * np.sqrt(mean) + 16))
    for r0 in range(0, n, 1024):
        rows = min(1024, n - r0)
        pos = np.cumsum(rng.geometric(density, size=(rows, kmax)), axis=1) - 1
        short = np.flatnonzero(pos[:, -1] < n)
        while short.size:
            pos[short] = np.cumsum(rng.geometric(density, size=(short.size, kmax)), axis=1) - 1
            short = short[pos[short, -1] < n]
        diag = (r0 + np.arange(rows))[:, None]
        keep = (pos < n) & (pos != diag)
        pos = np.where(keep, pos, n + 1)
        pos = np.concatenate([pos, diag], axis=1)
        pos.sort(axis=1)
        keep = pos < n
        cols.append(pos[keep].astype(np.int32))
        degs.append(keep.sum(axis=1))
    col = np.concatenate(cols)
    deg = np.concatenate(degs).astype(np.int64)
    rowptr = _rowptr(deg)
    row_of = np.repeat(np.arange(n), deg)
    val = rng.integers(1, max_int + 1, size=col.size).astype(np.float64)
    is_diag = col == row_of
    off = np.where(is_diag, 0.0, val)
    offsum = np.add.reduceat(off, rowptr[:-1]) if n else np.zeros(0)
    val[is_diag] = offsum + rng.integers(margin[0], margin[1] + 1, size=n)
    b = rng.integers(1, max_int + 1, size=n).astype(np.float64)
    return System(n=n, rowptr=rowptr, col=col, val=val, b=b,
                  name=f"diagonally dominant n={n} density={density}")


def skewed_chain(n=20000, zipf_a=1.6, max_deg=64, hubs=8, hub_deg=6000, goal_frac=0.02,
                 sink_frac=0.02, seed=1210_6412_8):
    """Chain with skewed out-degrees: Zipf(zipf_a) degrees capped at max_deg, plus `hubs`
    states with `hub_deg` distinct successors (the load-balancing case of row-wise
    kernels).  Successors uniform and distinct, weights U(0,1] normalised."""
    rng = np.random.default_rng(seed)
    d = np.minimum(rng.zipf(zipf_a, size=n), max_deg).astype(np.int64)
    hub_idx = np.sort(rng.choice(np.arange(1, n), size=min(hubs, n - 1), replace=False))
    d[hub_idx] = 1                      # placeholder row, replaced below
    col = _distinct_columns(rng, d, lambda r, s: rng.integers(0, n, size=np.shape(r), dtype=np.int64))
    # hub rows: hub_deg distinct successors each, drawn without replacement
    rowptr = _rowptr(d)
    pieces, start = [], 0
    for h in hub_idx:
        pieces.append(col[start:rowptr[h]])
        pieces.append(np.sort(rng.choice(n, size=min(hub_deg, n), replace=False)).astype(np.int32))
        start = rowptr[h + 1]
    pieces.append(col[start:])
    col = np.concatenate(pieces)
    d[hub_idx] = min(hub_deg, n)
    w = 1.0 - rng.random(col.size)
    cand = np.setdiff1d(np.arange(1, n), hub_idx)
    g, s = _goals_and_sinks(rng, n, max(1, int(round(goal_frac * n))), int(round(sink_frac * n)), cand)
    return _finish(n, _rowptr(d), col, w, rng, g, s, f"skewed n={n} zipf={zipf_a} hubs={hubs}x{hub_deg}")


def cascade_chain(blocks=64, width=4096, dmin=2, dmax=6, p_stay=0.9, goal_frac_last=0.02,
                  sink_frac=0.01, seed=1210_6412_8):
    """A chain of strongly connected stages: the shape the SCC order of §8 is meant for.

    States are numbered block by block.  Out-degree is uniform in dmin..dmax; each
    successor is, with probability ``p_stay``, a uniform state of the same block, else a
    uniform state of the next block (the last block keeps all its edges).  Weights are
    U(0,1] normalised.  ``goal_frac_last`` of the last block are goals; ``sink_frac`` of
    all states are absorbing.  Each block is mostly one large component, and the blocks
    form a path in the condensation.
    """
    rng = np.random.default_rng(seed)
    n = blocks * width
    d = rng.integers(dmin, dmax + 1, size=n).astype(np.int64)
    d = np.minimum(d, width)

    def draw(r, s):
        r = np.asarray(r, np.int64)
        blk = r // width
        stay = (rng.random(r.shape) < p_stay) | (blk == blocks - 1)
        tb = np.where(stay, blk, blk + 1)
        return tb * width + rng.integers(0, width, size=r.shape, dtype=np.int64)

    col = _distinct_columns(rng, d, draw)
    w = 1.0 - rng.random(col.size)
    last = np.arange((blocks - 1) * width, n)
    n_goal = max(1, int(round(goal_frac_last * width)))
    goal_idx = np.sort(rng.choice(last, size=n_goal, replace=False))
    pool = np.setdiff1d(np.arange(1, n), goal_idx)
    sink_idx = np.sort(rng.choice(pool, size=int(round(sink_frac * n)), replace=False))
    return _finish(n, _rowptr(d), col, w, rng, goal_idx, sink_idx,
                   f"cascade {blocks}x{width} p_stay={p_stay}")


def gamblers_ruin(N=20, p=0.4):
    """Random walk on 0..N, up with probability p, down with 1-p; 0 and N absorbing; GS={N}."""
    n = N + 1
    rows, cols, vals = [], [], []
    for i in range(n):
        if i == 0 or i == N:
            rows.append(i); cols.append(i); vals.append(1.0)
        else:
            rows += [i, i]; cols += [i - 1, i + 1]; vals += [1.0 - p, p]
    deg = np.bincount(np.asarray(rows), minlength=n)
    goal = np.zeros(n, np.uint8)
    goal[N] = 1
    return Chain(n=n, rowptr=_rowptr(deg.astype(np.int64)), col=np.asarray(cols, np.int32),
                 val=np.asarray(vals, np.float64), goal=goal, init=1, name=f"gambler N={N} p={p}")


def worked_chain():
    """The four-state chain drawn in §2, with state 3 the only goal (§2.2, §2.3)."""
    rowptr = np.array([0, 2, 3, 5, 6], np.int64)
    col = np.array([2, 3, 1, 0, 1, 3], np.int32)
    val = np.array([0.5, 0.5, 1.0, 0.4, 0.6, 1.0])
    goal = np.array([0, 0, 0, 1], np.uint8)
    return Chain(n=4, rowptr=rowptr, col=col, val=val, goal=goal, init=0, name="worked 4-state")


# (n, m) of the S? matrices in Table 1 (random quick sort / biased die).
TABLE1_QUICKSORT = [(92, 211), (118, 263), (142, 312), (173, 379), (198, 430), (228, 491),
                    (250, 536), (284, 606), (313, 669)]
TABLE1_BIASED_DIE = [(667, 1333), (1333, 2665), (2000, 3999), (2668, 5335), (3647, 7293),
                     (4647, 9293), (5647, 11293), (6647, 13293), (7647, 15293)]


def table1_chain(n, m, goal_frac=0.02, sink_frac=0.02, seed=1210_6412_6):
    """Random chain with n states and m stored transitions (the sizes of Table 1).

    Out-degrees are 1 plus a multinomial share of the m - n extra entries; successors
    are distinct and uniform, weights U(0,1] normalised.
    """
    rng = np.random.default_rng(seed + n)
    d = 1 + rng.multinomial(m - n, np.full(n, 1.0 / n)).astype(np.int64)
    d = np.minimum(d, n)
    col = _distinct_columns(rng, d, lambda r, s: rng.integers(0, n, size=np.shape(r), dtype=np.int64))
    w = 1.0 - rng.random(col.size)
    g, s = _goals_and_sinks(rng, n, max(1, int(round(goal_frac * n))), max(1, int(round(sink_frac * n))))
    return _finish(n, _rowptr(d), col, w, rng, g, s, f"table1 n={n} m={m}")
