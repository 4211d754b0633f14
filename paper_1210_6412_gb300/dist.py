"""Jacobi and BiCGStab on (I - A) x = b split by rows over several processes (one GPU each).

The related work of §8 runs Jacobi on two GPUs and its future work is a multi-GPU BiCGStab.
Here the rows of the system over S? (§2.3) are cut into contiguous blocks of about equal
work (stored entries plus a per-row share), one per rank.  Each rank keeps its block on its
own GPU as a ``reach_block`` of the CUDA library, with its columns renumbered: own rows
first, then the halo (the other ranks' columns the block references).

One iteration then needs, besides the block's kernels:
  * Jacobi (§3.1): an all-gather of the new iterate's own entries after every sweep, from
    which each rank fills its halo; every ``check_every`` sweeps a max all-reduce of the
    local max|x' - x| for the stopping rule.
  * BiCGStab (§3.2): all-gathers of p and s (the two products), sum all-reduces of q.r,
    q.v and (t.s, t.t), and max all-reduces of max|s| and max|r| for the stopping rule.

The solver loops are generators that yield their collectives (``Allgather``,
``Allreduce``) and receive the results, so one loop serves every communicator:
``TorchComm`` (torch.distributed: NCCL between GPUs, gloo between CPU processes) and
``LockstepComm`` (all ranks in one process, advanced in turn; the host performs each
collective between them, so no kernel ever waits for another).  The arithmetic is the
``local`` object's: ``CudaBlockOps`` runs it in the library's block kernels.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import (REACH_BLOCK_P, REACH_BLOCK_S, REACH_BLOCK_XP, REACH_BLOCK_XR, REACH_DEVICE, REACH_HOST,
               ReachError, lib)


# ------------------------------------------------------------------ partition and halo plan

def partition_rows(rowptr, parts):
    """Row boundaries [0 = b_0 < b_1 < ... < b_parts = n] that split the rows into contiguous
    blocks of about equal work: stored entries plus two units per row (the row's own reads
    and writes).  Every block gets at least one row (n >= parts is required)."""
    rowptr = np.asarray(rowptr, np.int64)
    n = rowptr.size - 1
    if parts < 1 or n < parts:
        raise ValueError("need 1 <= parts <= number of rows")
    cost = rowptr + 2 * np.arange(n + 1, dtype=np.int64)
    targets = cost[-1] * np.arange(1, parts, dtype=np.float64) / parts
    cuts = np.searchsorted(cost, targets, side="left").astype(np.int64)
    bounds = np.concatenate([[0], cuts, [n]]).astype(np.int64)
    for i in range(1, parts):            # strictly increasing, room for the blocks after it
        bounds[i] = min(max(bounds[i], bounds[i - 1] + 1), n - (parts - i))
    return bounds


@dataclass
class BlockPlan:
    """Rank `rank`'s rows [r0, r1) of the system with renumbered columns.

    rowptr/col/val: the block's CSR, col in [0, n_rows + n_halo) (own rows first); d, b:
    the block's diagonal and right-hand side; halo_ids: the global columns of the halo
    (ascending); halo_src: where each halo entry sits in the all-gathered vector, whose
    rank-r part holds rank r's own entries padded to max_rows."""
    rank: int
    bounds: np.ndarray
    r0: int
    r1: int
    max_rows: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    d: np.ndarray
    b: np.ndarray
    halo_ids: np.ndarray
    halo_src: np.ndarray

    @property
    def n_rows(self):
        return self.r1 - self.r0

    @property
    def n_halo(self):
        return int(self.halo_ids.size)

    @property
    def ext_len(self):
        """Length of an extended vector: own + halo entries, and at least max_rows (the
        all-gather sends its first max_rows entries)."""
        return max(self.n_rows + self.n_halo, self.max_rows)


def block_plan(rowptr, col, val, d, b, bounds, rank):
    """The BlockPlan of `rank` for the system (rowptr, col, val) over n rows with diagonal d
    and right-hand side b, cut at `bounds` (partition_rows)."""
    rowptr = np.asarray(rowptr, np.int64)
    col = np.asarray(col)
    bounds = np.asarray(bounds, np.int64)
    r0, r1 = int(bounds[rank]), int(bounds[rank + 1])
    lo, hi = int(rowptr[r0]), int(rowptr[r1])
    c = col[lo:hi].astype(np.int64)
    own = (c >= r0) & (c < r1)
    halo_ids = np.unique(c[~own])
    n_rows = r1 - r0
    local = np.empty(c.size, np.int64)
    local[own] = c[own] - r0
    local[~own] = n_rows + np.searchsorted(halo_ids, c[~own])
    max_rows = int(np.max(np.diff(bounds)))
    owner = np.searchsorted(bounds, halo_ids, side="right") - 1
    halo_src = owner * max_rows + (halo_ids - bounds[owner])
    return BlockPlan(rank=rank, bounds=bounds, r0=r0, r1=r1, max_rows=max_rows,
                     rowptr=rowptr[r0:r1 + 1] - lo, col=local.astype(np.int32),
                     val=np.asarray(val, np.float64)[lo:hi], d=np.asarray(d, np.float64)[r0:r1],
                     b=np.asarray(b, np.float64)[r0:r1], halo_ids=halo_ids, halo_src=halo_src.astype(np.int64))


# ------------------------------------------------------------------ collectives

@dataclass
class Allgather:
    """Every rank sends `send` (max_rows entries); the result is all ranks' sends in rank
    order, world * max_rows entries (a vector of the local ops' kind)."""
    send: object


@dataclass
class Allreduce:
    """Element-wise sum or max of a short list of floats over the ranks."""
    values: list
    op: str


class TorchComm:
    """Collectives over a torch.distributed process group (NCCL for CUDA tensors, gloo for
    CPU ones).  Scalars travel in a small tensor on `device`."""

    def __init__(self, device="cpu", group=None):
        import torch
        import torch.distributed as dist
        self.torch, self.dist, self.group = torch, dist, group
        self.device = torch.device(device)
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)

    def _perform(self, req):
        torch, dist = self.torch, self.dist
        if isinstance(req, Allgather):
            send = req.send if torch.is_tensor(req.send) else torch.from_numpy(np.ascontiguousarray(req.send))
            parts = [torch.empty_like(send) for _ in range(self.world)]
            dist.all_gather(parts, send.contiguous(), group=self.group)
            out = torch.cat(parts)
            return out if torch.is_tensor(req.send) else out.numpy()
        t = torch.tensor(req.values, dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM if req.op == "sum" else dist.ReduceOp.MAX, group=self.group)
        return t.cpu().tolist()

    def run(self, gen):
        res = None
        while True:
            try:
                req = gen.send(res)
            except StopIteration as stop:
                return stop.value
            res = self._perform(req)


class LockstepComm:
    """All ranks in one process: each rank's loop runs up to its next collective, then the
    host performs the collective over every rank's request and hands back the results.
    Kernels of different ranks never wait for each other; the host orders everything."""

    @staticmethod
    def run_all(gens, cat):
        """gens: one solver generator per rank; cat(list of vectors) concatenates vectors of
        the local ops' kind.  Returns the ranks' return values."""
        results = [None] * len(gens)
        done = [False] * len(gens)
        out = [None] * len(gens)
        while not all(done):
            reqs = []
            for i, g in enumerate(gens):
                if done[i]:
                    reqs.append(None)
                    continue
                try:
                    reqs.append(g.send(results[i]))
                except StopIteration as stop:
                    done[i] = True
                    out[i] = stop.value
                    reqs.append(None)
            live = [r for r in reqs if r is not None]
            if not live:
                break
            if len(live) != len(gens):
                raise RuntimeError("ranks left the solve loop at different iterations")
            if all(isinstance(r, Allgather) for r in live):
                res = cat([r.send for r in live])
            elif all(isinstance(r, Allreduce) for r in live) and len({r.op for r in live}) == 1:
                vals = np.array([r.values for r in live], np.float64)
                res = (vals.sum(0) if live[0].op == "sum" else vals.max(0)).tolist()
            else:
                raise RuntimeError("ranks asked for different collectives")
            results = [res] * len(gens)
        return out


# ------------------------------------------------------------------ the solver loops

def jacobi(local, plan, eps, max_iter, check_every=16):
    """Jacobi (§3.1) on the row-split system: every sweep x'_own = (b + A x_ext) / d on each
    block, then an all-gather of the own entries and the halo refill; every `check_every`
    sweeps (and after the last) the ranks' max|x' - x| is max-reduced and the loop stops when
    it is below eps.  Yields collectives; returns (own x, sweeps, last max|x' - x|, converged)."""
    xa, xb = local.zeros(plan.ext_len), local.zeros(plan.ext_len)
    it, delta = 0, float("inf")
    while it < max_iter:
        w = min(check_every, max_iter - it)
        for _ in range(w):
            dloc = local.jacobi(xa, xb)
            gathered = yield Allgather(local.head(xb, plan.max_rows))
            local.halo(gathered, xb)
            xa, xb = xb, xa
        it += w
        delta = (yield Allreduce([dloc()], "max"))[0]
        if delta < eps:
            return local.head(xa, plan.n_rows), it, delta, True
    return local.head(xa, plan.n_rows), it, delta, False


def bicgstab(local, plan, eps, max_iter):
    """Unpreconditioned BiCGStab (§3.2) on the row-split system, from x = 0 with shadow
    q = r = b, stopping and restarting exactly as the single-GPU solver.  Yields
    collectives; returns (own x, iterations, last max|s| or max|r|, status) with status
    "ok", "max_iter" or "breakdown"."""
    n = plan.n_rows
    x, r, q, v, t = (local.zeros(n) for _ in range(5))
    p, s = local.zeros(plan.ext_len), local.zeros(plan.ext_len)
    local.set_b(r)
    local.copy(q, r)
    rmax = (yield Allreduce([local.maxabs(r)], "max"))[0]
    if rmax < eps:
        return x, 0, rmax, "ok"
    y = a = w = 1.0
    restarted = False
    for it in range(1, max_iter + 1):
        y_prev = y
        y = (yield Allreduce([local.dot(q, r)[0]], "sum"))[0]
        if y == 0.0:
            if restarted:
                return x, it, rmax, "breakdown"
            restarted = True
            local.copy(q, r)
            local.fill0(p)
            local.fill0(v)
            y_prev, a, w = 1.0, 1.0, 1.0
            y = (yield Allreduce([local.dot(q, r)[0]], "sum"))[0]
        local.bicg_p(r, p, v, (y * a) / (y_prev * w), w)
        gathered = yield Allgather(local.head(p, plan.max_rows))
        local.halo(gathered, p)
        qv = (yield Allreduce([local.matvec(p, v, q)], "sum"))[0]
        if qv == 0.0:
            if restarted:
                return x, it, rmax, "breakdown"
            restarted = True
            local.copy(q, r)
            local.copy(p, r)
            gathered = yield Allgather(local.head(p, plan.max_rows))
            local.halo(gathered, p)
            qv_loc = local.matvec(p, v, q)
            y, qv = (yield Allreduce([local.dot(q, r)[0], qv_loc], "sum"))
            if qv == 0.0:
                return x, it, rmax, "breakdown"
        a = y / qv
        smax = (yield Allreduce([local.bicg_s(r, v, a, s)], "max"))[0]
        if smax < eps:
            local.bicg_xp(x, p, a)
            return x, it, smax, "ok"
        gathered = yield Allgather(local.head(s, plan.max_rows))
        local.halo(gathered, s)
        local.matvec(s, t, None)
        ts, tt = (yield Allreduce(list(local.dot(t, s, t)), "sum"))
        w = ts / tt
        rmax = (yield Allreduce([local.bicg_xr(x, p, s, t, a, w, r)], "max"))[0]
        if rmax < eps:
            return x, it, rmax, "ok"
        if w == 0.0:
            if restarted:
                return x, it, rmax, "breakdown"
            restarted = True
            local.copy(q, r)
            local.fill0(p)
            local.fill0(v)
            y, a, w = 1.0, 1.0, 1.0
    return x, max_iter, rmax, "max_iter"


# ------------------------------------------------------------------ the block on a GPU

def gathered_len(plan: BlockPlan) -> int:
    """Length of an all-gathered vector: every rank's own entries padded to max_rows."""
    return (len(plan.bounds) - 1) * plan.max_rows


class CudaBlockOps:
    """The local arithmetic of the loops above in the library's row-block kernels
    (reach_block_*), on CUDA tensors of the current device and its current stream."""

    def __init__(self, plan: BlockPlan):
        import torch
        self.torch = torch
        self.plan = plan
        self.dev = torch.device("cuda", torch.cuda.current_device())
        # torch's vector work and the block's kernels share torch's current stream
        self.tstream = torch.cuda.current_stream()
        self.stream = self.tstream.cuda_stream
        self.scal = torch.zeros(4, dtype=torch.float64, device=self.dev)
        self._b = torch.from_numpy(np.ascontiguousarray(plan.b)).to(self.dev)
        blk = C.c_void_p()
        st = lib().reach_block_create(C.byref(blk), plan.n_rows, plan.n_halo, plan.rowptr.ctypes.data,
                                      plan.col.ctypes.data, plan.val.ctypes.data, plan.d.ctypes.data,
                                      plan.b.ctypes.data, plan.halo_src.ctypes.data, gathered_len(plan),
                                      REACH_HOST, self.stream)
        if st != 0:
            raise ReachError(st, lib().reach_block_last_error(None).decode() or "reach_block_create")
        self.blk = blk

    def close(self):
        if getattr(self, "blk", None):
            lib().reach_block_destroy(self.blk)
            self.blk = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ok(self, st, what):
        if st != 0:
            raise ReachError(st, lib().reach_block_last_error(self.blk).decode() or what)

    @staticmethod
    def _p(t):
        return t.data_ptr() if t is not None else None

    def _scalar(self, k):
        # the reductions run on the block's stream; reading them waits for it
        self.tstream.synchronize()
        return float(self.scal[k].item())

    # vectors
    def zeros(self, n):
        return self.torch.zeros(max(n, 1), dtype=self.torch.float64, device=self.dev)

    def head(self, v, n):
        return v[:n]

    def copy(self, dst, src):
        dst[:self.plan.n_rows].copy_(src[:self.plan.n_rows])

    def fill0(self, v):
        v.zero_()

    def set_b(self, r):
        r[:self.plan.n_rows].copy_(self._b)

    # block kernels
    def halo(self, gathered, x_ext):
        self._ok(lib().reach_block_halo(self.blk, gathered.data_ptr(), x_ext.data_ptr()), "reach_block_halo")

    def jacobi(self, x_ext, x_new):
        self._ok(lib().reach_block_jacobi(self.blk, x_ext.data_ptr(), x_new.data_ptr(), self.scal.data_ptr()),
                 "reach_block_jacobi")
        return lambda: self._scalar(0)

    def matvec(self, u_ext, y, w):
        self._ok(lib().reach_block_matvec(self.blk, u_ext.data_ptr(), y.data_ptr(), self._p(w),
                                          self.scal.data_ptr() if w is not None else None), "reach_block_matvec")
        return self._scalar(0) if w is not None else None

    def dot(self, u, v, w=None):
        self._ok(lib().reach_block_dot(self.blk, u.data_ptr(), v.data_ptr(), self._p(w), self.scal.data_ptr()),
                 "reach_block_dot")
        return (self._scalar(0), self._scalar(1) if w is not None else 0.0)

    def maxabs(self, v):
        # max|v| of an own vector through the S-stage kernel with alpha = 0 (s = v)
        zero, out = self.zeros(self.plan.n_rows), self.zeros(self.plan.n_rows)
        return self.bicg_s(v, zero, 0.0, out)

    def _upd(self, stage, alpha, beta, omega, x=None, r=None, p=None, v=None, s=None, t=None, out=True):
        self._ok(lib().reach_block_bicgstab_update(self.blk, stage, alpha, beta, omega, self._p(x), self._p(r),
                                                   self._p(p), self._p(v), self._p(s), self._p(t),
                                                   self.scal.data_ptr() if out else None),
                 "reach_block_bicgstab_update")

    def bicg_p(self, r, p, v, beta, omega):
        self._upd(REACH_BLOCK_P, 0.0, beta, omega, r=r, p=p, v=v, out=False)

    def bicg_s(self, r, v, alpha, s):
        self._upd(REACH_BLOCK_S, alpha, 0.0, 0.0, r=r, v=v, s=s)
        return self._scalar(0)

    def bicg_xr(self, x, p, s, t, alpha, omega, r):
        self._upd(REACH_BLOCK_XR, alpha, 0.0, omega, x=x, r=r, p=p, s=s, t=t)
        return self._scalar(0)

    def bicg_xp(self, x, p, alpha):
        self._upd(REACH_BLOCK_XP, alpha, 0.0, 0.0, x=x, p=p, out=False)




# ------------------------------------------------------------------ whole solve

def collect(local, plan, x_own):
    """All-gather every rank's own entries of x (the loops' result) into the vector over all
    rows of the system, in row order.  Yields one collective; returns a host array."""
    buf = local.zeros(plan.ext_len)
    local.copy(buf, x_own)
    gathered = yield Allgather(local.head(buf, plan.max_rows))
    g = gathered.cpu().numpy() if hasattr(gathered, "cpu") else np.asarray(gathered)
    b = plan.bounds
    return np.concatenate([g[r * plan.max_rows: r * plan.max_rows + (b[r + 1] - b[r])] for r in range(len(b) - 1)])


def solve_distributed(n, rowptr, col, val, goal, comm, method="jacobi", eps=1e-10, max_iter=1_000_000,
                      check_every=16, mode=0):
    """Pr(s |= <> GS) for every state with the rows of (I - A) x = b split over the ranks of
    `comm` (a TorchComm; one GPU per rank).  Every rank runs the partition and extraction
    (§2.2, §2.3) on its own GPU, keeps its row block, and the ranks iterate together.
    Returns (x over all states as a host array, info dict) on every rank."""
    from . import Solver
    with Solver(n, rowptr, col, val, goal, mode=mode) as s:
        cls = s.classes()
        sysm = get_system(s.ctx)
    bounds = partition_rows(sysm["rowptr"], comm.world)
    plan = block_plan(sysm["rowptr"], sysm["col"], sysm["val"], sysm["d"], sysm["b"], bounds, comm.rank)
    ops = CudaBlockOps(plan)
    try:
        if method == "jacobi":
            x_own, it, last, ok = comm.run(jacobi(ops, plan, eps, max_iter, check_every))
            status = "ok" if ok else "max_iter"
        elif method == "bicgstab":
            x_own, it, last, status = comm.run(bicgstab(ops, plan, eps, max_iter))
        else:
            raise ValueError("method must be 'jacobi' or 'bicgstab'")
        xq = comm.run(collect(ops, plan, x_own))
    finally:
        ops.close()
    x = np.zeros(n)
    x[cls == 1] = 1.0
    x[sysm["state"]] = xq
    return x, {"iters": it, "last": last, "status": status, "rows": plan.n_rows, "halo": plan.n_halo,
               "bounds": bounds.tolist()}


def get_system(ctx):
    """The extracted system over S? of a context (reach_get_system), as host arrays."""
    nq, mq = C.c_int64(0), C.c_int64(0)
    L = lib()
    st = L.reach_get_system(ctx, C.byref(nq), C.byref(mq), None, None, None, None, None, None, REACH_HOST)
    if st != 0:
        raise ReachError(st, L.reach_last_error(ctx).decode())
    out = {"rowptr": np.empty(nq.value + 1, np.int64), "col": np.empty(max(mq.value, 1), np.int32),
           "val": np.empty(max(mq.value, 1), np.float64), "d": np.empty(max(nq.value, 1), np.float64),
           "b": np.empty(max(nq.value, 1), np.float64), "state": np.empty(max(nq.value, 1), np.int64)}
    st = L.reach_get_system(ctx, None, None, *(out[k].ctypes.data for k in ("rowptr", "col", "val", "d", "b",
                                                                             "state")), REACH_HOST)
    if st != 0:
        raise ReachError(st, L.reach_last_error(ctx).decode())
    out["col"], out["val"] = out["col"][:mq.value], out["val"][:mq.value]
    for k in ("d", "b", "state"):
        out[k] = out[k][:nq.value]
    return out
