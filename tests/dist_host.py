"""Host (numpy) arithmetic for the row-split solver loops of paper_1210_6412_gb300.dist.

Test infrastructure: it stands in for the CUDA row-block kernels so that the partition,
the halo plan, the loops' control flow and their collectives can run on CPU processes
(gloo) or in one process (LockstepComm) and be compared with the oracle.  Each operation
restates the block kernel's definition in plain numpy; the Jacobi sweep sums a row's
entries in stored (ascending global column) order, as the oracle's sweep does.
"""
import numpy as np
import scipy.sparse as sp


class HostBlockOps:
    def __init__(self, plan):
        self.plan = plan
        self.n = plan.n_rows
        self.ne = plan.n_rows + plan.n_halo
        self.a = sp.csr_matrix((plan.val, plan.col.astype(np.int64), plan.rowptr), shape=(self.n, self.ne))
        self.d = plan.d
        self.b = plan.b

    # vectors
    def zeros(self, n):
        return np.zeros(max(n, 1))

    def head(self, v, n):
        return v[:n]

    def copy(self, dst, src):
        dst[:self.n] = src[:self.n]

    def fill0(self, v):
        v[:] = 0.0

    def set_b(self, r):
        r[:self.n] = self.b

    # block operations
    def halo(self, gathered, x):
        x[self.n:self.ne] = np.asarray(gathered)[self.plan.halo_src]

    def jacobi(self, x_ext, x_new):
        xe = x_ext[:self.ne]
        xn = (self.b + self.a @ xe) / self.d
        delta = float(np.max(np.abs(xn - x_ext[:self.n]))) if self.n else 0.0
        x_new[:self.n] = xn
        return lambda: delta

    def matvec(self, u_ext, y, w):
        y[:self.n] = self.d * u_ext[:self.n] - self.a @ u_ext[:self.ne]
        return float(w[:self.n] @ y[:self.n]) if w is not None else None

    def dot(self, u, v, w=None):
        return float(u[:self.n] @ v[:self.n]), (float(u[:self.n] @ w[:self.n]) if w is not None else 0.0)

    def maxabs(self, v):
        return float(np.max(np.abs(v[:self.n])))

    def bicg_p(self, r, p, v, beta, omega):
        p[:self.n] = r[:self.n] + beta * (p[:self.n] - omega * v[:self.n])

    def bicg_s(self, r, v, alpha, s):
        s[:self.n] = r[:self.n] - alpha * v[:self.n]
        return float(np.max(np.abs(s[:self.n])))

    def bicg_xr(self, x, p, s, t, alpha, omega, r):
        x[:self.n] = x[:self.n] + alpha * p[:self.n] + omega * s[:self.n]
        r[:self.n] = s[:self.n] - omega * t[:self.n]
        return float(np.max(np.abs(r[:self.n])))

    def bicg_xp(self, x, p, alpha):
        x[:self.n] = x[:self.n] + alpha * p[:self.n]


def system_of(c, mode=0):
    """(rowptr, col, val, d, b, q) of a chain's system over S? from the oracle: A without its
    diagonal, d = 1 - A_ii (the layout the library's reach_get_system returns)."""
    import oracle as O
    cls = O.partition(c.n, c.rowptr, c.col, c.val, c.goal, mode)
    q, a, b = O.extract_system(c.n, c.rowptr, c.col, c.val, cls)
    d = 1.0 - a.diagonal()
    off = (a - sp.diags(a.diagonal())).tocsr()
    off.eliminate_zeros()
    off.sort_indices()
    return off.indptr.astype(np.int64), off.indices.astype(np.int32), off.data, d, b, q, O.system_matrix(a)


def gloo_worker(rank, world, port, chain, method, eps, max_iter, check_every, out):
    """One CPU rank: the row block of `chain`'s system, the loop over gloo collectives."""
    import os
    import torch.distributed as dist
    from paper_1210_6412_gb300 import dist as D
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rp, ci, v, d, b, q, _ = system_of(chain)
        comm = D.TorchComm("cpu")
        bounds = D.partition_rows(rp, world)
        plan = D.block_plan(rp, ci, v, d, b, bounds, rank)
        ops = HostBlockOps(plan)
        gen = D.jacobi(ops, plan, eps, max_iter, check_every) if method == "jacobi" else \
            D.bicgstab(ops, plan, eps, max_iter)
        res = comm.run(gen)
        xq = comm.run(D.collect(ops, plan, res[0]))
        out.put((rank, xq, res[1], res[2], res[3], plan.n_halo))
    finally:
        dist.destroy_process_group()
