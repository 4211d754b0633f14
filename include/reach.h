/*
 * reach.h -- C ABI of the GB300 (sm_103a) reachability-probability solver.
 *
 * Problem (Cormie-Bowins, "A Comparison of Sequential and GPU Implementations of
 * Iterative Methods to Compute Reachability Probabilities", GRAPHITE 2012):
 * given a discrete-time Markov chain (S, P, s0) with row-stochastic P (§2) and a
 * set of goal states GS, compute x_s = Pr(s |= <> GS) for every state (§2.1).
 * The states are split into S=0, S=1 and S? by graph search (§2.2); on S? the
 * values solve (I - A) x = b with A = P restricted to S? and b_s the one-step
 * probability of entering S=1 (§2.3), by Jacobi (§3.1) or BiCGStab (§3.2).
 *
 * Conventions shared by every entry point:
 *   - Status is the return value; no exception crosses the ABI.  After a failure
 *     reach_last_error() gives a one-line reason.
 *   - The matrix is compressed row storage (§4): rowptr int64[n+1] (rowptr[0] = 0,
 *     rowptr[n] = m), col int32[m] in [0, n), val float64[m].  Columns need not be
 *     sorted; duplicate (s, s') entries are summed; an entry with value 0 is no
 *     edge.  Every row must sum to 1 within 1e-9.
 *   - `flags` says where caller pointers live: REACH_HOST or REACH_DEVICE (memory
 *     of the current CUDA device).  Inputs are copied, so the caller keeps
 *     ownership and may free them when the call returns; outputs are written
 *     into caller-allocated buffers.
 *   - All device work of a context runs on the stream given to reach_create
 *     (NULL = the legacy default stream).  Calls that return data to the host
 *     synchronise that stream; calls with REACH_DEVICE outputs do not, except where
 *     stated.  A context is not thread-safe.
 *   - Precision: FP64 unless a method says otherwise.
 */
#ifndef REACH_H_
#define REACH_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct reach_ctx reach_ctx;
typedef struct reach_batch reach_batch;

typedef enum {
  REACH_OK = 0,
  REACH_EINVAL = 1,      /* bad argument or input that is not a Markov chain */
  REACH_ENOMEM = 2,      /* device allocation failed */
  REACH_ECUDA = 3,       /* a CUDA runtime call failed */
  REACH_ESTATE = 4,      /* call out of order (e.g. solve before precompute) */
  REACH_ENOTCONV = 5,    /* max_iter reached before the stopping rule held */
  REACH_EBREAKDOWN = 6,  /* BiCGStab breakdown that a restart did not cure */
  REACH_ETIMEOUT = 7     /* a bounded device-side wait gave up */
} reach_status;

enum { REACH_HOST = 0, REACH_DEVICE = 1 };

/* Partition modes (§2.2).  PROB01: S=0 = states that cannot reach GS; S=1 =
 * states that cannot reach S=0 along a path avoiding GS (GS included); S? = rest.
 * PROB0_ONLY: S=1 = GS, so S? = S \ (S=0 u GS) and b_s = P(s, GS), the system as
 * written in §2.3.  Both give the same x. */
typedef enum { REACH_PROB01 = 0, REACH_PROB0_ONLY = 1 } reach_precomp_mode;

/* Solvers.  JACOBI_FP64: x_i <- (b_i + sum_{j != i} A_ij x_j) / (1 - A_ii), double
 * buffered (§3.1), stop when max|x' - x| < eps.  The sweeps run on the Jacobi form
 * D^-1 A, D^-1 b (d_i = 1 - A_ii), scaled once per system, so no sweep divides.
 * JACOBI_MIXED: the same iteration run as defect correction -- every refine_k sweeps an
 * FP64 residual r / d = D^-1 b + D^-1 A x - x (the values D^-1 A as FP32 hi + lo pairs),
 * then refine_k - 1 FP32 sweeps on (I - D^-1 A) e = r / d, then x += e in FP64; stop when
 * max|r_i / d_i| < eps (the FP64 Jacobi step).
 * BICGSTAB_FP64: unpreconditioned BiCGStab (§3.2) with x = 0 and shadow q = b;
 * stop when max|s| < eps after the a-step (then x += a p) or max|r| < eps. */
typedef enum {
  REACH_JACOBI_FP64 = 0,
  REACH_JACOBI_MIXED = 1,
  REACH_BICGSTAB_FP64 = 2,
  /* The FP64 Jacobi iteration and stopping rule of JACOBI_FP64 with a different sweep:
   * work is split over stored entries instead of rows, by a segmented reduction over
   * the flat entry array (the related work of §8 runs Jacobi on a segmented scan), so
   * very long rows do not serialise on one warp.  Only the summation order differs. */
  REACH_JACOBI_SEG = 3,
  /* Jacobi one level of strongly connected components at a time, in reverse
   * topological order (the future-work idea of §8): the decomposition of reach_scc
   * (computed on first use), then for level 0, 1, ...: a level of single-row
   * components is exact after one sweep; any other level runs the FP64 Jacobi sweep of
   * §3.1 on its own rows, with all other rows held fixed, until max|x' - x| < eps over
   * them.  max_iter bounds the total sweeps over all levels (at least one per level).
   * info->iters counts those sweeps; ms_solve includes the decomposition when this call
   * computed it. */
  REACH_SCC_JACOBI = 4
} reach_method;

typedef struct {
  int64_t iters;          /* Jacobi sweeps or BiCGStab iterations performed */
  int64_t n_q;            /* |S?| */
  int64_t m_q;            /* stored off-diagonal entries of A */
  double last_delta;      /* stopping quantity at exit (max|dx|, max|s| or max|r|) */
  double resid_inf;       /* FP64 max_i |b - (I - A) x|_i at exit */
  double ms_precompute;   /* device time of the last reach_precompute */
  double ms_solve;        /* device time of this solve (CUDA events on the stream) */
  double bytes_moved;     /* algorithmic HBM bytes of this solve */
  int32_t status;         /* reach_status of the solve */
  int32_t refinements;    /* JACOBI_MIXED: FP64 residual steps taken */
  /* Certified bound on max_i |x*_i - x_i| over S?, where x* solves the stored FP64 system
   * (I - A) x* = b exactly (x = 1 on S=1 and 0 on S=0 are exact): ||(I - A)^-1||_inf times
   * an upper bound of the exact ||b - (I - A) x||_inf of the returned x, with the residual's
   * rounding error bounded and every step rounded upward.  The norm bound is the smaller of
   * Varah's, 1 / min_i (|d_i| - sum_j |A_ij|) (Varah 1975; d_i - sum_j A_ij is a chain
   * state's one-step probability of leaving S?), taken at reach_precompute, and the one
   * from reach_norm_bound.  +inf when neither is available (some S? state cannot leave S?
   * in one step and reach_norm_bound was not called).  reach_grad: the bound on the adjoint
   * solution y from Varah's margin over the columns of A.  reach_norm_bound: its norm bound
   * from the approximate tau alone. */
  double err_bound;
} reach_info;

/* Strongly connected components of the digraph of A over S? (an edge i -> j for each
 * stored off-diagonal A_ij), from reach_scc. */
typedef struct {
  int64_t n_q;            /* rows of the system (|S?|) */
  int64_t n_scc;          /* components */
  int64_t n_levels;       /* levels of the condensation (the solve order of REACH_SCC_JACOBI) */
  int64_t n_trivial;      /* single-row components */
  int64_t largest;        /* rows of the largest component */
  int32_t exact;          /* 1: the components are exact; 0: the colouring hit its round cap
                           * and the cyclic core left after trimming is one block (still a
                           * valid solve order, coarser than the components) */
  int32_t rounds;         /* colouring rounds run */
  double ms;              /* device time of the decomposition */
  int64_t passes;         /* passes over a frontier or over all rows (trimming, colouring,
                           * searches and levels): the decomposition's sequential depth */
} reach_scc_info;

/* Create a context holding a copy of P and the goal mask (§2, §4).
 * goal: uint8[n], nonzero marks GS.  Validates the chain on the device (column
 * range, finite values in [0, 1], row sums) and returns REACH_EINVAL with a reason
 * when it fails.  stream: a cudaStream_t, or NULL.  *out is set on success only. */
reach_status reach_create(reach_ctx** out, int64_t n, int64_t m, const int64_t* rowptr,
                          const int32_t* col, const double* val, const uint8_t* goal,
                          int32_t flags, void* stream);

/* A general sparse system M x = b instead of a chain: the random diagonally dominant
 * matrices of §6 that the paper solves with the same Jacobi (§3.1) and BiCGStab (§3.2).
 * M in the CSR layout above (finite values, any sign; duplicates summed; every diagonal
 * entry non-zero), b: float64[n], same memory kind.  The context is ready for
 * reach_solve at once (every row is an unknown; no partition, reach_precompute returns
 * REACH_ESTATE): Jacobi runs x_i <- (b_i - sum_{j != i} M_ij x_j) / M_ii and BiCGStab
 * runs on M.  reach_grad is not defined for it (REACH_ESTATE). */
reach_status reach_system_create(reach_ctx** out, int64_t n, int64_t m, const int64_t* rowptr,
                                 const int32_t* col, const double* val, const double* b,
                                 int32_t flags, void* stream);

/* Partition S into S=0 / S=1 / S? by backward search over the underlying digraph
 * (§2.2), then build A (off-diagonal, CSR over S? in ascending state order),
 * d = 1 - diag(A) and b (§2.3).  mode: reach_precomp_mode.  Narrow search levels run on
 * one thread-block cluster, medium ones top-down over the reversed digraph (built on the
 * first such level), wide ones bottom-up over P itself; the resulting classes are the
 * same.  REACH_BFS_CLUSTER=0, REACH_BFS_LQ=0 and REACH_BFS_PULL=0 in the environment
 * switch off the cluster, its shared-memory queues and the bottom-up levels. */
reach_status reach_precompute(reach_ctx* ctx, int32_t mode);

/* Class of every state after reach_precompute: 0 = S=0, 1 = S=1, 2 = S?.
 * cls: uint8[n] in host or device memory per flags. */
reach_status reach_get_classes(reach_ctx* ctx, uint8_t* cls, int32_t flags);

/* Solve (I - A) x = b on S? (§2.3) with `method` and write the full vector
 * x_out[n] = Pr(s |= <> GS) (1 on S=1, 0 on S=0).  eps > 0; max_iter >= 1;
 * refine_k (JACOBI_MIXED) >= 2 and even, 0 = default 16; x0: optional float64[n]
 * starting point (its S? entries are used; NULL = 0), same memory kind as x_out.
 * info may be NULL.  Returns REACH_ENOTCONV when max_iter ran out (x_out still
 * holds the last iterate).  Synchronises the stream.
 * Small systems (16-bit columns, fitting the shared memory of 16 SMs) run the mixed method,
 * and FP64 Jacobi up to 10240 stored entries, as one launch on a thread-block cluster of
 * 16 CTAs with the matrix in shared memory, the iterate exchanged through distributed
 * shared memory and one cluster barrier per sweep; same iteration, stopping rule and
 * iteration count.  REACH_SMALL=0 in the environment turns this off, REACH_SMALL=1 uses
 * it for FP64 Jacobi whenever the system fits. */
reach_status reach_solve(reach_ctx* ctx, int32_t method, double eps, int64_t max_iter,
                         int32_t refine_k, const double* x0, double* x_out, int32_t flags,
                         reach_info* info);

/* The system over S? that reach_precompute extracted (§2.3), for callers that split it
 * (e.g. over several GPUs with the row blocks below): n_q and m_q (host, may be NULL), A
 * off-diagonal in CSR (rowptr int64[n_q+1], col int32[m_q] in [0, n_q), val float64[m_q];
 * rows and columns in ascending state order), d = 1 - A_ii float64[n_q], b float64[n_q] and
 * state int64[n_q] (the state of each row).  Any array pointer may be NULL (not written);
 * call with NULL arrays first to read the sizes.  Arrays per flags.  Synchronises the
 * stream. */
reach_status reach_get_system(reach_ctx* ctx, int64_t* n_q, int64_t* m_q, int64_t* rowptr, int32_t* col,
                              double* val, double* d, double* b, int64_t* state, int32_t flags);

/* Certified upper bound of ||(I - A)^-1||_inf for the current chain system (§2.3), for the/* Certified upper bound of ||(I - A)^-1||_inf for the current chain system (§2.3), for the
 * error bound of every later reach_solve.  Solves (I - A) tau = 1 -- tau_s is the expected
 * number of steps a walk from s spends in S? -- with `method` (JACOBI_FP64, JACOBI_MIXED or
 * BICGSTAB_FP64; eps and max_iter as in reach_solve; refinement period 16), then checks the
 * approximate tau' it returns: with c = min_i ((I - A) tau')_i, bounded from below with
 * directed rounding, c > 0 gives ||(I - A)^-1||_inf <= max_i tau'_i / c, because
 * (I - A)^-1 >= 0 entrywise for a chain.  This needs no exit margin, so it bounds chains
 * whose states do not all leave S? in one step, and it is close to the true norm when tau'
 * is accurate.  *kinv (host, may be NULL) receives the norm bound now in use (the smaller
 * of this one and Varah's; +inf if c <= 0).  info (may be NULL) describes the tau solve.
 * The system's b is restored afterwards; the context's last solution for reach_grad is
 * kept.  REACH_ESTATE for a general system (reach_system_create), where (I - A)^-1 >= 0
 * does not hold.  A tau solve that hits max_iter still yields a valid (looser) bound and
 * returns REACH_OK.  Synchronises the stream. */
reach_status reach_norm_bound(reach_ctx* ctx, int32_t method, double eps, int64_t max_iter, double* kinv,
                              reach_info* info);

/* Strongly connected components of the digraph of A over S? and their levels (§8:
 * the paper's future work takes the components in reverse topological order).  After
 * reach_precompute (or reach_system_create).  The decomposition runs on the device
 * once per system and is kept for REACH_SCC_JACOBI.  label: int32[n?] or NULL, the
 * component of every S? row (rows in ascending state order, as in A), named by its
 * largest row index; level: int32[n?] or NULL, the component's level -- 0 when no
 * edge leaves it, else one above the highest component it has an edge to.  Host or
 * device memory per flags.  info may be NULL.  max_rounds bounds the colouring rounds
 * (0 = 256); past it the cyclic core is kept as one block (info->exact = 0).
 * Synchronises the stream. */
reach_status reach_scc(reach_ctx* ctx, int32_t* label, int32_t* level, int32_t flags, int32_t max_rounds,
                       reach_scc_info* info);

/* Autotuner for the row mapping of `method` on the current system (after
 * reach_precompute).  Times every candidate mapping of the method's dominant kernel --
 * lanes per row 1 (the paper's one thread per row, §5.1; tried only when rows average at
 * most 8 entries), 2, 4, 8, 16, 32, half a warp or a warp with 16-byte vector loads
 * (reported as 48 and 64; 66 for the FP32 sweep with four quads per trip), or
 * entry-balanced tiles of 4096 stored entries (reported as 128: the segmented sweep of
 * REACH_JACOBI_SEG, and for BiCGStab a segmented product followed by the elementwise M u
 * with its dot products; it wins when a few rows are very long) -- for a few launches and
 * keeps the fastest for later solves of this context.  Two FP32-sweep variants are not
 * candidates and are chosen only through the REACH_LANES environment variable: 72 (the
 * correction vector staged in shared memory) and 80 (rows staged by bulk copies).  For
 * JACOBI_FP64 it also picks the sweeps between convergence checks, used when
 * reach_solve gets refine_k = 0.  Setting REACH_AUTOTUNE=1 in the environment makes the
 * first reach_solve of each method run it.  Outputs (host, may be NULL): the chosen
 * mapping, its time per sweep in ms, and the sweeps between checks.  Rows of this
 * library's kernels are cut the same way for every method; the paper itself fixes the
 * one-thread-per-row mapping. */
reach_status reach_autotune(reach_ctx* ctx, int32_t method, int32_t* lanes, double* sweep_ms,
                            int32_t* check_every);

/* Average device time, in ms, of `launches` (1..1000) back-to-back launches of one
 * solver kernel on the context stream, in the layout the solves use, measured with
 * CUDA events on that stream after one warm-up launch: kernel 0 = FP64 Jacobi sweep
 * (§3.1), 1 = FP32 sweep of the mixed method, 2 = its FP64 residual step, 3 = the
 * BiCGStab product v = (I - A) p (§3.2).  For roofline figures (bytes or flops of one
 * launch over this time).  Overwrites solve workspace: solve again before reach_grad. */
reach_status reach_time_kernel(reach_ctx* ctx, int32_t kernel, int32_t launches, double* avg_ms);

/* Gradient of x_init with respect to every stored entry of P, in input order:
 * grad[k] = y_s * x_{col[k]} for an entry of row s in S?, else 0, where
 * (I - A)^T y = e_init is solved by Jacobi on the transposed system (FP64, stop at
 * max|y' - y| < eps).  Uses the x of the last successful reach_solve (REACH_ESTATE
 * without one).  init in [0, n).  grad: float64[m] per flags. */
reach_status reach_grad(reach_ctx* ctx, int64_t init, double eps, int64_t max_iter,
                        double* grad, int32_t flags, reach_info* info);

/* reach_grad with the adjoint system solved by `method`: REACH_JACOBI_FP64 (what reach_grad
 * does) or REACH_BICGSTAB_FP64 -- BiCGStab of §3.2 on (I - A)^T, with the stopping rule of
 * the forward BiCGStab.  Any other method: REACH_EINVAL.  Arguments as in reach_grad. */
reach_status reach_grad_method(reach_ctx* ctx, int32_t method, int64_t init, double eps, int64_t max_iter,
                               double* grad, int32_t flags, reach_info* info);

/* Parametric chains: P_e = softmax over the out-edges of each row of
 * theta[cls_e] + offset_e.  All pointers are device memory; rows must be non-empty;
 * cls_e in [0, n_classes).  p_out: float64[m].  Runs on `stream`, no sync. */
reach_status reach_param_probs(int64_t n, int64_t m, const int64_t* rowptr, const int32_t* cls,
                               const double* offset, const double* theta, int32_t n_classes,
                               double* p_out, void* stream);

/* Chain rule through the row softmax: dl_f = P_f (g_f - sum_e P_e g_e) per row and
 * g_theta[c] = sum of dl_f over edges of class c.  Device pointers; g_theta:
 * float64[n_classes], overwritten.  Runs on `stream`, no sync. */
reach_status reach_param_grad_theta(int64_t n, int64_t m, const int64_t* rowptr,
                                    const int32_t* cls, const double* p, const double* g_p,
                                    int32_t n_classes, double* g_theta, void* stream);

/* ---- Batched multi-RHS: K <= 8 goal sets over one chain ---------------------------
 * Many independent chains are solved together by passing their block-diagonal union
 * (state ids offset per chain).  Each goal set j has its own partition (§2.2) and
 * system (§2.3); one pass over the matrix serves all K right-hand sides.
 *
 * goals: uint8[k * n], goal set j in goals[j*n .. j*n + n); nonzero marks GS_j.  P is
 * validated as in reach_create.  The context copies every input. */
reach_status reach_batch_create(reach_batch** out, int64_t n, int64_t m, const int64_t* rowptr,
                                const int32_t* col, const double* val, int32_t k,
                                const uint8_t* goals, int32_t flags, void* stream);

/* S=0_j / S=1_j / S?_j for every goal set j (mode as in reach_precompute) by a
 * bit-parallel backward fixed point over P (one bit per goal set), plus the
 * off-diagonal part of P over all states as FP32 hi + lo pairs and d = 1 - P(s,s). */
reach_status reach_batch_precompute(reach_batch* b, int32_t mode);

/* Classes as uint8[k * n] (0 = S=0, 1 = S=1, 2 = S?), goal-set major. */
reach_status reach_batch_get_classes(reach_batch* b, uint8_t* cls, int32_t flags);

/* Jacobi on every right-hand side at once, as FP32 sweeps with an FP64 residual and
 * correction every refine_k sweeps (even, in [2, 62]; 0 = 32):
 * x_j[s] <- sum_{s' != s} P(s,s') x_j[s'] / (1 - P(s,s)) on S?_j, with x_j = 1 on
 * S=1_j and 0 on S=0_j.  Stops when the largest FP64 Jacobi step over all S?_j is
 * below eps -- per chain once reach_batch_set_chains has named the chains; info->iters
 * is then the sweep count of the slowest chain and info->last_delta the largest last
 * step; info->err_bound is +inf (no norm bound per goal set is computed for a batch).
 * x_out: float64[k * n], goal-set major.  Synchronises the stream. */
reach_status reach_batch_solve(reach_batch* b, double eps, int64_t max_iter, int32_t refine_k,
                               double* x_out, int32_t flags, reach_info* info);

/* Autotuner of the batched solve (after reach_batch_precompute): times every variant of
 * the FP32 multi-RHS sweep on this batch -- 0: two lanes per row, each gathering four
 * right-hand sides as one 16-byte load (the default); 1: eight lanes per row, one
 * right-hand side each; 2: as 0 with the gathers of the corrections marked evict-last
 * in L2 (the matrix and the streamed vectors are evict-first); 3: as 0 with the index
 * and value loads of a row's next four entries issued before the current gathers
 * complete; 4: 2 and 3 together -- for a few launches each and keeps the fastest.  Then
 * it times one FP64 residual step c and picks the refinement period
 * k = sqrt(2 N c / t) for N = 500 sweeps and sweep time t (even, in [8, 62]), used by
 * reach_batch_solve when it gets refine_k = 0.  Setting REACH_AUTOTUNE=1 in the
 * environment makes the first reach_batch_solve run it.  Outputs (host, may be NULL): the
 * variant, its time per sweep in ms, the period.  The rows a chain solve visits and its
 * results do not depend on the variant; only the summation order of the sweeps does. */
reach_status reach_batch_autotune(reach_batch* b, int32_t* variant, double* sweep_ms, int32_t* refine_k);

/* The chains of a batch whose matrix is the block-diagonal union of independent chains:/* The chains of a batch whose matrix is the block-diagonal union of independent chains:
 * chain c owns states [offsets[c], offsets[c+1]) and no positive entry of P leaves it.
 * With chains set, reach_batch_solve applies its stopping rule to each chain on its own
 * (the largest FP64 Jacobi step over the chain's S?_j, all goal sets): a chain that
 * meets it leaves the later sweeps untouched, so its x is exactly the x of solving that
 * chain alone with the same eps and refine_k.  Until this is called the whole batch is
 * one chain.  offsets: int64[n_chains + 1] in host memory, offsets[0] = 0,
 * non-decreasing, offsets[n_chains] = n.  REACH_EINVAL (and the chains stay as they
 * were) for bad offsets or a positive entry of P that crosses a chain boundary.
 * Synchronises the stream. */
reach_status reach_batch_set_chains(reach_batch* b, int32_t n_chains, const int64_t* offsets);

/* Per chain, after reach_batch_solve: iters[c] = the sweep count at which chain c met
 * the stopping rule (-1 if it did not within max_iter), last[c] = its last FP64 Jacobi
 * step (max over its S?_j).  Host arrays of n_chains entries; either may be NULL. */
reach_status reach_batch_chain_info(reach_batch* b, int64_t* iters, double* last);

/* Release the batch.  NULL is a no-op. */
void reach_batch_destroy(reach_batch* b);

/* ---- Row blocks for a solve spread over several GPUs -------------------------------
 * The related work of §8 runs Jacobi on two GPUs and its future work is a multi-GPU
 * BiCGStab; both split the rows of (I - A) x = b (§2.3).  A row block is one process's
 * share on its own GPU: rows [r0, r1) of A (off-diagonal entries) with d = 1 - A_ii and b,
 * its columns renumbered so that the block's own rows are columns [0, n_rows) and every
 * other column it references (its halo) is a column in [n_rows, n_rows + n_halo).  A vector
 * that a product reads is EXTENDED: n_rows own entries followed by n_halo halo entries.
 * The caller exchanges own entries between the processes (e.g. an NCCL all-gather into a
 * "gathered" vector) and reach_block_halo fills the halo entries from it:
 * halo entry j = gathered[halo_src[j]].  The caller also reduces the scalars each call
 * returns (sums of dot products, maxima) over the processes.  Every call below runs
 * asynchronously on the block's stream; vectors and scalar outputs are device memory. */
typedef struct reach_block reach_block;

/* rowptr int64[n_rows+1] (rowptr[0] = 0), col int32[m] in [0, n_rows + n_halo), val
 * float64[m] = A_ij (i != j), d float64[n_rows] (non-zero), b float64[n_rows],
 * halo_src int64[n_halo] in [0, gathered_len).  Pointers per flags; copied. */
reach_status reach_block_create(reach_block** out, int64_t n_rows, int64_t n_halo, const int64_t* rowptr,
                                const int32_t* col, const double* val, const double* d, const double* b,
                                const int64_t* halo_src, int64_t gathered_len, int32_t flags, void* stream);

/* x_ext[n_rows + j] = gathered[halo_src[j]] for every halo entry j. */
reach_status reach_block_halo(reach_block* blk, const double* gathered, double* x_ext);

/* One Jacobi sweep (§3.1) of the block: x_new_i = (b_i + sum_j A_ij x_ext_j) / d_i for its
 * rows (on the Jacobi form A_ij / d_i, b_i / d_i), and *delta = max_i |x_new_i - x_ext_i|
 * over them (one double, device). */
reach_status reach_block_jacobi(reach_block* blk, const double* x_ext, double* x_new, double* delta);

/* y = (I - A) u on the block's rows: y_i = d_i u_ext_i - sum_j A_ij u_ext_j.  With w (not
 * NULL): *dot = sum_i w_i y_i over the block's rows (the local part of a dot product). */
reach_status reach_block_matvec(reach_block* blk, const double* u_ext, double* y, const double* w, double* dot);

/* out[0] = u . v over the block's rows, and out[1] = u . w when w is not NULL. */
reach_status reach_block_dot(reach_block* blk, const double* u, const double* v, const double* w, double* out);

/* The vector updates of one BiCGStab iteration (§3.2) on the block's rows:
 *   REACH_BLOCK_P:  p = r + beta (p - omega v)
 *   REACH_BLOCK_S:  s = r - alpha v, *out = max_i |s_i|
 *   REACH_BLOCK_XR: x += alpha p + omega s, r = s - omega t, *out = max_i |r_i|
 *   REACH_BLOCK_XP: x += alpha p (the last step when max|s| met the stopping rule)
 * Arguments a stage does not use may be NULL. */
enum { REACH_BLOCK_P = 0, REACH_BLOCK_S = 1, REACH_BLOCK_XR = 2, REACH_BLOCK_XP = 3 };
reach_status reach_block_bicgstab_update(reach_block* blk, int32_t stage, double alpha, double beta, double omega,
                                         double* x, double* r, double* p, const double* v, double* s,
                                         const double* t, double* out);

/* Last error of the block's calls.  NULL: "". */
const char* reach_block_last_error(const reach_block* blk);

/* Release the block.  NULL is a no-op. */
void reach_block_destroy(reach_block* blk);

/* ---- Allocation-free Jacobi solve ----------------------------------------------------
 * The paper has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- code inside a host application that owns all device memory through its
 * own pool, code on a path where cudaMalloc/cudaFree would stall the device, or code
 * that must not hit out-of-memory once running.  It allocates nothing.  The caller
 * passes an already extracted system over S? in device memory (A off-diagonal CSR with
 * rowptr int64[n_q+1] and col int32 in [0, n_q), val float64; b and d = 1 - A_ii as
 * float64[n_q]) and x float64[n_q] (start vector in, solution out).  It runs Jacobi
 * sweeps x <- (b + A x) / d and checks max|x' - x| < eps every check_every (even, >= 2)
 * sweeps and after the last sweep, running at most max_iter sweeps (the last window is
 * shortened to fit); *iters_out and *delta_out (host, may be NULL) receive the sweep
 * count and the last max|x' - x|.
 * Scratch (the second Jacobi vector) lives in a fixed device array inside the library,
 * sized for n_q <= 524288 (4 MiB + 4 KiB, held on every device that loads the library
 * until the process exits); larger n_q returns REACH_EINVAL.  Every call looks up that
 * array's address on the current device (a lookup that allocates nothing); the first call
 * on a device also loads the library's device code there, so make that first call before
 * any stream capture.  `stream` must belong to the current device (REACH_EINVAL
 * otherwise).  Every call on a device shares the array, so calls that overlap on the GPU
 * (other streams or threads) race: serialise them.  Returns REACH_ENOTCONV when max_iter
 * runs out, REACH_ECUDA when a launch or copy fails.  Synchronises `stream` after every
 * check. */
reach_status reach_jacobi_solve_noalloc(int64_t n_q, const int64_t* rowptr, const int32_t* col,
                                        const double* val, const double* b, const double* d,
                                        double eps, int64_t max_iter, int32_t check_every,
                                        double* x, int64_t* iters_out, double* delta_out,
                                        void* stream);

/* Last error message of ctx (NULL: of the calling thread's last context-free call). */
const char* reach_last_error(const reach_ctx* ctx);

/* Release every device buffer of the context.  NULL is a no-op. */
void reach_destroy(reach_ctx* ctx);

/* Library version string. */
const char* reach_version(void);

#ifdef __cplusplus
}
#endif
#endif /* REACH_H_ */
