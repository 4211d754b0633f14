// Graph precompute of §2.2-§2.3 on the device: input validation, the reversed
// underlying digraph, backward breadth-first search for S=0 and S=1, the
// partition, and extraction of A (off-diagonal), d = 1 - A_ii and b over S?.
#include <algorithm>
#include <cstdlib>

#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace reach {

constexpr int SCAN_NT = 1024;
constexpr int SCAN_IPT = 8;
constexpr int SCAN_TILE = SCAN_NT * SCAN_IPT;

// ------------------------------------------------------------------ scans

RDEV int64_t block_incl_scan(int64_t v, int64_t* sh, int64_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    int64_t s = lane < nw ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t t = __shfl_up_sync(FULL, s, o);
      if (lane >= o) s += t;
    }
    sh[lane] = s;
  }
  __syncthreads();
  if (w > 0) v += sh[w - 1];
  *total = sh[nw - 1];
  __syncthreads();
  return v;
}

template <typename T>
__global__ void __launch_bounds__(SCAN_NT) k_scan_reduce(const T* __restrict__ in, int64_t n,
                                                          int64_t* __restrict__ bsum) {
  __shared__ int64_t sh[32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int64_t s = 0;
#pragma unroll
  for (int j = 0; j < SCAN_IPT; ++j) {
    int64_t i = base + threadIdx.x + (int64_t)j * SCAN_NT;
    if (i < n) s += (int64_t)in[i];
  }
  int64_t tot;
  block_incl_scan(s, sh, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SCAN_NT) k_scan_top(int64_t* bsum, int64_t nb, int64_t* total) {
  __shared__ int64_t sh[32];
  int64_t carry = 0;
  for (int64_t t0 = 0; t0 < nb; t0 += SCAN_NT) {
    int64_t i = t0 + threadIdx.x;
    int64_t v = i < nb ? bsum[i] : 0, tot;
    int64_t incl = block_incl_scan(v, sh, &tot);
    if (i < nb) bsum[i] = carry + incl - v;
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

template <typename T>
__global__ void __launch_bounds__(SCAN_NT) k_scan_apply(const T* __restrict__ in, int64_t n,
                                                         const int64_t* __restrict__ bsum,
                                                         int64_t* __restrict__ out) {
  __shared__ int64_t sh[32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_IPT;
  int64_t loc[SCAN_IPT];
  int64_t s = 0;
#pragma unroll
  for (int j = 0; j < SCAN_IPT; ++j) {
    int64_t i = base + j;
    loc[j] = s;
    s += i < n ? (int64_t)in[i] : 0;
  }
  int64_t tot;
  int64_t incl = block_incl_scan(s, sh, &tot);
  const int64_t off = bsum[blockIdx.x] + incl - s;
#pragma unroll
  for (int j = 0; j < SCAN_IPT; ++j) {
    int64_t i = base + j;
    if (i < n) out[i] = off + loc[j];
  }
}

// out[i] = sum_{j<i} in[j] for i in [0, n], so out has n+1 entries; *total_dev = out[n].
template <typename T>
static cudaError_t exclusive_scan(const T* in, int64_t* out, int64_t n, int64_t* total_dev,
                                  int64_t* bsum, cudaStream_t s) {
  const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nb > 0) {
    k_scan_reduce<T><<<(unsigned)nb, SCAN_NT, 0, s>>>(in, n, bsum);
  }
  k_scan_top<<<1, SCAN_NT, 0, s>>>(bsum, nb, out + n);
  if (nb > 0) k_scan_apply<T><<<(unsigned)nb, SCAN_NT, 0, s>>>(in, n, bsum, out);
  if (total_dev) cudaMemcpyAsync(total_dev, out + n, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ validation

template <int G>
__global__ void k_validate(int64_t n, int64_t m, const int64_t* __restrict__ rp,
                           const int32_t* __restrict__ col, const double* __restrict__ val,
                           double tol, unsigned* err, int64_t* bad_row, int general) {
  RowGroups rg = RowGroups::make<G>();
  for (int64_t s = rg.first; warp_has_row<G>(s, n); s += rg.stride) {
    bool act = s < n;
    unsigned e = 0;
    double sum = 0.0;
    if (act) {
      int64_t lo = rp[s], hi = rp[s + 1];
      if (lo < 0 || hi < lo || hi > m) {
        e |= VERR_ROWPTR;
      } else {
        for (int64_t k = lo + rg.lane; k < hi; k += G) {
          int32_t cc = col[k];
          double v = val[k];
          if (cc < 0 || (int64_t)cc >= n) e |= VERR_COL;
          // a chain needs probabilities; a general system only finite entries
          // checked on the bits (integer units, not the narrow FP64 pipe): a finite value has
          // an exponent below all ones; a probability is +-0 or a positive value up to 1.0
          const unsigned long long ub = (unsigned long long)__double_as_longlong(v);
          const bool bad = general ? ((ub >> 52) & 0x7ffull) == 0x7ffull
                                   : !((ub & 0x7fffffffffffffffull) == 0ull || ub <= 0x3ff0000000000000ull);
          if (bad) e |= VERR_VAL;
          sum += v;
        }
      }
    }
    sum = group_sum<G>(sum);
    if (!general && act && rg.lane == 0 && !(e & VERR_ROWPTR) && !(fabs(sum - 1.0) <= tol)) e |= VERR_ROWSUM;
    if (e) {
      atomicOr(err, e);
      atomicMin((unsigned long long*)bad_row, (unsigned long long)s);
    }
  }
}

// Longest row of P (rows of a bad rowptr count as 0; validation reports those).
__global__ void k_max_row(int64_t n, const int64_t* __restrict__ rp, unsigned long long* out) {
  unsigned long long mx = 0ull;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t len = rp[s + 1] - rp[s];
    if (len > 0 && (unsigned long long)len > mx) mx = (unsigned long long)len;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(FULL, mx, o);
    mx = y > mx ? y : mx;
  }
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

// Rows this long, or longer, make the row-wise graph kernels take a warp per row: with
// fewer lanes a few very long rows (hubs) would serialise on a handful of them.
constexpr int64_t LONG_ROW = 4096;

int graph_group(reach_ctx* c, int64_t rows, int64_t nnz) {
  return c->max_row >= LONG_ROW ? 32 : pick_group(rows, nnz);
}

cudaError_t launch_validate(reach_ctx* c) {
  const int64_t mean = c->n ? c->m / c->n : 0;
  cudaMemsetAsync(c->verr, 0, sizeof(unsigned), c->stream);
  cudaMemsetAsync(c->vrow, 0x7f, sizeof(int64_t), c->stream);
  cudaMemsetAsync(c->maxrow, 0, sizeof(unsigned long long), c->stream);
  k_max_row<<<grid_for(c, (const void*)k_max_row, 256, c->n), 256, 0, c->stream>>>(c->n, c->rowptr, c->maxrow);
  unsigned long long mr = 0ull;
  cudaError_t e = cudaMemcpyAsync(&mr, c->maxrow, sizeof(mr), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return e;
  c->max_row = (int64_t)mr;
  if (mean >= 16 || c->max_row >= LONG_ROW) {
    int grid = grid_for(c, (const void*)k_validate<32>, 256, c->n * 32);
    k_validate<32><<<grid, 256, 0, c->stream>>>(c->n, c->m, c->rowptr, c->col, c->val, 1e-9,
                                                c->verr, c->vrow, c->general ? 1 : 0);
  } else {
    int grid = grid_for(c, (const void*)k_validate<4>, 256, c->n * 4);
    k_validate<4><<<grid, 256, 0, c->stream>>>(c->n, c->m, c->rowptr, c->col, c->val, 1e-9,
                                               c->verr, c->vrow, c->general ? 1 : 0);
  }
  return cudaGetLastError();
}

// A general system needs every diagonal entry non-zero (Jacobi divides by it).
__global__ void k_check_diag(int64_t nq, const double* __restrict__ d, unsigned* err, int64_t* bad_row) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (d[i] == 0.0) {
      atomicOr(err, VERR_ROWSUM);
      atomicMin((unsigned long long*)bad_row, (unsigned long long)i);
    }
  }
}

cudaError_t check_diagonal(reach_ctx* c) {
  cudaMemsetAsync(c->verr, 0, sizeof(unsigned), c->stream);
  cudaMemsetAsync(c->vrow, 0x7f, sizeof(int64_t), c->stream);
  if (c->n_q > 0)
    k_check_diag<<<grid_for(c, (const void*)k_check_diag, 256, c->n_q), 256, 0, c->stream>>>(
        c->n_q, c->d, c->verr, c->vrow);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ reversed digraph

template <int G>
__global__ void k_rev_count(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const double* __restrict__ val, uint32_t* cnt) {
  RowGroups rg = RowGroups::make<G>();
  for (int64_t s = rg.first; s < n; s += rg.stride) {
    for (int64_t k = rp[s] + rg.lane; k < rp[s + 1]; k += G)
      if (val[k] > 0.0) atomicAdd(cnt + col[k], 1u);
  }
}

template <int G>
__global__ void k_rev_fill(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const double* __restrict__ val, uint32_t* cnt,
                           const int64_t* __restrict__ trp, int32_t* __restrict__ tcol) {
  RowGroups rg = RowGroups::make<G>();
  for (int64_t s = rg.first; s < n; s += rg.stride) {
    for (int64_t k = rp[s] + rg.lane; k < rp[s + 1]; k += G) {
      if (val[k] > 0.0) {
        int32_t cc = col[k];
        uint32_t pos = atomicSub(cnt + cc, 1u) - 1u;
        tcol[trp[cc] + pos] = (int32_t)s;
      }
    }
  }
}

cudaError_t build_reverse_pattern(reach_ctx* c) {
  cudaStream_t s = c->stream;
  const int64_t n = c->n;
  uint32_t* cnt = reinterpret_cast<uint32_t*>(c->queue);   // n entries of scratch
  cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * n, s);
  const int g = graph_group(c, n, c->m);
  int64_t* bsum = reinterpret_cast<int64_t*>(c->part);
#define REV_LAUNCH(G)                                                                         \
  {                                                                                           \
    int grid = grid_for(c, (const void*)k_rev_count<G>, 256, n * G);                          \
    k_rev_count<G><<<grid, 256, 0, s>>>(n, c->rowptr, c->col, c->val, cnt);                  \
    exclusive_scan<uint32_t>(cnt, c->t_rowptr, n, nullptr, bsum, s);                          \
    k_rev_fill<G><<<grid, 256, 0, s>>>(n, c->rowptr, c->col, c->val, cnt, c->t_rowptr, c->t_col); \
  }
  switch (g) {
    case 2: REV_LAUNCH(2) break;
    case 4: REV_LAUNCH(4) break;
    case 8: REV_LAUNCH(8) break;
    case 16: REV_LAUNCH(16) break;
    default: REV_LAUNCH(32) break;
  }
#undef REV_LAUNCH
  return cudaGetLastError();
}

// ------------------------------------------------------------------ backward BFS

RDEV uint32_t agg_inc(uint32_t* ctr) {
  cg::coalesced_group g = cg::coalesced_threads();
  uint32_t prev = 0;
  if (g.thread_rank() == 0) prev = atomicAdd(ctr, (uint32_t)g.size());
  prev = g.shfl(prev, 0);
  return prev + g.thread_rank();
}

RDEV bool bit_of(const uint32_t* v, int64_t s) { return (v[s >> 5] >> (s & 31)) & 1u; }

// Fetches the line holding *p into L2 without waiting for it.
RDEV void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Sources: kind 0 = goal states; kind 1 = states NOT marked in `other` (S=0).  avoid_goal:
// goal states are marked visited from the start without being sources, so the search never
// enters them and no level has to read the goal mask (their bits mean nothing afterwards).
__global__ void k_bfs_init(int64_t n, int kind, int avoid_goal, const uint8_t* __restrict__ goal,
                           const uint32_t* __restrict__ other, uint32_t* vis, int32_t* q0,
                           BfsState* st) {
  const int64_t words = (n + 31) >> 5;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words;
       w += (int64_t)gridDim.x * blockDim.x) {
    uint32_t bits = 0, blocked = 0;
    for (int j = 0; j < 32; ++j) {
      int64_t s = w * 32 + j;
      if (s >= n) break;
      bool src = kind == 0 ? goal[s] != 0 : !bit_of(other, s);
      if (src) bits |= 1u << j;
      else if (avoid_goal && goal[s]) blocked |= 1u << j;
    }
    vis[w] = bits | blocked;
    int nb = __popc(bits);
    if (nb) {
      uint32_t base = atomicAdd(&st->count[0], (uint32_t)nb);
      for (int j = 0; j < 32; ++j)
        if (bits & (1u << j)) q0[base++] = (int32_t)(w * 32 + j);
    }
  }
}

template <int G>
__global__ void k_bfs_level(const int64_t* __restrict__ trp, const int32_t* __restrict__ tcol,
                            const uint8_t* __restrict__ goal, int avoid_goal, uint32_t* vis,
                            int32_t* qa, int32_t* qb, BfsState* st, unsigned* ticket,
                            cudaGraphConditionalHandle h, int use_cond) {
  const int L = st->level;
  const int cur = L % 3, nxt = (L + 1) % 3;
  const uint32_t cnt = st->count[cur];
  if (cnt == 0) {  // the search already ended (in the cluster kernel of this body)
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
    return;
  }
  // the frontier count of level L - 1 becomes the push target of level L + 1 (the rule of
  // the cluster kernel too, whichever kernel runs each level)
  if (blockIdx.x == 0 && threadIdx.x == 0) st->count[(L + 2) % 3] = 0u;
  const int32_t* qc = (L & 1) ? qb : qa;
  int32_t* qn = (L & 1) ? qa : qb;
  RowGroups rg = RowGroups::make<G>();
  for (int64_t i = rg.first; i < (int64_t)cnt; i += rg.stride) {
    const int32_t v = qc[i];
    const int64_t hi = trp[v + 1];
    for (int64_t k = trp[v] + rg.lane; k < hi; k += G) {
      const int32_t u = tcol[k];
      const uint32_t bit = 1u << (u & 31);
      if (__ldcg(vis + (u >> 5)) & bit) continue;
      const uint32_t old = atomicOr(vis + (u >> 5), bit);
      if (!(old & bit)) {
        qn[agg_inc(&st->count[nxt])] = u;
        prefetch_l2(trp + u);   // the next level reads u's row of the reversed graph
      }
    }
  }
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    const uint32_t next = atomicAdd(&st->count[nxt], 0u);
    st->level = L + 1;
    *ticket = 0u;
    if (use_cond) cudaGraphSetConditional(h, next > 0 ? 1u : 0u);
  }
}

template <int G>
static void launch_level(reach_ctx* c, int grid, int avoid_goal, uint32_t* vis,
                         cudaGraphConditionalHandle h, int use_cond, cudaStream_t s) {
  k_bfs_level<G><<<grid, 256, 0, s>>>(c->t_rowptr, c->t_col, c->goal, avoid_goal, vis, c->queue,
                                      c->queue + c->n, c->bfs, c->ticket, h, use_cond);
}

// Levels with small frontiers on one thread-block cluster, many per launch: the
// cluster's hardware barrier (a fraction of a microsecond) replaces the kernel boundary
// and the grid-wide ticket of k_bfs_level, which dominate a deep search through narrow
// frontiers (a model checker's layered state space: thousands of levels of a few
// thousand states).  The launch returns, with the search state as k_bfs_level keeps it,
// when the frontier is empty or its estimated edges exceed max_edges; k_bfs_level then
// runs the next level on the whole GPU.  Frontier counts, the queue and the visited
// bits are read through L2 (other SMs of the cluster wrote them).
constexpr int BFS_CL_NT = 512;

template <int G>
__global__ void __launch_bounds__(BFS_CL_NT, 1) k_bfs_cluster(const int64_t* __restrict__ trp,
                                                              const int32_t* __restrict__ tcol,
                                                              const uint8_t* __restrict__ goal, int avoid_goal,
                                                              uint32_t* vis, int32_t* qa, int32_t* qb, BfsState* st,
                                                              double mean_deg, double max_edges, int64_t max_levels) {
  cg::cluster_group cl = cg::this_cluster();
  const int64_t tid = (int64_t)cl.block_rank() * blockDim.x + threadIdx.x;
  const int64_t groups = (int64_t)cl.num_blocks() * blockDim.x / G;
  const int lane = threadIdx.x & (G - 1);
  int L = *(volatile int32_t*)&st->level;
  for (int64_t it = 0; it < max_levels; ++it) {
    const int cur = L % 3, nxt = (L + 1) % 3;
    const uint32_t cnt = *(volatile uint32_t*)&st->count[cur];
    // the same values in every thread: written before the last barrier, not since
    if (cnt == 0 || (double)cnt * mean_deg > max_edges) break;
    // the frontier count of level L - 1, read by every thread before the last barrier
    if (tid == 0) st->count[(L + 2) % 3] = 0u;
    const int32_t* qc = (L & 1) ? qb : qa;
    int32_t* qn = (L & 1) ? qa : qb;
    for (int64_t i = tid / G; i < (int64_t)cnt; i += groups) {
      const int32_t v = __ldcg(qc + i);
      const int64_t hi = trp[v + 1];
      for (int64_t k = trp[v] + lane; k < hi; k += G) {
        const int32_t u = tcol[k];
        const uint32_t bit = 1u << (u & 31);
        // no read-before-atomic filter here: on a narrow level it would add a round trip
        const uint32_t old = atomicOr(vis + (u >> 5), bit);
        if (!(old & bit)) {
          __stcg(qn + agg_inc(&st->count[nxt]), u);
          prefetch_l2(trp + u);   // the next level reads u's row of the reversed graph
        }
      }
    }
    cl.sync();  // the next frontier is complete (one barrier per level)
    ++L;
  }
  if (tid == 0) st->level = L;
}

// Cluster size the device can host for k_bfs_cluster<G> (16, else 8, else 0 = none).
template <int G>
static int bfs_cluster_size(reach_ctx* c) {
  const void* fn = (const void*)k_bfs_cluster<G>;
  for (int cs : {16, 8}) {
    if (cs > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(BFS_CL_NT);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, fn, &cfg) == cudaSuccess && nc > 0) return cs;
    cudaGetLastError();
  }
  return 0;
}

// Estimated frontier edges up to which a level runs on the cluster.  Per level the
// cluster needs about a microsecond plus its edges at a few thousand per microsecond;
// the grid-wide level about 10 microseconds (launch, ticket) plus its edges at tens of
// thousands per microsecond; they cross near 24K edges.
constexpr double BFS_CLUSTER_EDGES = 24576.0;

template <int G>
static cudaError_t launch_cluster_levels(reach_ctx* c, int cs, int avoid_goal, uint32_t* vis, cudaStream_t s) {
  const void* fn = (const void*)k_bfs_cluster<G>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(BFS_CL_NT);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const int64_t* trp = c->t_rowptr;
  const int32_t* tcol = c->t_col;
  const uint8_t* goal = c->goal;
  int32_t* qa = c->queue;
  int32_t* qb = c->queue + c->n;
  BfsState* st = c->bfs;
  double mean_deg = c->n > 0 ? std::max(1.0, (double)c->m / (double)c->n) : 1.0;
  double max_edges = BFS_CLUSTER_EDGES;
  int64_t max_levels = c->n + 2;
  void* args[] = {&trp, &tcol, &goal, &avoid_goal, &vis, &qa, &qb, &st, &mean_deg, &max_edges, &max_levels};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

static int cluster_dispatch_size(reach_ctx* c, int g) {
  switch (g) {
    case 2: return bfs_cluster_size<2>(c);
    case 4: return bfs_cluster_size<4>(c);
    case 8: return bfs_cluster_size<8>(c);
    case 16: return bfs_cluster_size<16>(c);
    default: return bfs_cluster_size<32>(c);
  }
}

static cudaError_t cluster_dispatch(reach_ctx* c, int g, int cs, int avoid_goal, uint32_t* vis, cudaStream_t s) {
  switch (g) {
    case 2: return launch_cluster_levels<2>(c, cs, avoid_goal, vis, s);
    case 4: return launch_cluster_levels<4>(c, cs, avoid_goal, vis, s);
    case 8: return launch_cluster_levels<8>(c, cs, avoid_goal, vis, s);
    case 16: return launch_cluster_levels<16>(c, cs, avoid_goal, vis, s);
    default: return launch_cluster_levels<32>(c, cs, avoid_goal, vis, s);
  }
}

static void level_dispatch(reach_ctx* c, int g, int grid, int avoid_goal, uint32_t* vis,
                           cudaGraphConditionalHandle h, int use_cond, cudaStream_t s) {
  switch (g) {
    case 2: launch_level<2>(c, grid, avoid_goal, vis, h, use_cond, s); break;
    case 4: launch_level<4>(c, grid, avoid_goal, vis, h, use_cond, s); break;
    case 8: launch_level<8>(c, grid, avoid_goal, vis, h, use_cond, s); break;
    case 16: launch_level<16>(c, grid, avoid_goal, vis, h, use_cond, s); break;
    default: launch_level<32>(c, grid, avoid_goal, vis, h, use_cond, s); break;
  }
}

// Backward search from the sources over reversed edges (§2.2).  source_kind 0:
// GS, marks vis[0..] = "can reach GS".  source_kind 1: S=0 (states not marked by
// the first search), with predecessors that are goals skipped when avoid_goal;
// marks vis[words..] = "reaches S=0 along a path avoiding GS".
cudaError_t bfs_backward(reach_ctx* c, int source_kind, bool avoid_goal) {
  const int64_t n = c->n;
  const int64_t words = (n + 31) >> 5;
  uint32_t* vis = c->vis + (source_kind == 0 ? 0 : words);
  const uint32_t* other = c->vis;
  cudaStream_t s = c->stream;
  cudaMemsetAsync(c->bfs, 0, sizeof(BfsState), s);
  cudaMemsetAsync(c->ticket, 0, sizeof(unsigned), s);
  int ig = grid_for(c, (const void*)k_bfs_init, 256, words);
  k_bfs_init<<<ig, 256, 0, s>>>(n, source_kind, avoid_goal ? 1 : 0, c->goal, other, vis, c->queue, c->bfs);
  const int g = pick_group(n, c->m);
  const int grid = c->sm_count * 4;
  // small frontiers run on one cluster (0: no cluster launch available, or disabled)
  const char* ev = std::getenv("REACH_BFS_CLUSTER");
  const int cs = (ev && ev[0] == '0') ? 0 : cluster_dispatch_size(c, g);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (c->device_loops) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle h;
    e = cudaGraphCreate(&graph, 0);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
    if (e == cudaSuccess) {
      cudaGraph_t body = np.conditional.phGraph_out[0];
      e = cudaStreamBeginCaptureToGraph(c->cap, body, nullptr, nullptr, 0,
                                        cudaStreamCaptureModeRelaxed);
      if (e == cudaSuccess) {
        if (cs > 0) e = cluster_dispatch(c, g, cs, avoid_goal ? 1 : 0, vis, c->cap);
        level_dispatch(c, g, grid, avoid_goal ? 1 : 0, vis, h, 1, c->cap);
        const cudaError_t e2 = cudaStreamEndCapture(c->cap, &body);
        if (e == cudaSuccess) e = e2;
      }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    return e;
  }
  // host-driven level loop
  BfsState hs;
  for (int64_t level = 0; level <= n + 1; ++level) {
    if (cs > 0 && (e = cluster_dispatch(c, g, cs, avoid_goal ? 1 : 0, vis, s)) != cudaSuccess) return e;
    level_dispatch(c, g, grid, avoid_goal ? 1 : 0, vis, cudaGraphConditionalHandle(), 0, s);
    e = cudaMemcpyAsync(&hs, c->bfs, sizeof(hs), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (hs.count[hs.level % 3] == 0) break;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ partition + extraction

__global__ void k_classify(int64_t n, int mode, const uint8_t* __restrict__ goal,
                           const uint32_t* __restrict__ vis0, const uint32_t* __restrict__ vis1,
                           uint8_t* __restrict__ cls, uint8_t* __restrict__ qflag) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    uint8_t k;
    // (the S=1 search marks goal states visited without entering them: a goal is S=1)
    if (!bit_of(vis0, s)) k = CLS_S0;
    else if (goal[s]) k = CLS_S1;
    else if (mode == REACH_PROB01) k = bit_of(vis1, s) ? CLS_SQ : CLS_S1;
    else k = CLS_SQ;
    cls[s] = k;
    qflag[s] = k == CLS_SQ;
  }
}

template <int G>
__global__ void k_extract_count(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                const double* __restrict__ val, const uint8_t* __restrict__ cls,
                                const int64_t* __restrict__ qidx, int64_t* __restrict__ acnt,
                                double* __restrict__ d, double* __restrict__ b,
                                int64_t* __restrict__ qstate, int general) {
  RowGroups rg = RowGroups::make<G>();
  for (int64_t s = rg.first; warp_has_row<G>(s, n); s += rg.stride) {
    const bool act = s < n && cls[s] == CLS_SQ;
    double diag = 0.0, bs = 0.0, cnt = 0.0;
    if (act) {
      for (int64_t k = rp[s] + rg.lane; k < rp[s + 1]; k += G) {
        const double v = val[k];
        if (v == 0.0) continue;
        const int32_t cc = col[k];
        if ((int64_t)cc == s) {
          diag += v;
        } else {
          const uint8_t kc = cls[cc];
          if (kc == CLS_SQ) cnt += 1.0;
          else if (kc == CLS_S1) bs += v;
        }
      }
    }
    diag = group_sum<G>(diag);
    bs = group_sum<G>(bs);
    cnt = group_sum<G>(cnt);
    if (act && rg.lane == 0) {
      const int64_t i = qidx[s];
      acnt[i] = (int64_t)cnt;
      // chain: d = 1 - A_ii of I - A; general system M x = b: d = M_ii, b given
      d[i] = general ? diag : 1.0 - diag;
      if (!general) b[i] = bs;
      qstate[i] = s;
    }
  }
}

template <int G>
__global__ void k_extract_fill(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                               const double* __restrict__ val, const uint8_t* __restrict__ cls,
                               const int64_t* __restrict__ qidx, const int64_t* __restrict__ arp,
                               int32_t* __restrict__ acol, double* __restrict__ aval, int general) {
  RowGroups rg = RowGroups::make<G>();
  const int wl = threadIdx.x & 31;
  const unsigned gmask = G == 32 ? FULL : (((1u << G) - 1u) << (wl & ~(G - 1)));
  const unsigned lt = (1u << wl) - 1u;
  for (int64_t s = rg.first; warp_has_row<G>(s, n); s += rg.stride) {
    const bool act = s < n && cls[s] == CLS_SQ;
    int64_t lo = 0, hi = 0, out = 0;
    if (act) {
      lo = rp[s];
      hi = rp[s + 1];
      out = arp[qidx[s]];
    }
    const unsigned trips = __reduce_max_sync(FULL, (unsigned)((hi - lo + G - 1) / G));
    for (unsigned t = 0; t < trips; ++t) {
      const int64_t k = lo + (int64_t)t * G + rg.lane;
      bool p = false;
      int32_t cq = 0;
      double v = 0.0;
      if (act && k < hi) {
        v = val[k];
        const int32_t cc = col[k];
        p = v != 0.0 && (int64_t)cc != s && cls[cc] == CLS_SQ;
        if (p) cq = (int32_t)qidx[cc];
      }
      const unsigned mine = __ballot_sync(FULL, p) & gmask;
      if (p) {
        const int64_t pos = out + __popc(mine & lt);
        acol[pos] = cq;
        aval[pos] = general ? -v : v;   // general system: A = -(off-diagonal of M)
      }
      out += __popc(mine);
    }
  }
}

// Jacobi form: Aj_ij = A_ij / d_i, bj_i = b_i / d_i (IEEE division, once per system).
template <int G>
__global__ void k_jform(int64_t nq, const int64_t* __restrict__ rp, const double* __restrict__ av,
                        const double* __restrict__ b, const double* __restrict__ d, double* __restrict__ aj,
                        double* __restrict__ bj) {
  RowGroups rg = RowGroups::make<G>();
  for (int64_t i = rg.first; i < nq; i += rg.stride) {
    const double di = d[i];
    // a row without a self-loop has d_i = 1 exactly and needs no division: on GB300 an FP64
    // division is a long sequence on the narrow FP64 pipe (3.7x the sweep time on sparse rows)
    if (di == 1.0) {
      for (int64_t k = rp[i] + rg.lane; k < rp[i + 1]; k += G) aj[k] = av[k];
      if (rg.lane == 0 && bj) bj[i] = b[i];
    } else {
      for (int64_t k = rp[i] + rg.lane; k < rp[i + 1]; k += G) aj[k] = av[k] / di;
      if (rg.lane == 0 && bj) bj[i] = b[i] / di;
    }
  }
}

template <int G>
static void jform_launch(reach_ctx* c, int64_t nq, const int64_t* rp, const double* av, const double* b,
                         double* aj, double* bj) {
  k_jform<G><<<grid_for(c, (const void*)k_jform<G>, 256, nq * G), 256, 0, c->stream>>>(nq, rp, av, b, c->d, aj, bj);
}

static void jform_dispatch(reach_ctx* c, int g, int64_t nq, const int64_t* rp, const double* av,
                           const double* b, double* aj, double* bj) {
  switch (g) {
    case 2: jform_launch<2>(c, nq, rp, av, b, aj, bj); break;
    case 4: jform_launch<4>(c, nq, rp, av, b, aj, bj); break;
    case 8: jform_launch<8>(c, nq, rp, av, b, aj, bj); break;
    case 16: jform_launch<16>(c, nq, rp, av, b, aj, bj); break;
    default: jform_launch<32>(c, nq, rp, av, b, aj, bj); break;
  }
}


template <int G>
static void extract_launch(reach_ctx* c, int64_t* acnt, int pass) {
  const int grid = grid_for(c, pass == 0 ? (const void*)k_extract_count<G> : (const void*)k_extract_fill<G>,
                            256, c->n * G);
  if (pass == 0)
    k_extract_count<G><<<grid, 256, 0, c->stream>>>(c->n, c->rowptr, c->col, c->val, c->cls, c->qidx,
                                                    acnt, c->d, c->b, c->qstate, c->general ? 1 : 0);
  else
    k_extract_fill<G><<<grid, 256, 0, c->stream>>>(c->n, c->rowptr, c->col, c->val, c->cls, c->qidx,
                                                   c->a_rowptr, c->a_col, c->a_val, c->general ? 1 : 0);
}

static void extract_dispatch(reach_ctx* c, int g, int64_t* acnt, int pass) {
  switch (g) {
    case 2: extract_launch<2>(c, acnt, pass); break;
    case 4: extract_launch<4>(c, acnt, pass); break;
    case 8: extract_launch<8>(c, acnt, pass); break;
    case 16: extract_launch<16>(c, acnt, pass); break;
    default: extract_launch<32>(c, acnt, pass); break;
  }
}

template <typename T>
static cudaError_t dmalloc(T** p, int64_t count) {
  if (*p) {
    cudaFree(*p);
    *p = nullptr;
  }
  if (count <= 0) count = 1;
  return cudaMalloc((void**)p, sizeof(T) * (size_t)count);
}

cudaError_t exclusive_scan_u8(reach_ctx* c, const uint8_t* in, int64_t* out, int64_t n, int64_t* total_dev) {
  return exclusive_scan<uint8_t>(in, out, n, total_dev, reinterpret_cast<int64_t*>(c->part), c->stream);
}

cudaError_t exclusive_scan_u32(reach_ctx* c, const uint32_t* in, int64_t* out, int64_t n) {
  return exclusive_scan<uint32_t>(in, out, n, nullptr, reinterpret_cast<int64_t*>(c->part), c->stream);
}

cudaError_t classify_and_extract(reach_ctx* c, int mode) {
  const int64_t n = c->n, words = (n + 31) >> 5;
  uint8_t* qflag = reinterpret_cast<uint8_t*>(c->queue);   // scratch: n bytes
  k_classify<<<grid_for(c, (const void*)k_classify, 256, n), 256, 0, c->stream>>>(
      n, mode, c->goal, c->vis, c->vis + words, c->cls, qflag);
  return extract_rows(c);
}

// Every state kept as a row (batched solves: the classes differ per right-hand side,
// so the off-diagonal part of P and d = 1 - P_ss are extracted for all states).
cudaError_t extract_all_rows(reach_ctx* c) {
  cudaMemsetAsync(c->cls, CLS_SQ, c->n, c->stream);
  cudaMemsetAsync(c->queue, 1, c->n, c->stream);
  return extract_rows(c);
}

// Scan of the S? flags (bytes in c->queue) into qidx, then A, d, b over those rows.
cudaError_t extract_rows(reach_ctx* c) {
  cudaStream_t s = c->stream;
  const int64_t n = c->n;
  uint8_t* qflag = reinterpret_cast<uint8_t*>(c->queue);
  int64_t* bsum = reinterpret_cast<int64_t*>(c->part);
  int64_t* nq_dev = reinterpret_cast<int64_t*>(c->st);     // scratch word
  exclusive_scan<uint8_t>(qflag, c->qidx, n, nq_dev, bsum, s);
  int64_t nq = 0;
  cudaError_t e = cudaMemcpyAsync(&nq, nq_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  c->n_q = nq;
  // per-row arrays of the system
  if ((e = dmalloc(&c->a_rowptr, nq + 1)) != cudaSuccess) return e;
  if ((e = dmalloc(&c->d, nq)) != cudaSuccess) return e;
  if ((e = dmalloc(&c->b, nq)) != cudaSuccess) return e;
  if ((e = dmalloc(&c->qstate, nq)) != cudaSuccess) return e;
  int64_t* acnt = nullptr;
  if ((e = dmalloc(&acnt, nq)) != cudaSuccess) return e;
  const int g = graph_group(c, n, c->m);
  if (nq > 0) extract_dispatch(c, g, acnt, 0);
  int64_t* mq_dev = reinterpret_cast<int64_t*>(c->st) + 1;
  exclusive_scan<int64_t>(acnt, c->a_rowptr, nq, mq_dev, bsum, s);
  int64_t mq = 0;
  e = cudaMemcpyAsync(&mq, mq_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(acnt);
  if (e != cudaSuccess) return e;
  c->m_q = mq;
  // +8 entries of slack so vector loads of the last row stay inside the allocation
  if ((e = dmalloc(&c->a_col, mq + 8)) != cudaSuccess) return e;
  if ((e = dmalloc(&c->a_val, mq + 8)) != cudaSuccess) return e;
  cudaMemsetAsync(c->a_col + mq, 0, 8 * sizeof(int32_t), s);
  cudaMemsetAsync(c->a_val + mq, 0, 8 * sizeof(double), s);
  if (nq > 0) extract_dispatch(c, g, nullptr, 1);
  // the Jacobi form, the hi/lo split and the transposed system are rebuilt on demand
  if (c->a_jv) { cudaFree(c->a_jv); c->a_jv = nullptr; }
  if (c->bj) { cudaFree(c->bj); c->bj = nullptr; }
  if (c->at_jv) { cudaFree(c->at_jv); c->at_jv = nullptr; }
  if (c->a_hi) { cudaFree(c->a_hi); c->a_hi = nullptr; }
  if (c->a_lo) { cudaFree(c->a_lo); c->a_lo = nullptr; }
  if (c->a_col16) { cudaFree(c->a_col16); c->a_col16 = nullptr; }
  if (c->at_rowptr) { cudaFree(c->at_rowptr); c->at_rowptr = nullptr; }
  if (c->at_col) { cudaFree(c->at_col); c->at_col = nullptr; }
  if (c->at_val) { cudaFree(c->at_val); c->at_val = nullptr; }
  if (c->at_b) { cudaFree(c->at_b); c->at_b = nullptr; }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ mixed-precision split

__global__ void k_split(int64_t m, const double* __restrict__ v, float* __restrict__ hi,
                        float* __restrict__ lo) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double x = v[k];
    const float h = __double2float_rn(x);
    hi[k] = h;
    lo[k] = __double2float_rn(x - (double)h);
  }
}

__global__ void k_narrow(int64_t m, const int32_t* __restrict__ col, uint16_t* __restrict__ col16) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (int64_t)gridDim.x * blockDim.x)
    col16[k] = (uint16_t)col[k];
}

cudaError_t split_hilo(reach_ctx* c) {
  if (c->a_hi && c->a_lo) return cudaSuccess;
  cudaError_t e;
  if ((e = dmalloc(&c->a_hi, c->m_q + 8)) != cudaSuccess) return e;
  if ((e = dmalloc(&c->a_lo, c->m_q + 8)) != cudaSuccess) return e;
  const int64_t mm = c->m_q + 8;   // slack entries are zeros of a_jv
  k_split<<<grid_for(c, (const void*)k_split, 256, mm), 256, 0, c->stream>>>(mm, c->a_jv, c->a_hi, c->a_lo);
  // 16-bit column indices when every S? index fits: 2 bytes less per entry in the sweeps
  if (c->n_q <= 65536 && !c->a_col16) {
    if ((e = dmalloc(&c->a_col16, c->m_q + 8)) != cudaSuccess) return e;
    k_narrow<<<grid_for(c, (const void*)k_narrow, 256, mm), 256, 0, c->stream>>>(mm, c->a_col, c->a_col16);
  }
  return cudaGetLastError();
}

cudaError_t build_jacobi_form(reach_ctx* c) {
  if (c->a_jv && c->bj) return cudaSuccess;
  const int64_t nq = c->n_q, mq = c->m_q;
  cudaError_t e;
  if ((e = dmalloc(&c->a_jv, mq + 8)) != cudaSuccess) return e;
  if ((e = dmalloc(&c->bj, nq)) != cudaSuccess) return e;
  cudaMemsetAsync(c->a_jv + mq, 0, 8 * sizeof(double), c->stream);
  if (nq > 0) jform_dispatch(c, graph_group(c, nq, mq), nq, c->a_rowptr, c->a_val, c->b, c->a_jv, c->bj);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ transposed system

__global__ void k_tcount(int64_t mq, const int32_t* __restrict__ acol, uint32_t* cnt) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < mq;
       k += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(cnt + acol[k], 1u);
}

template <int G>
__global__ void k_tfill(int64_t nq, const int64_t* __restrict__ arp, const int32_t* __restrict__ acol,
                        const double* __restrict__ aval, uint32_t* cnt, const int64_t* __restrict__ trp,
                        int32_t* __restrict__ tcol, double* __restrict__ tval) {
  RowGroups rg = RowGroups::make<G>();
  for (int64_t i = rg.first; i < nq; i += rg.stride) {
    for (int64_t k = arp[i] + rg.lane; k < arp[i + 1]; k += G) {
      const int32_t j = acol[k];
      const uint32_t pos = atomicSub(cnt + j, 1u) - 1u;
      tcol[trp[j] + pos] = (int32_t)i;
      tval[trp[j] + pos] = aval[k];
    }
  }
}

// Rows of the transposed matrix arrive in atomic order; sorting each by source
// row makes the adjoint's summation order (and so its rounding) reproducible.
__global__ void k_tsort(int64_t nq, const int64_t* __restrict__ trp, int32_t* tcol, double* tval) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nq;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lo = trp[j], hi = trp[j + 1];
    if (hi - lo > 256) continue;
    for (int64_t a = lo + 1; a < hi; ++a) {
      const int32_t kc = tcol[a];
      const double kv = tval[a];
      int64_t p = a - 1;
      while (p >= lo && tcol[p] > kc) {
        tcol[p + 1] = tcol[p];
        tval[p + 1] = tval[p];
        --p;
      }
      tcol[p + 1] = kc;
      tval[p + 1] = kv;
    }
  }
}

cudaError_t build_transposed_system(reach_ctx* c) {
  if (c->at_rowptr) return cudaSuccess;
  cudaStream_t s = c->stream;
  const int64_t nq = c->n_q, mq = c->m_q;
  cudaError_t e;
  if ((e = dmalloc(&c->at_rowptr, nq + 1)) != cudaSuccess) return e;
  if ((e = dmalloc(&c->at_col, mq + 8)) != cudaSuccess) return e;
  if ((e = dmalloc(&c->at_val, mq + 8)) != cudaSuccess) return e;
  if ((e = dmalloc(&c->at_b, nq + 1)) != cudaSuccess) return e;
  cudaMemsetAsync(c->at_col + mq, 0, 8 * sizeof(int32_t), s);
  cudaMemsetAsync(c->at_val + mq, 0, 8 * sizeof(double), s);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(c->queue);
  cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (size_t)(nq > 0 ? nq : 1), s);
  if (mq > 0) k_tcount<<<grid_for(c, (const void*)k_tcount, 256, mq), 256, 0, s>>>(mq, c->a_col, cnt);
  exclusive_scan<uint32_t>(cnt, c->at_rowptr, nq, nullptr, reinterpret_cast<int64_t*>(c->part), s);
  const int g = pick_group(nq, mq);
#define TF(G) k_tfill<G><<<grid_for(c, (const void*)k_tfill<G>, 256, nq * G), 256, 0, s>>>( \
      nq, c->a_rowptr, c->a_col, c->a_val, cnt, c->at_rowptr, c->at_col, c->at_val)
  if (nq > 0) {
    switch (g) {
      case 2: TF(2); break;
      case 4: TF(4); break;
      case 8: TF(8); break;
      case 16: TF(16); break;
      default: TF(32); break;
    }
    k_tsort<<<grid_for(c, (const void*)k_tsort, 128, nq), 128, 0, s>>>(nq, c->at_rowptr, c->at_col, c->at_val);
  }
  // Jacobi form of the transposed system: row j scaled by 1 / d_j
  if ((e = dmalloc(&c->at_jv, mq + 8)) != cudaSuccess) return e;
  cudaMemsetAsync(c->at_jv + mq, 0, 8 * sizeof(double), s);
  if (nq > 0) jform_dispatch(c, g, nq, c->at_rowptr, c->at_val, nullptr, c->at_jv, nullptr);
#undef TF
  return cudaGetLastError();
}

}  // namespace reach
