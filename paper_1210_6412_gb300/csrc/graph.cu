// Graph precompute of §2.2-§2.3 on the device: input validation, the reversed
// underlying digraph, backward breadth-first search for S=0 and S=1, the
// partition, and extraction of A (off-diagonal), d = 1 - A_ii and b over S?.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <utility>

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
  const int lane = threadIdx.x & 31;
  // a warp takes 32 consecutive words and reserves its queue slots with one atomic
  for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; w0 < words;
       w0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t w = w0 + lane;
    uint32_t bits = 0, blocked = 0;
    if (w < words) {
      for (int j = 0; j < 32; ++j) {
        int64_t s = w * 32 + j;
        if (s >= n) break;
        bool src = kind == 0 ? goal[s] != 0 : !bit_of(other, s);
        if (src) bits |= 1u << j;
        else if (avoid_goal && goal[s]) blocked |= 1u << j;
      }
      vis[w] = bits | blocked;
    }
    const uint32_t nb = (uint32_t)__popc(bits);
    uint32_t inc = nb;   // inclusive scan of the warp's source counts
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += y;
    }
    uint32_t base = 0;
    if (lane == 31 && inc) base = atomicAdd(&st->count[0], inc);
    base = __shfl_sync(FULL, base, 31) + inc - nb;
    for (int j = 0; j < 32; ++j)
      if (bits & (1u << j)) q0[base++] = (int32_t)(w * 32 + j);
  }
}

template <int G>
__global__ void k_bfs_level(const int64_t* __restrict__ trp, const int32_t* __restrict__ tcol,
                            uint32_t* vis, int32_t* qa, int32_t* qb, BfsState* st, unsigned* ticket,
                            double mean_deg, double pull_edges, cudaGraphConditionalHandle h, int use_cond) {
  const int L = st->level;
  const int cur = L % 3, nxt = (L + 1) % 3;
  const uint32_t cnt = st->count[cur];
  if (cnt == 0) {  // the search already ended (in the cluster kernel of this body)
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
    return;
  }
  if ((double)cnt * mean_deg > pull_edges) return;   // a wide level: k_bfs_pull's
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
static void launch_level(reach_ctx* c, int grid, uint32_t* vis, double pull_edges,
                         cudaGraphConditionalHandle h, int use_cond, cudaStream_t s) {
  const double mean_deg = c->n > 0 ? std::max(1.0, (double)c->m / (double)c->n) : 1.0;
  k_bfs_level<G><<<grid, 256, 0, s>>>(c->t_rowptr, c->t_col, vis, c->queue, c->queue + c->n, c->bfs,
                                      c->ticket, mean_deg, pull_edges, h, use_cond);
}

// One level of the backward search computed from the other end (bottom-up): every state
// not yet marked reads its own successors in P and is marked, and queued, if one of them
// is marked (a blocked goal does not count).  A wide level costs one pass over the
// unmarked states' rows, most of which stop at their first marked successor, against one
// atomic per reversed edge of the frontier top-down; the reversed graph is not read.
// Marks made during the pass may serve later states of the same pass: each is still a
// path to the sources, so the search reaches the same set (§2.2), in fewer levels.
constexpr int PULL_NT = 256;     // threads of a k_bfs_pull block
constexpr int PULL_BUF = 2048;   // marked states a block collects before one queue reservation

template <int G>
__global__ void __launch_bounds__(PULL_NT) k_bfs_pull(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const double* __restrict__ val, const uint8_t* __restrict__ goal, int avoid_goal,
                           uint32_t* vis, int32_t* qa, int32_t* qb, BfsState* st, unsigned* ticket,
                           double mean_deg, double pull_edges, int32_t level_cap,
                           cudaGraphConditionalHandle h, int use_cond) {
  const int L = st->level;
  const int cur = L % 3, nxt = (L + 1) % 3;
  const uint32_t cnt = st->count[cur];
  if (cnt == 0) {   // no sources, or the search ended: the loop must stop here too
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
    return;
  }
  if (!((double)cnt * mean_deg > pull_edges)) return;   // k_bfs_level's
  if (blockIdx.x == 0 && threadIdx.x == 0) st->count[(L + 2) % 3] = 0u;
  int32_t* qn = (L & 1) ? qa : qb;
  // marked states collect in shared memory and reach the queue a buffer at a time: one
  // global atomic per flush instead of one per warp step (a same-address atomic per warp
  // serialised in L2 and bounded the pass)
  constexpr int ROWS = PULL_NT / G;
  __shared__ int32_t sbuf[PULL_BUF];
  __shared__ uint32_t scnt, sbase;
  if (threadIdx.x == 0) scnt = 0u;
  __syncthreads();
  auto flush = [&]() {
    if (threadIdx.x == 0) sbase = scnt ? atomicAdd(&st->count[nxt], scnt) : 0u;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < scnt; i += PULL_NT) qn[sbase + i] = sbuf[i];
    __syncthreads();
    if (threadIdx.x == 0) scnt = 0u;
    __syncthreads();
  };
  const int lane = threadIdx.x & (G - 1);
  const int wl = threadIdx.x & 31;
  const unsigned gmask = G == 32 ? FULL : (((1u << G) - 1u) << (wl & ~(G - 1)));
  for (int64_t s0 = (int64_t)blockIdx.x * ROWS; s0 < n; s0 += (int64_t)gridDim.x * ROWS) {
    const int64_t s = s0 + threadIdx.x / G;
    bool done = true;
    int64_t k = 0, hi = 0;
    if (s < n && !((__ldcg(vis + (s >> 5)) >> (s & 31)) & 1u)) {
      k = rp[s] + lane;
      hi = rp[s + 1];
      done = false;
    }
    bool hit = false;
    // G successors per trip; the group stops at its first marked one (flags equal in a group)
    while (__any_sync(FULL, !done)) {
      bool m = false;
      if (!done && k < hi) {
        const int32_t cc = col[k];
        m = val[k] > 0.0 && ((__ldcg(vis + (cc >> 5)) >> (cc & 31)) & 1u) && !(avoid_goal && goal[cc]);
      }
      const unsigned b = __ballot_sync(FULL, m) & gmask;
      const unsigned more = __ballot_sync(FULL, !done && k + G < hi) & gmask;
      if (!done) {
        if (b) hit = done = true;
        else if (!more) done = true;
      }
      k += G;
    }
    if (hit && lane == 0) {
      atomicOr(vis + (s >> 5), 1u << (s & 31));
      sbuf[atomicAdd(&scnt, 1u)] = (int32_t)s;
    }
    __syncthreads();
    if (scnt > PULL_BUF - ROWS) flush();   // room for one more step's marks
  }
  flush();
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
    if (use_cond) cudaGraphSetConditional(h, next > 0 && L + 1 < level_cap ? 1u : 0u);
  }
}

template <int G>
static void launch_pull(reach_ctx* c, int avoid_goal, uint32_t* vis, double pull_edges, int32_t level_cap,
                        cudaGraphConditionalHandle h, int use_cond, cudaStream_t s) {
  const double mean_deg = c->n > 0 ? std::max(1.0, (double)c->m / (double)c->n) : 1.0;
  const int grid = grid_for(c, (const void*)k_bfs_pull<G>, PULL_NT, c->n * G);
  k_bfs_pull<G><<<grid, PULL_NT, 0, s>>>(c->n, c->rowptr, c->col, c->val, c->goal, avoid_goal, vis, c->queue,
                                     c->queue + c->n, c->bfs, c->ticket, mean_deg, pull_edges, level_cap,
                                     h, use_cond);
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

// Entries of a reversed row that one lane of k_bfs_cluster_lq handles at a time.
constexpr int BFS_ILP = 8;

// The same level loop with the frontier held in the CTAs' shared memory.  A state found by
// CTA r goes into r's own queue (a shared-memory counter, no atomics in global memory) and
// r stores its queue length into a slot of every CTA before the level's barrier.  After it
// every thread sums the same slots, and the groups of the whole cluster deal the states of
// all queues among themselves, reading them from the owners' shared memory (a CTA that kept
// its own states would soon hold most of the frontier: who finds a state first keeps it).
// While a CTA waits at the barrier it loads the reversed-graph row bounds of the states it
// found and fetches their rows into L2, so the next level mostly reads L2.  A full queue
// spills to the global queue (the level's global counter, as in k_bfs_level), which all
// CTAs expand next level.  On the way out to k_bfs_level the CTAs append their queues to
// the global queue: the search state is the one k_bfs_level keeps.
template <int G>
__global__ void __launch_bounds__(BFS_CL_NT, 1) k_bfs_cluster_lq(const int64_t* __restrict__ trp,
                                                                 const int32_t* __restrict__ tcol, uint32_t* vis,
                                                                 int32_t* qa, int32_t* qb, BfsState* st,
                                                                 double mean_deg, double max_edges,
                                                                 int64_t max_levels, uint32_t cap) {
  extern __shared__ int32_t lq[];   // [2][cap]: the queues of even and odd levels
  __shared__ uint32_t lcnt[2], lspill[2];
  // [level parity][CTA]: every CTA's queue length (low word) and spilled states (high word)
  __shared__ unsigned long long pub[2][16];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), nb = (int)cl.num_blocks();
  const int t = threadIdx.x, lane = t & (G - 1);
  const int64_t ctid = (int64_t)rank * blockDim.x + t;
  const int64_t cgroups = (int64_t)nb * blockDim.x / G;
  if (t < 2) lcnt[t] = lspill[t] = 0u;
  if (t < 32) pub[t >> 4][t & 15] = 0ull;
  cl.sync();   // every slot is zero before any CTA publishes into it
  int L = *(volatile int32_t*)&st->level;
  uint32_t spill = 0, local_tot = 0;
  bool wide = false;
  for (int64_t it = 0;; ++it) {
    const int cur = L % 3, nxt = (L + 1) % 3, p = L & 1;
    // the same values in every thread: written before the last barrier, not since.  The
    // spilled states of a level are counted by the CTAs too; only the frontier this launch
    // starts from is known from the global count alone.
    local_tot = 0;
    uint32_t pspill = 0;
    for (int r = 0; r < nb; ++r) {
      const unsigned long long w = *(volatile unsigned long long*)&pub[p][r];
      local_tot += (uint32_t)w;
      pspill += (uint32_t)(w >> 32);
    }
    spill = it == 0 ? *(volatile uint32_t*)&st->count[cur] : pspill;
    const uint32_t tot = spill + local_tot;
    if (tot == 0) break;
    if (it >= max_levels || (double)tot * mean_deg > max_edges) {
      wide = true;
      break;
    }
    // the global count of level L - 1, read by every thread before the last barrier
    if (ctid == 0) st->count[(L + 2) % 3] = 0u;
    const int32_t* qc = (L & 1) ? qb : qa;
    int32_t* qn = (L & 1) ? qa : qb;
    int32_t* lc = lq + (size_t)p * cap;
    int32_t* ln = lq + (size_t)(p ^ 1) * cap;
    uint32_t* ncnt = &lcnt[p ^ 1];
    uint32_t* nspill = &lspill[p ^ 1];
    for (int64_t i = ctid / G; i < (int64_t)tot; i += cgroups) {
      int32_t v;
      if (i < (int64_t)local_tot) {   // entry i of the CTAs' queues taken in rank order
        uint32_t o = 0, acc = 0;
        while ((uint32_t)i >= acc + (uint32_t)*(volatile unsigned long long*)&pub[p][o])
          acc += (uint32_t)*(volatile unsigned long long*)&pub[p][o++];
        v = *cl.map_shared_rank(lc + ((uint32_t)i - acc), o);
      } else {
        v = __ldcg(qc + (i - (int64_t)local_tot));
      }
      const int64_t lo = trp[v], hi = trp[v + 1];
      // BFS_ILP entries per lane at a time: their loads, then their atomics, are issued
      // together, so a long row costs about one round trip of each instead of one per entry
      for (int64_t k0 = lo + lane; k0 < hi; k0 += (int64_t)G * BFS_ILP) {
        int32_t u[BFS_ILP];
        uint32_t old[BFS_ILP];
#pragma unroll
        for (int j = 0; j < BFS_ILP; ++j) u[j] = k0 + (int64_t)j * G < hi ? tcol[k0 + (int64_t)j * G] : -1;
#pragma unroll
        for (int j = 0; j < BFS_ILP; ++j) old[j] = u[j] >= 0 ? atomicOr(vis + (u[j] >> 5), 1u << (u[j] & 31)) : ~0u;
#pragma unroll
        for (int j = 0; j < BFS_ILP; ++j) {
          if (!((old[j] >> (u[j] & 31)) & 1u)) {
            cg::coalesced_group g = cg::coalesced_threads();
            uint32_t base = 0;
            if (g.thread_rank() == 0) base = atomicAdd(ncnt, (uint32_t)g.size());
            const uint32_t slot = g.shfl(base, 0) + g.thread_rank();
            if (slot < cap) ln[slot] = u[j];
            else {
              __stcg(qn + agg_inc(&st->count[nxt]), u[j]);
              atomicAdd(nspill, 1u);
            }
            prefetch_l2(trp + u[j]);   // its row bounds are read before the next level
          }
        }
      }
    }
    __syncthreads();   // this CTA's expansion is done: its next queue is final
    const uint32_t nmine = min(*ncnt, cap);
    if (t == 0) {
      const unsigned long long w = ((unsigned long long)*nspill << 32) | nmine;
      for (int r = 0; r < nb; ++r) *cl.map_shared_rank(&pub[p ^ 1][rank], r) = w;
      lcnt[p] = lspill[p] = 0u;   // the counters of the level just expanded serve level L + 2
    }
    auto token = cl.barrier_arrive();   // the next frontier is complete, the lengths published
    // meanwhile the rows of this CTA's next states into L2 (hints: nothing waits for them)
    for (uint32_t i = t; i < nmine; i += blockDim.x) {
      const int32_t u = ln[i];
      const int64_t lo = trp[u], hi = trp[u + 1];
      if (hi > lo) {
        prefetch_l2(tcol + lo);
        if (((lo ^ (hi - 1)) >> 5) != 0) prefetch_l2(tcol + hi - 1);   // a row across two lines
      }
    }
    cl.barrier_wait(std::move(token));
    ++L;
  }
  if (wide) {
    const int p = L & 1;
    cl.sync();   // every CTA has read the global count of level L before it changes
    uint32_t off = spill;
    for (int r = 0; r < rank; ++r) off += (uint32_t)pub[p][r];
    const uint32_t mine = (uint32_t)pub[p][rank];
    int32_t* qc = (L & 1) ? qb : qa;
    for (uint32_t i = t; i < mine; i += blockDim.x) __stcg(qc + off + i, lq[(size_t)p * cap + i]);
    if (ctid == 0) st->count[L % 3] = spill + local_tot;
  }
  if (ctid == 0) st->level = L;
}

// States per CTA queue of k_bfs_cluster_lq (two queues per CTA: 128 KB of shared memory).
constexpr uint32_t BFS_LQ_CAP = 16384;

// The level loop on the cluster keeps its frontier in shared memory unless REACH_BFS_LQ=0.
static bool bfs_local_queues() {
  const char* e = std::getenv("REACH_BFS_LQ");
  return !(e && e[0] == '0');
}

template <int G>
static const void* bfs_cluster_fn(bool lq) {
  return lq ? (const void*)k_bfs_cluster_lq<G> : (const void*)k_bfs_cluster<G>;
}

static size_t bfs_cluster_smem(bool lq) { return lq ? 2 * sizeof(int32_t) * BFS_LQ_CAP : 0; }

// Cluster size the device can host for the cluster level loop (16, else 8, else 0 = none).
template <int G>
static int bfs_cluster_size(reach_ctx* c, bool lq) {
  const void* fn = bfs_cluster_fn<G>(lq);
  if (lq && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bfs_cluster_smem(lq)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  for (int cs : {16, 8}) {
    if (cs > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(BFS_CL_NT);
    cfg.dynamicSmemBytes = bfs_cluster_smem(lq);
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
static cudaError_t launch_cluster_levels(reach_ctx* c, int cs, bool lq, int avoid_goal, uint32_t* vis,
                                         cudaStream_t s) {
  const void* fn = bfs_cluster_fn<G>(lq);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(BFS_CL_NT);
  cfg.dynamicSmemBytes = bfs_cluster_smem(lq);
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
  uint32_t cap = BFS_LQ_CAP;
  if (lq) {
    // the opt-in shared memory limit is an attribute of the device in use: set per launch
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bfs_cluster_smem(lq));
    if (e != cudaSuccess) return e;
    void* args[] = {&trp, &tcol, &vis, &qa, &qb, &st, &mean_deg, &max_edges, &max_levels, &cap};
    return cudaLaunchKernelExC(&cfg, fn, args);
  }
  void* args[] = {&trp, &tcol, &goal, &avoid_goal, &vis, &qa, &qb, &st, &mean_deg, &max_edges, &max_levels};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

static int cluster_dispatch_size(reach_ctx* c, int g, bool lq) {
  switch (g) {
    case 2: return bfs_cluster_size<2>(c, lq);
    case 4: return bfs_cluster_size<4>(c, lq);
    case 8: return bfs_cluster_size<8>(c, lq);
    case 16: return bfs_cluster_size<16>(c, lq);
    default: return bfs_cluster_size<32>(c, lq);
  }
}

static cudaError_t cluster_dispatch(reach_ctx* c, int g, int cs, bool lq, int avoid_goal, uint32_t* vis,
                                    cudaStream_t s) {
  switch (g) {
    case 2: return launch_cluster_levels<2>(c, cs, lq, avoid_goal, vis, s);
    case 4: return launch_cluster_levels<4>(c, cs, lq, avoid_goal, vis, s);
    case 8: return launch_cluster_levels<8>(c, cs, lq, avoid_goal, vis, s);
    case 16: return launch_cluster_levels<16>(c, cs, lq, avoid_goal, vis, s);
    default: return launch_cluster_levels<32>(c, cs, lq, avoid_goal, vis, s);
  }
}

static void level_dispatch(reach_ctx* c, int g, int grid, uint32_t* vis, double pull_edges,
                           cudaGraphConditionalHandle h, int use_cond, cudaStream_t s) {
  switch (g) {
    case 2: launch_level<2>(c, grid, vis, pull_edges, h, use_cond, s); break;
    case 4: launch_level<4>(c, grid, vis, pull_edges, h, use_cond, s); break;
    case 8: launch_level<8>(c, grid, vis, pull_edges, h, use_cond, s); break;
    case 16: launch_level<16>(c, grid, vis, pull_edges, h, use_cond, s); break;
    default: launch_level<32>(c, grid, vis, pull_edges, h, use_cond, s); break;
  }
}

static void pull_dispatch(reach_ctx* c, int g, int avoid_goal, uint32_t* vis, double pull_edges,
                          int32_t level_cap, cudaGraphConditionalHandle h, int use_cond, cudaStream_t s) {
  switch (g) {
    case 2: launch_pull<2>(c, avoid_goal, vis, pull_edges, level_cap, h, use_cond, s); break;
    case 4: launch_pull<4>(c, avoid_goal, vis, pull_edges, level_cap, h, use_cond, s); break;
    case 8: launch_pull<8>(c, avoid_goal, vis, pull_edges, level_cap, h, use_cond, s); break;
    case 16: launch_pull<16>(c, avoid_goal, vis, pull_edges, level_cap, h, use_cond, s); break;
    default: launch_pull<32>(c, avoid_goal, vis, pull_edges, level_cap, h, use_cond, s); break;
  }
}

// Runs body(stream, handle, use_cond) until the frontier is empty or level_cap levels are
// done: as a conditional-while graph (the kernels set the condition) or, with host loops,
// with a read of the search state after each body.
template <typename Body>
static cudaError_t run_levels(reach_ctx* c, int64_t level_cap, Body body) {
  cudaStream_t s = c->stream;
  cudaError_t e = cudaSuccess;
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
      cudaGraph_t g = np.conditional.phGraph_out[0];
      e = cudaStreamBeginCaptureToGraph(c->cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
      if (e == cudaSuccess) {
        e = body(c->cap, h, 1);
        const cudaError_t e2 = cudaStreamEndCapture(c->cap, &g);
        if (e == cudaSuccess) e = e2;
      }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    return e;
  }
  BfsState hs;
  for (int64_t it = 0; it <= c->n + 1; ++it) {
    if ((e = body(s, cudaGraphConditionalHandle(), 0)) != cudaSuccess) return e;
    e = cudaMemcpyAsync(&hs, c->bfs, sizeof(hs), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (hs.count[hs.level % 3] == 0 || hs.level >= level_cap) break;
  }
  return cudaGetLastError();
}

// Rows of at least this mean length make the search start bottom-up and without the
// reversed graph: every level is a pass over the unmarked states' rows, which mostly stop
// at their first marked successor.  Such chains are a few levels deep; one still going
// after BFS_DENSE_LEVELS levels starts again with the reversed graph.
constexpr double BFS_DENSE_DEG = 32.0;
constexpr int32_t BFS_DENSE_LEVELS = 8;

// Levels whose frontier has more reversed edges than this run bottom-up (k_bfs_pull).
static double bfs_pull_edges(reach_ctx* c) {
  return std::max(4.0 * BFS_CLUSTER_EDGES, (double)c->m / 64.0);
}

// Backward search from the sources (§2.2).  source_kind 0: GS, marks vis[0..] = "can reach
// GS".  source_kind 1: S=0 (states not marked by the first search), with goal states never
// entered when avoid_goal; marks vis[words..] = "reaches S=0 along a path avoiding GS".
// Narrow levels run on one thread-block cluster, others top-down on the whole GPU over the
// reversed graph, wide ones bottom-up over P (REACH_BFS_PULL=0: never bottom-up).
cudaError_t bfs_backward(reach_ctx* c, int source_kind, bool avoid_goal) {
  const int64_t n = c->n;
  const int64_t words = (n + 31) >> 5;
  uint32_t* vis = c->vis + (source_kind == 0 ? 0 : words);
  const uint32_t* other = c->vis;
  cudaStream_t s = c->stream;
  const int ag = avoid_goal ? 1 : 0;
  const char* pv = std::getenv("REACH_BFS_PULL");
  const bool pull_ok = !(pv && pv[0] == '0');
  const double mean_deg = n > 0 ? std::max(1.0, (double)c->m / (double)n) : 1.0;
  const int gp = graph_group(c, n, c->m);
  auto init = [&]() {
    cudaMemsetAsync(c->bfs, 0, sizeof(BfsState), s);
    cudaMemsetAsync(c->ticket, 0, sizeof(unsigned), s);
    const int ig = grid_for(c, (const void*)k_bfs_init, 256, words);
    k_bfs_init<<<ig, 256, 0, s>>>(n, source_kind, ag, c->goal, other, vis, c->queue, c->bfs);
  };
  cudaError_t e;
  if (pull_ok && mean_deg >= BFS_DENSE_DEG) {
    init();
    e = run_levels(c, BFS_DENSE_LEVELS, [&](cudaStream_t st, cudaGraphConditionalHandle h, int uc) {
      pull_dispatch(c, gp, ag, vis, 0.0, BFS_DENSE_LEVELS, h, uc, st);
      return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
    BfsState hs;
    e = cudaMemcpyAsync(&hs, c->bfs, sizeof(hs), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess || hs.count[hs.level % 3] == 0) return e;
  }
  // the reversed graph (its count pass borrows the queues: before the search starts)
  if (!c->rev_ready) {
    if ((e = build_reverse_pattern(c)) != cudaSuccess) return e;
    c->rev_ready = true;
  }
  init();
  const int g = pick_group(n, c->m);
  const int grid = c->sm_count * 4;
  // small frontiers run on one cluster (0: no cluster launch available, or disabled)
  const char* ev = std::getenv("REACH_BFS_CLUSTER");
  const bool lq = bfs_local_queues();
  const int cs = (ev && ev[0] == '0') ? 0 : cluster_dispatch_size(c, g, lq);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const double pull_edges = pull_ok ? bfs_pull_edges(c) : INFINITY;
  return run_levels(c, INT32_MAX, [&](cudaStream_t st, cudaGraphConditionalHandle h, int uc) {
    cudaError_t le = cs > 0 ? cluster_dispatch(c, g, cs, lq, ag, vis, st) : cudaSuccess;
    level_dispatch(c, g, grid, vis, pull_edges, h, uc, st);
    if (pull_ok) pull_dispatch(c, gp, ag, vis, pull_edges, INT32_MAX, h, uc, st);
    return le != cudaSuccess ? le : cudaGetLastError();
  });
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

// Jacobi form: Aj_ij = A_ij / d_i, bj_i = b_i / d_i (IEEE division, once per system).  With
// kmin it also reduces Varah's row-dominance margin min_i (|d_i| - sum_j |A_ij|) into *kmin
// as an ordered key, the sum rounded upward and the difference downward: a guaranteed lower
// bound of the exact margin, from the same pass over A.
template <int G>
__global__ void k_jform(int64_t nq, const int64_t* __restrict__ rp, const double* __restrict__ av,
                        const double* __restrict__ b, const double* __restrict__ d, double* __restrict__ aj,
                        double* __restrict__ bj, unsigned long long* kmin) {
  RowGroups rg = RowGroups::make<G>();
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  double lo_min = inf;
  for (int64_t i = rg.first; warp_has_row<G>(i, nq); i += rg.stride) {
    double sa = 0.0, di = 1.0;
    if (i < nq) {
      di = d[i];
      // a row without a self-loop has d_i = 1 exactly and needs no division: on GB300 an FP64
      // division is a long sequence on the narrow FP64 pipe (3.7x the sweep time on sparse rows)
      if (di == 1.0) {
        for (int64_t k = rp[i] + rg.lane; k < rp[i + 1]; k += G) {
          const double a = av[k];
          aj[k] = a;
          sa = __dadd_ru(sa, fabs(a));
        }
        if (rg.lane == 0 && bj) bj[i] = b[i];
      } else {
        for (int64_t k = rp[i] + rg.lane; k < rp[i + 1]; k += G) {
          const double a = av[k];
          aj[k] = a / di;
          sa = __dadd_ru(sa, fabs(a));
        }
        if (rg.lane == 0 && bj) bj[i] = b[i] / di;
      }
    }
    if (kmin) {
      sa = group_sum_ru<G>(sa);
      if (i < nq && rg.lane == 0) {
        const double m = __dadd_rd(fabs(di), -sa);
        lo_min = fmin(lo_min, m != m ? -inf : m);
      }
    }
  }
  if (kmin) {
    lo_min = -warp_max(-lo_min);
    if ((threadIdx.x & 31) == 0) atomicMin(kmin, ordered_key(lo_min));
  }
}

template <int G>
static void jform_launch(reach_ctx* c, int64_t nq, const int64_t* rp, const double* av, const double* b,
                         double* aj, double* bj, unsigned long long* kmin) {
  k_jform<G><<<grid_for(c, (const void*)k_jform<G>, 256, nq * G), 256, 0, c->stream>>>(nq, rp, av, b, c->d, aj,
                                                                                      bj, kmin);
}

static void jform_dispatch(reach_ctx* c, int g, int64_t nq, const int64_t* rp, const double* av,
                           const double* b, double* aj, double* bj, unsigned long long* kmin = nullptr) {
  switch (g) {
    case 2: jform_launch<2>(c, nq, rp, av, b, aj, bj, kmin); break;
    case 4: jform_launch<4>(c, nq, rp, av, b, aj, bj, kmin); break;
    case 8: jform_launch<8>(c, nq, rp, av, b, aj, bj, kmin); break;
    case 16: jform_launch<16>(c, nq, rp, av, b, aj, bj, kmin); break;
    default: jform_launch<32>(c, nq, rp, av, b, aj, bj, kmin); break;
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
  c->varah_key = false;
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

// The Jacobi form of the system (§3.1), with Varah's margin of its rows from the same pass.
cudaError_t build_jacobi_form(reach_ctx* c) {
  if (c->a_jv && c->bj) return cudaSuccess;
  const int64_t nq = c->n_q, mq = c->m_q;
  cudaError_t e;
  if ((e = dmalloc(&c->a_jv, mq + 8)) != cudaSuccess) return e;
  if ((e = dmalloc(&c->bj, nq)) != cudaSuccess) return e;
  cudaMemsetAsync(c->a_jv + mq, 0, 8 * sizeof(double), c->stream);
  cudaMemsetAsync(c->keys + VARAH_KEY, 0xff, sizeof(unsigned long long), c->stream);
  if (nq > 0)
    jform_dispatch(c, graph_group(c, nq, mq), nq, c->a_rowptr, c->a_val, c->b, c->a_jv, c->bj, c->keys + VARAH_KEY);
  c->varah_key = true;
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
