// Small systems on one thread-block cluster, with the matrix held in shared memory.
//
// Below a few thousand unknowns a Jacobi sweep (§3.1) is a few microseconds of work, and a
// kernel boundary per sweep (about 2.5 us inside a graph) is the cost.  The state spaces
// of §7 (Table 1: 92 to 7647 states) are all in this range.  Here one cluster of 16 CTAs
// runs the whole iteration in one launch:
//   * rows are split over the CTAs by cost (stored entries + 2 per row); each CTA copies its
//     rows of the system (column indices as 16-bit, values, the row's constant term) into
//     its shared memory once;
//   * every CTA keeps a full copy of the iterate in its shared memory, so the gathers of a
//     sweep are shared-memory loads;
//   * after a sweep each CTA stores its rows' new values into every CTA's copy through
//     distributed shared memory, and the hardware cluster barrier (release / acquire)
//     makes them visible: one barrier per sweep, no kernel boundary;
//   * the stopping quantity max|x' - x| is reduced per CTA, and each CTA stores its max
//     into a slot of every CTA (plain distributed-shared-memory stores); after the next
//     barrier every CTA takes the max of the same values, so all CTAs take the same
//     decision.
// There are no waits other than the hardware barrier, and every loop is bounded by
// max_iter.  The FP64 Jacobi form (a5) and the mixed method (a6: FP64 residual with hi +
// lo values, FP32 sweeps, FP64 update) run here with the stopping rules and iteration
// counts of the graph-driven solvers.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdlib>

#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace reach {
namespace {

constexpr int SM_NT = 512;          // threads per CTA
constexpr int SM_CL = 16;           // most CTAs of the cluster (16 is a non-portable size)
constexpr size_t SM_SMEM_MAX = 220 * 1024;   // dynamic part (the static part is below 1 KB)

// Rows of CTA `rank` of `nc`: [first row whose cost reaches rank * C / nc, ...), cost(i) =
// rowptr[i] + 2 i.
RDEV int64_t cost_bound(const int64_t* __restrict__ rp, int64_t nq, int rank, int nc) {
  if (rank <= 0) return 0;
  if (rank >= nc) return nq;
  const int64_t total = rp[nq] + 2 * nq;
  const int64_t target = (total * rank + nc - 1) / nc;
  int64_t lo = 0, hi = nq;            // smallest i with cost(i) >= target
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (rp[mid] + 2 * mid >= target) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

template <typename T>
RDEV T* carve(unsigned char*& p, int64_t count) {
  T* r = reinterpret_cast<T*>(p);
  p += ((size_t)count * sizeof(T) + 15) & ~size_t(15);
  return r;
}

RDEV unsigned long long bits_of(double v) {
  const double a = fabs(v);
  return a != a ? 0x7ff0000000000000ull : (unsigned long long)__double_as_longlong(a);
}

template <int G>
RDEV unsigned long long group_max_bits(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(FULL, v, o);
    v = y > v ? y : v;
  }
  return v;
}

// Cluster-wide max of non-negative bit patterns without atomics: the CTA reduces its
// threads' values, then thread 0 stores the CTA's max into slot [rank] of buffer `buf` in
// every CTA (plain distributed-shared-memory stores).  After the next cluster barrier each
// CTA takes the max of its own copy of the nc slots (cluster_max_read).  Check c uses
// buffer c % 2: a buffer is rewritten two checks later, after every CTA read it.
RDEV void cluster_max_publish(unsigned long long mx, unsigned long long* wbuf,
                              unsigned long long* const (*red)[SM_CL], int buf, int rank, int nc) {
  mx = group_max_bits<32>(mx);
  const int warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if ((threadIdx.x & 31) == 0) wbuf[warp] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned long long v = threadIdx.x < nw ? wbuf[threadIdx.x] : 0ull;
    v = group_max_bits<32>(v);
    if (threadIdx.x < nc) red[buf][threadIdx.x][rank] = v;
  }
}

RDEV double cluster_max_read(const unsigned long long (*loc)[SM_CL], int buf, int nc) {
  unsigned long long b = 0ull;
  for (int r = 0; r < nc; ++r) b = loc[buf][r] > b ? loc[buf][r] : b;
  return __longlong_as_double((long long)(b > 0x7ff0000000000000ull ? 0x7ff0000000000000ull : b));
}

// Row boundaries of every CTA (bnd[0..nc]) into shared memory.
RDEV void cluster_bounds(const int64_t* __restrict__ rp, int64_t nq, int nc, int32_t* bnd) {
  if (threadIdx.x <= (unsigned)nc) bnd[threadIdx.x] = (int32_t)cost_bound(rp, nq, threadIdx.x, nc);
  __syncthreads();
}

// Copies the other CTAs' rows of a replicated vector from their copies into this CTA's:
// warp q pulls the rows of CTA q (coalesced distributed-shared-memory loads, eight in
// flight per lane), so one pass costs about one remote round trip.  (Pushing rows into
// every other CTA with 16-byte remote stores instead measured 1.3x slower per sweep.)
template <typename T>
RDEV void pull_others(T* buf, T* const* rem, const int32_t* bnd, int rank, int nc) {
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (q >= nc || q == rank) return;
  const T* src = rem[q];
  const int32_t lo = bnd[q], hi = bnd[q + 1];
  constexpr int U = 8;
  for (int32_t j = lo + lane; j < hi; j += 32 * U) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = j + 32 * u < hi ? src[j + 32 * u] : T(0);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (j + 32 * u < hi) buf[j + 32 * u] = v[u];
  }
}

// Row dot product over shared-memory data: G lanes per row, each lane taking B = 4 entries
// per trip with every index and value load of the trip issued before its gathers, so a
// row costs one shared-memory round trip per trip and level.  Slots past the row end read
// index 0 with value 0.
template <int G, typename V, typename X, typename ACC>
RDEV ACC srow(int32_t lo, int32_t hi, int lane, const uint16_t* ci, const V* av, const X* x, ACC s) {
  constexpr int B = 4;
  for (int32_t e = lo + lane; e < hi; e += B * G) {
    int c[B];
    V v[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const bool ok = e + u * G < hi;
      c[u] = ok ? (int)ci[e + u * G] : 0;
      v[u] = ok ? av[e + u * G] : V(0);
    }
    X g[B];
#pragma unroll
    for (int u = 0; u < B; ++u) g[u] = x[c[u]];
#pragma unroll
    for (int u = 0; u < B; ++u) s = fma((ACC)v[u], (ACC)g[u], s);
  }
  return s;
}

// ---------------------------------------------------------------- FP64 Jacobi

// Shared-memory layout of one CTA: xs[0], xs[1] (full iterate copies, nq each), then its
// own rows: av (Jacobi-form values), ci (columns), rp (row starts, own rows + 1), bj.
// A sweep reads the full copy xs[cur] and writes its own rows of xs[cur ^ 1], locally;
// the next sweep first pulls the other CTAs' rows of that buffer.  A CTA overwrites its
// rows of a buffer only one barrier after every CTA has pulled them.
template <int G>
__global__ void __launch_bounds__(SM_NT, 1) k_small_jacobi(int64_t nq, const int64_t* __restrict__ arp,
                                                           const int32_t* __restrict__ acol,
                                                           const double* __restrict__ ajv,
                                                           const double* __restrict__ bjv, double* x,
                                                           int k, SolveState* st) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long red[2][SM_CL];                 // per-rank maxima, two buffers
  __shared__ unsigned long long* redrem[2][SM_CL];              // the same slots in every CTA
  __shared__ unsigned long long wbuf[SM_NT / 32];
  __shared__ double* xrem[2][SM_CL];
  __shared__ int32_t bnd[SM_CL + 1];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), nc = (int)cl.num_blocks();
  cluster_bounds(arp, nq, nc, bnd);
  const int64_t r0 = bnd[rank], r1 = bnd[rank + 1];
  const int64_t nr = r1 - r0, e0 = arp[r0], ne = arp[r1] - e0;
  unsigned char* p = smem;
  double* xs[2];
  xs[0] = carve<double>(p, nq);
  xs[1] = carve<double>(p, nq);
  double* av = carve<double>(p, ne);
  uint16_t* ci = carve<uint16_t>(p, ne);
  int32_t* rp = carve<int32_t>(p, nr + 1);
  double* bj = carve<double>(p, nr);
  for (int64_t j = threadIdx.x; j < nq; j += blockDim.x) xs[0][j] = x[j];
  for (int64_t e = threadIdx.x; e < ne; e += blockDim.x) {
    av[e] = ajv[e0 + e];
    ci[e] = (uint16_t)acol[e0 + e];
  }
  for (int64_t i = threadIdx.x; i <= nr; i += blockDim.x) rp[i] = (int32_t)(arp[r0 + i] - e0);
  for (int64_t i = threadIdx.x; i < nr; i += blockDim.x) bj[i] = bjv[r0 + i];
  if (threadIdx.x < 2 * SM_CL) {
    const int b = threadIdx.x / SM_CL, r = threadIdx.x % SM_CL;
    xrem[b][r] = r < nc ? cl.map_shared_rank(xs[b], r) : nullptr;
    redrem[b][r] = r < nc ? cl.map_shared_rank(&red[b][0], r) : nullptr;
    red[b][r] = 0ull;
  }
  cl.sync();
  const double eps = st->eps;
  const int64_t max_iter = st->max_iter;
  const int lane = threadIdx.x & (G - 1);
  const int64_t grp = threadIdx.x / G, ngrp = blockDim.x / G;
  int cur = 0;
  int64_t it = 0;
  int32_t status = REACH_ENOTCONV;
  double last = 0.0;
  // groups of k sweeps, the last of each checked (the graph solver's rule)
  for (int64_t c = 0;; ++c) {
    for (int j = 0; j < k; ++j) {
      const bool check = j == k - 1;
      if (c > 0 || j > 0) {      // the first sweep reads the start vector every CTA loaded
        pull_others(xs[cur], xrem[cur], bnd, rank, nc);
        __syncthreads();
      }
      const double* xa = xs[cur];
      double* xn = xs[cur ^ 1];
      unsigned long long mx = 0ull;
      for (int64_t base = 0; base < nr; base += ngrp) {
        const int64_t i = base + grp;
        double s = 0.0;
        if (i < nr) s = srow<G>(rp[i], rp[i + 1], lane, ci, av, xa, s);
        s = group_sum<G>(s);
        if (i < nr && lane == 0) {
          const double xv = bj[i] + s;
          if (check) {
            const unsigned long long b = bits_of(xv - xa[r0 + i]);
            mx = b > mx ? b : mx;
          }
          xn[r0 + i] = xv;
        }
      }
      if (check) cluster_max_publish(mx, wbuf, redrem, (int)(c & 1), rank, nc);
      cl.sync();   // every CTA's rows of xs[cur ^ 1] are written; the maxima are in
      cur ^= 1;
    }
    it += k;
    last = cluster_max_read(red, (int)(c & 1), nc);
    if (last < eps) {
      status = REACH_OK;
      break;
    }
    if (it >= max_iter) break;
  }
  for (int64_t i = threadIdx.x; i < nr; i += blockDim.x) x[r0 + i] = xs[cur][r0 + i];
  if (rank == 0 && threadIdx.x == 0) {
    st->iter = it;
    st->last = last;
    st->status = status;
    st->done = 1;
  }
  cl.sync();   // no CTA leaves while others may still read its shared memory
}

// ---------------------------------------------------------------- mixed precision

// Shared-memory layout: ds[0], ds[1] (FP32 corrections, nq each), x (FP64, nq), xf (FP32
// copy of x, nq), then own rows: hi, lo (FP32 values), ci, rp, bj (FP64), r (FP32
// residual).  One period: pull x and xf; FP64 residual r = bj + Aj x - x of own rows (also
// the first correction d_0, into own rows of ds[1]); k - 1 FP32 sweeps d_j = r + Aj_hi
// d_{j-1}, each pulling the other rows of d_{j-1} first; the last sweep adds its d straight
// into own rows of x and xf.  One cluster barrier per step.
template <int G>
__global__ void __launch_bounds__(SM_NT, 1) k_small_mixed(int64_t nq, const int64_t* __restrict__ arp,
                                                          const int32_t* __restrict__ acol,
                                                          const float* __restrict__ ahi,
                                                          const float* __restrict__ alo,
                                                          const double* __restrict__ bjv, double* x,
                                                          int k, SolveState* st) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long red[2][SM_CL];
  __shared__ unsigned long long* redrem[2][SM_CL];
  __shared__ unsigned long long wbuf[SM_NT / 32];
  __shared__ float* drem[2][SM_CL];
  __shared__ double* xrem[SM_CL];
  __shared__ float* xfrem[SM_CL];
  __shared__ int32_t bnd[SM_CL + 1];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), nc = (int)cl.num_blocks();
  cluster_bounds(arp, nq, nc, bnd);
  const int64_t r0 = bnd[rank], r1 = bnd[rank + 1];
  const int64_t nr = r1 - r0, e0 = arp[r0], ne = arp[r1] - e0;
  unsigned char* p = smem;
  float* ds[2];
  ds[0] = carve<float>(p, nq);
  ds[1] = carve<float>(p, nq);
  double* xs = carve<double>(p, nq);
  float* xfs = carve<float>(p, nq);
  float* hi = carve<float>(p, ne);
  float* lo = carve<float>(p, ne);
  uint16_t* ci = carve<uint16_t>(p, ne);
  int32_t* rp = carve<int32_t>(p, nr + 1);
  double* bj = carve<double>(p, nr);
  float* rr = carve<float>(p, nr);
  for (int64_t j = threadIdx.x; j < nq; j += blockDim.x) {
    const double v = x[j];
    xs[j] = v;
    xfs[j] = (float)v;
  }
  for (int64_t e = threadIdx.x; e < ne; e += blockDim.x) {
    hi[e] = ahi[e0 + e];
    lo[e] = alo[e0 + e];
    ci[e] = (uint16_t)acol[e0 + e];
  }
  for (int64_t i = threadIdx.x; i <= nr; i += blockDim.x) rp[i] = (int32_t)(arp[r0 + i] - e0);
  for (int64_t i = threadIdx.x; i < nr; i += blockDim.x) bj[i] = bjv[r0 + i];
  if (threadIdx.x < SM_CL) {
    const int r = threadIdx.x;
    drem[0][r] = r < nc ? cl.map_shared_rank(ds[0], r) : nullptr;
    drem[1][r] = r < nc ? cl.map_shared_rank(ds[1], r) : nullptr;
    xrem[r] = r < nc ? cl.map_shared_rank(xs, r) : nullptr;
    xfrem[r] = r < nc ? cl.map_shared_rank(xfs, r) : nullptr;
    redrem[0][r] = r < nc ? cl.map_shared_rank(&red[0][0], r) : nullptr;
    redrem[1][r] = r < nc ? cl.map_shared_rank(&red[1][0], r) : nullptr;
    red[0][r] = red[1][r] = 0ull;
  }
  cl.sync();
  const double eps = st->eps;
  const int64_t max_iter = st->max_iter;
  const int lane = threadIdx.x & (G - 1);
  const int64_t grp = threadIdx.x / G, ngrp = blockDim.x / G;
  int64_t it = 0, refinements = 0;
  int32_t status = REACH_ENOTCONV;
  double last = 0.0;
  for (int64_t t = 0;; ++t) {
    if (t > 0) {                 // the first residual reads the start vector every CTA loaded
      pull_others(xs, xrem, bnd, rank, nc);
      pull_others(xfs, xfrem, bnd, rank, nc);
      __syncthreads();
    }
    unsigned long long mx = 0ull;
    for (int64_t base = 0; base < nr; base += ngrp) {
      const int64_t i = base + grp;
      double s = 0.0;
      float sl = 0.0f;
      if (i < nr) {
        s = srow<G>(rp[i], rp[i + 1], lane, ci, hi, xs, s);
        sl = srow<G>(rp[i], rp[i + 1], lane, ci, lo, xfs, sl);
      }
      s = group_sum<G>(s);
      sl = group_sum<G>(sl);
      if (i < nr && lane == 0) {
        const double r = ((bj[i] + s) + (double)sl) - xs[r0 + i];
        const float rf = __double2float_rn(r);
        mx = bits_of(r) > mx ? bits_of(r) : mx;
        rr[i] = rf;
        ds[1][r0 + i] = rf;
      }
    }
    cluster_max_publish(mx, wbuf, redrem, (int)(t & 1), rank, nc);
    cl.sync();
    last = cluster_max_read(red, (int)(t & 1), nc);
    // the stopping rule and iteration count of the graph-driven mixed solve
    ++refinements;
    ++it;
    if (last < eps) {
      status = REACH_OK;
      break;
    }
    if (it + (k - 1) > max_iter) break;
    it += k - 1;
    // k - 1 FP32 sweeps: ds[1] -> ds[0] -> ds[1] ...; the last (k even: into ds[0]) updates x
    for (int j = 1; j < k; ++j) {
      const int src = j & 1, dst = src ^ 1;
      pull_others(ds[src], drem[src], bnd, rank, nc);
      __syncthreads();
      const float* din = ds[src];
      const bool final_sweep = j == k - 1;
      for (int64_t base = 0; base < nr; base += ngrp) {
        const int64_t i = base + grp;
        float s = 0.0f;
        if (i < nr) s = srow<G>(rp[i], rp[i + 1], lane, ci, hi, din, s);
        s = group_sum<G>(s);
        if (i < nr && lane == 0) {
          const float v = rr[i] + s;
          if (final_sweep) {
            const double xv = xs[r0 + i] + (double)v;   // x += d in FP64
            xs[r0 + i] = xv;
            xfs[r0 + i] = (float)xv;
          } else {
            ds[dst][r0 + i] = v;
          }
        }
      }
      cl.sync();
    }
  }
  for (int64_t i = threadIdx.x; i < nr; i += blockDim.x) x[r0 + i] = xs[r0 + i];
  if (rank == 0 && threadIdx.x == 0) {
    st->iter = it;
    st->last = last;
    st->status = status;
    st->refinements = (int32_t)refinements;
    st->done = 1;
  }
  cl.sync();
}

// Largest rows and entries any CTA of an nc-CTA split gets (the kernels' own cost split).
__global__ void k_small_extents(const int64_t* __restrict__ rp, int64_t nq, int nc, int64_t* out) {
  if (threadIdx.x != 0) return;
  int64_t rmax = 0, emax = 0;
  for (int r = 0; r < nc; ++r) {
    const int64_t a = cost_bound(rp, nq, r, nc), b = cost_bound(rp, nq, r + 1, nc);
    rmax = b - a > rmax ? b - a : rmax;
    emax = rp[b] - rp[a] > emax ? rp[b] - rp[a] : emax;
  }
  out[0] = rmax;
  out[1] = emax;
}

// Bytes of shared memory per CTA for a system of nq rows when no CTA gets more than rcap
// rows and ecap entries.
size_t small_smem(bool mixed, int64_t nq, int64_t ecap, int64_t rcap) {
  auto al = [](size_t b) { return (b + 15) & ~size_t(15); };
  if (mixed)
    return 2 * al(4 * nq) + al(8 * nq) + al(4 * nq) + 2 * al(4 * ecap) + al(2 * ecap) + al(4 * (rcap + 1)) +
           al(8 * rcap) + al(4 * rcap);
  return 2 * al(8 * nq) + al(8 * ecap) + al(2 * ecap) + al(4 * (rcap + 1)) + al(8 * rcap);
}

// Lanes per row: as many as let one pass of the CTA's thread groups cover the rows of the
// fullest CTA, at most a lane per 4 entries of the mean row (a lane's trip), at least 1.
int small_lanes(int64_t nq, int64_t m, int64_t max_rows) {
  const double rows = (double)max_rows;
  const double mean = nq > 0 ? (double)m / (double)nq : 0.0;
  int g = 1;
  while (g < 32 && (double)(SM_NT / (2 * g)) >= rows && 4.0 * (2 * g) <= mean + 3.0) g *= 2;
  return g;
}

template <typename K>
cudaError_t launch_small(reach_ctx* c, K kernel, size_t smem, int nc, void** args) {
  const void* fn = (const void*)kernel;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nc);
  cfg.blockDim = dim3(SM_NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = nc;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  // a cluster that the device cannot place is not launched: the caller falls back
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg) != cudaSuccess || clusters < 1) {
    cudaGetLastError();
    return cudaErrorNotSupported;
  }
  return cudaLaunchKernelExC(&cfg, fn, args);
}

// REACH_SMALL=0: never take the cluster; REACH_SMALL=1: whenever the system fits (also FP64
// Jacobi above its entry limit); unset: the measured choice below.
int small_mode() {
  const char* v = std::getenv("REACH_SMALL");
  if (v && v[0] == '0') return 0;
  if (v && v[0] == '1') return 1;
  return 2;
}
bool small_enabled() { return small_mode() != 0; }

// Rows and entries per CTA of every cluster size, measured once per system (c->small_ext,
// cleared when the system changes).  Returns false when the measurement failed.
bool small_extents(reach_ctx* c) {
  if (c->small_ext[0][0] >= 0) return true;
  int64_t* dev = reinterpret_cast<int64_t*>(c->part);
  for (int i = 0, nc = 1; nc <= SM_CL; ++i, nc *= 2) {
    k_small_extents<<<1, 32, 0, c->stream>>>(c->a_rowptr, c->n_q, nc, dev + 2 * i);
  }
  int64_t h[10];
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, dev, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  for (int i = 0; i < 5; ++i) {
    c->small_ext[i][0] = h[2 * i];
    c->small_ext[i][1] = h[2 * i + 1];
  }
  return true;
}

// CTAs of the cluster for this system: one CTA (only its own barrier) when a thread per row
// covers the whole system, else 16, if the shared memory holds it; else 0 (no cluster:
// 16-bit columns and 220 KB per CTA are the limits).  Measured per sweep of the mixed method:
// 92 states 1.04 -> 0.74 us and 313 states 1.11 -> 0.91 us with one CTA instead of 16; with 2
// to 8 CTAs the larger systems were slower than with 16 (667 states: 1.29 against 1.10 us on
// 2 CTAs; 4096 states: 3.1 against 2.3 us on 8), the work per CTA outweighing the barrier.
int small_cluster(reach_ctx* c, bool mixed) {
  if (!small_enabled() || c->n_q < 1 || c->n_q > 65536) return 0;
  if (!small_extents(c)) return 0;
  if (c->small_ext[0][0] <= SM_NT && small_smem(mixed, c->n_q, c->small_ext[0][1], c->small_ext[0][0]) <= SM_SMEM_MAX)
    return 1;
  return small_smem(mixed, c->n_q, c->small_ext[4][1], c->small_ext[4][0]) <= SM_SMEM_MAX ? SM_CL : 0;
}

int small_index(int nc) { return nc >= 16 ? 4 : nc >= 8 ? 3 : nc >= 4 ? 2 : nc >= 2 ? 1 : 0; }

bool small_fits(reach_ctx* c, bool mixed) { return small_cluster(c, mixed) > 0; }

}  // namespace

// FP64 Jacobi takes the cluster only up to this many stored entries: an SM of GB300
// completes two FP64 lanes per clock, so the FP64 work of 16 SMs outgrows the kernel
// boundary it saves.  Measured per sweep (cluster against graph): 92 states / 211 entries
// 1.4 against 3.2 us, 3647 / 7293 2.5 against 3.6 us, 7647 / 15293 4.1 against 3.7 us,
// 4096 / 64K 3.6 against 2.9 us.  The mixed method's FP32 sweeps stay cheap on 16 SMs:
// 2.3 against 3.3 us per sweep at 4096 / 64K, so it takes the cluster whenever it fits.
constexpr int64_t SMALL_FP64_MAX_ENTRIES = 10240;

bool small_system(reach_ctx* c, int method) {
  if (c->general || c->tune.g != 0) return false;   // a forced row mapping keeps the graph solvers
  if (method == REACH_JACOBI_FP64)
    return (small_mode() == 1 || c->m_q <= SMALL_FP64_MAX_ENTRIES) && small_fits(c, false);
  if (method == REACH_JACOBI_MIXED) return small_fits(c, true);
  return false;
}

#define SMALL_DISPATCH(G, FN, ...)                 \
  switch (G) {                                    \
    case 1: FN<1>(__VA_ARGS__); break;            \
    case 2: FN<2>(__VA_ARGS__); break;            \
    case 4: FN<4>(__VA_ARGS__); break;            \
    case 8: FN<8>(__VA_ARGS__); break;            \
    case 16: FN<16>(__VA_ARGS__); break;          \
    default: FN<32>(__VA_ARGS__); break;          \
  }

template <int G>
static cudaError_t run_small_jacobi(reach_ctx* c, int k, int nc, cudaError_t* out) {
  int64_t nq = c->n_q;
  const int i = small_index(nc);
  const size_t smem = small_smem(false, c->n_q, c->small_ext[i][1], c->small_ext[i][0]);
  void* args[] = {&nq, &c->a_rowptr, &c->a_col, &c->a_jv, &c->bj, &c->x, &k, &c->st};
  *out = launch_small(c, k_small_jacobi<G>, smem, nc, args);
  return *out;
}

template <int G>
static cudaError_t run_small_mixed(reach_ctx* c, int k, int nc, cudaError_t* out) {
  int64_t nq = c->n_q;
  const int i = small_index(nc);
  const size_t smem = small_smem(true, c->n_q, c->small_ext[i][1], c->small_ext[i][0]);
  void* args[] = {&nq, &c->a_rowptr, &c->a_col, &c->a_hi, &c->a_lo, &c->bj, &c->x, &k, &c->st};
  *out = launch_small(c, k_small_mixed<G>, smem, nc, args);
  return *out;
}

// The whole FP64 Jacobi or mixed solve of a small system in one cluster launch.  c->x holds
// the start vector and receives the result; the solve state gets the iteration count, the
// last stopping quantity and the status.  The caller reports the residual afterwards.
// cudaErrorNotSupported (nothing launched): the device cannot place the cluster.
cudaError_t solve_small(reach_ctx* c, int method, int k) {
  cudaError_t e = cudaSuccess;
  const int nc = small_cluster(c, method == REACH_JACOBI_MIXED);
  if (nc < 1) return cudaErrorNotSupported;
  const int g = small_lanes(c->n_q, c->m_q, c->small_ext[small_index(nc)][0]);
  if (method == REACH_JACOBI_MIXED) {
    SMALL_DISPATCH(g, run_small_mixed, c, k, nc, &e);
  } else {
    SMALL_DISPATCH(g, run_small_jacobi, c, k, nc, &e);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

}  // namespace reach
