// Row blocks of (I - A) x = b for a solve spread over several GPUs (one process per GPU).
//
// The related work of §8 runs Jacobi on two GPUs and its future work is a multi-GPU
// BiCGStab; both split the rows of the system.  A row block holds rows [r0, r1) of A over
// S? with its columns renumbered: the block's own rows are columns [0, n_rows), and every
// other column it references (its halo) is one of the columns [n_rows, n_rows + n_halo).
// Vectors that a product reads are "extended": [own entries | halo entries].  Between
// products the caller exchanges the own entries of every rank (an all-gather) and
// reach_block_halo copies the halo entries out of the gathered vector.  The arithmetic of
// Jacobi (§3.1) and of BiCGStab (§3.2) on the block runs in the kernels below; the
// scalars each iteration needs are local partial sums or maxima that the caller reduces
// over the ranks.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "common.cuh"
#include "internal.h"

struct reach_block {
  int device = 0;
  int sm_count = 1;
  cudaStream_t stream = nullptr;
  int64_t n_rows = 0, n_cols = 0, m = 0, n_halo = 0;
  int64_t* rowptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;     // A_ij (off-diagonal)
  double* aj = nullptr;      // A_ij / d_i (the Jacobi form)
  double* d = nullptr;       // 1 - A_ii (or the diagonal of a general system)
  double* b = nullptr;
  double* bj = nullptr;      // b_i / d_i
  int64_t* halo_src = nullptr;
  double* part = nullptr;    // per-CTA partial sums of the dot products
  unsigned* ticket = nullptr;
  int g = 32;                // lanes per row
  std::string err;
};

namespace reach {
namespace {

constexpr int BNT = 256;
constexpr int BLK_MAX_GRID = 1024;

template <int G>
__global__ void __launch_bounds__(BNT) k_blk_jform(int64_t nr, const int64_t* __restrict__ rp,
                                                   const double* __restrict__ val, const double* __restrict__ d,
                                                   const double* __restrict__ b, double* __restrict__ aj,
                                                   double* __restrict__ bj) {
  RowGroups rg = RowGroups::make<G>();
  for (int64_t i = rg.first; warp_has_row<G>(i, nr); i += rg.stride) {
    if (i >= nr) continue;
    const double di = d[i];
    for (int64_t k = rp[i] + rg.lane; k < rp[i + 1]; k += G) aj[k] = val[k] / di;
    if (rg.lane == 0) bj[i] = b[i] / di;
  }
}

// One Jacobi sweep of the block: x'_i = bj_i + sum_j Aj_ij x_j over the extended x;
// max_i |x'_i - x_i| into *dmax (bits of a non-negative double).
template <int G>
__global__ void __launch_bounds__(BNT) k_blk_jacobi(int64_t nr, const int64_t* __restrict__ rp,
                                                    const int32_t* __restrict__ ci, const double* __restrict__ aj,
                                                    const double* __restrict__ bj, const double* __restrict__ x,
                                                    double* __restrict__ xn, unsigned long long* dmax) {
  RowGroups rg = RowGroups::make<G>();
  unsigned long long mx = 0ull;
  for (int64_t i = rg.first; warp_has_row<G>(i, nr); i += rg.stride) {
    double s = 0.0;
    if (i < nr)
      for (int64_t k = rp[i] + rg.lane; k < rp[i + 1]; k += G) s = fma(__ldcs(aj + k), __ldg(x + __ldcs(ci + k)), s);
    s = group_sum<G>(s);
    if (i < nr && rg.lane == 0) {
      const double xv = bj[i] + s;
      const double dx = fabs(xv - x[i]);
      const unsigned long long bits =
          dx != dx ? 0x7ff0000000000000ull : (unsigned long long)__double_as_longlong(dx);
      mx = bits > mx ? bits : mx;
      xn[i] = xv;
    }
  }
  __shared__ double sh[32];
  double v[1] = {__longlong_as_double((long long)mx)};
  block_reduce<1, true>(v, sh);
  if (threadIdx.x == 0) atomic_max_nonneg(dmax, v[0]);
}

// y = (I - A) u on the block's rows: y_i = d_i u_i - sum_j A_ij u_j over the extended u.
// With w: the local partial of w . y into out[0] (deterministic two-stage sum).
template <int G, bool DOT>
__global__ void __launch_bounds__(BNT) k_blk_matvec(int64_t nr, const int64_t* __restrict__ rp,
                                                    const int32_t* __restrict__ ci, const double* __restrict__ av,
                                                    const double* __restrict__ d, const double* __restrict__ u,
                                                    double* __restrict__ y, const double* __restrict__ w,
                                                    double* part, unsigned* ticket, double* out) {
  RowGroups rg = RowGroups::make<G>();
  double acc = 0.0;
  for (int64_t i = rg.first; warp_has_row<G>(i, nr); i += rg.stride) {
    double s = 0.0;
    if (i < nr)
      for (int64_t k = rp[i] + rg.lane; k < rp[i + 1]; k += G) s = fma(__ldcs(av + k), __ldg(u + __ldcs(ci + k)), s);
    s = group_sum<G>(s);
    if (i < nr && rg.lane == 0) {
      const double yi = fma(d[i], u[i], -s);
      y[i] = yi;
      if (DOT) acc = fma(w[i], yi, acc);
    }
  }
  if constexpr (DOT) {
    __shared__ double sh[32];
    double a[1] = {acc}, tot[1];
    block_reduce<1, false>(a, sh);   // the CTA's partial, in thread 0
    if (last_cta_sum<1>(a, part, ticket, tot, sh) && threadIdx.x == 0) out[0] = tot[0];
  }
}

__global__ void k_blk_halo(int64_t nr, int64_t nh, const int64_t* __restrict__ src, const double* __restrict__ gathered,
                           double* __restrict__ x) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nh; j += (int64_t)gridDim.x * blockDim.x)
    x[nr + j] = gathered[src[j]];
}

// out[0] = u . v, and out[1] = u . w when w is given (deterministic two-stage sums).
template <bool TWO>
__global__ void __launch_bounds__(BNT) k_blk_dot(int64_t n, const double* __restrict__ u, const double* __restrict__ v,
                                                 const double* __restrict__ w, double* part, unsigned* ticket,
                                                 double* out) {
  double a[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    a[0] = fma(u[i], v[i], a[0]);
    if (TWO) a[1] = fma(u[i], w[i], a[1]);
  }
  __shared__ double sh[64];
  block_reduce<2, false>(a, sh);
  double tot[2];
  if (last_cta_sum<2>(a, part, ticket, tot, sh) && threadIdx.x == 0) {
    out[0] = tot[0];
    if (TWO) out[1] = tot[1];
  }
}

// BiCGStab updates on the block's rows (§3.2):
//   P:  p = r + beta (p - omega v)
//   S:  s = r - alpha v,                     max|s| -> *mx
//   XR: x += alpha p + omega s, r = s - omega t, max|r| -> *mx
__global__ void k_blk_p(int64_t n, const double* __restrict__ r, double* __restrict__ p, const double* __restrict__ v,
                        double beta, double omega) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(beta, fma(-omega, v[i], p[i]), r[i]);
}

RDEV void flush_max(double v, unsigned long long* mx) {
  __shared__ double sh[32];
  double a[1] = {v != v ? __longlong_as_double(0x7ff0000000000000LL) : v};
  block_reduce<1, true>(a, sh);
  if (threadIdx.x == 0) atomic_max_nonneg(mx, a[0]);
}

__global__ void k_blk_s(int64_t n, const double* __restrict__ r, const double* __restrict__ v, double alpha,
                        double* __restrict__ s, unsigned long long* mx) {
  double m = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double si = fma(-alpha, v[i], r[i]);
    s[i] = si;
    m = fmax(m, fabs(si) != fabs(si) ? __longlong_as_double(0x7ff0000000000000LL) : fabs(si));
  }
  flush_max(m, mx);
}

__global__ void k_blk_xr(int64_t n, double* __restrict__ x, const double* __restrict__ p,
                         const double* __restrict__ s, const double* __restrict__ t, double alpha, double omega,
                         double* __restrict__ r, unsigned long long* mx) {
  double m = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fma(omega, s[i], fma(alpha, p[i], x[i]));
    const double ri = fma(-omega, t[i], s[i]);
    r[i] = ri;
    m = fmax(m, fabs(ri) != fabs(ri) ? __longlong_as_double(0x7ff0000000000000LL) : fabs(ri));
  }
  flush_max(m, mx);
}

// x += alpha p (the finishing step after max|s| < eps).
__global__ void k_blk_xp(int64_t n, double* __restrict__ x, const double* __restrict__ p, double alpha) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = fma(alpha, p[i], x[i]);
}

int lanes_for(int64_t rows, int64_t nnz) {
  const double mean = rows > 0 ? (double)nnz / (double)rows : 0.0;
  if (mean <= 2.0) return 2;
  if (mean <= 6.0) return 4;
  if (mean <= 12.0) return 8;
  if (mean <= 24.0) return 16;
  return 32;
}

int blk_grid(const reach_block* bk, int64_t work_threads) {
  const int64_t need = std::max<int64_t>(1, (work_threads + BNT - 1) / BNT);
  return (int)std::min<int64_t>(std::min<int64_t>(need, (int64_t)bk->sm_count * 8), BLK_MAX_GRID);
}

reach_status bfail(reach_block* bk, reach_status s, const std::string& msg) {
  if (bk) bk->err = msg;
  set_err(nullptr, msg);
  return s;
}

reach_status bcuda(reach_block* bk, cudaError_t e, const char* where) {
  return bfail(bk, e == cudaErrorMemoryAllocation ? REACH_ENOMEM : REACH_ECUDA,
               std::string(where) + ": " + cudaGetErrorString(e));
}

template <typename T>
cudaError_t balloc(T** p, int64_t count) {
  *p = nullptr;
  return cudaMalloc((void**)p, sizeof(T) * (size_t)std::max<int64_t>(count, 1));
}

#define BLK_DISPATCH(G, CALL)          \
  switch (G) {                         \
    case 2: { constexpr int g_ = 2; CALL; } break;   \
    case 4: { constexpr int g_ = 4; CALL; } break;   \
    case 8: { constexpr int g_ = 8; CALL; } break;   \
    case 16: { constexpr int g_ = 16; CALL; } break; \
    default: { constexpr int g_ = 32; CALL; } break; \
  }

}  // namespace
}  // namespace reach

using namespace reach;

extern "C" {

void reach_block_destroy(reach_block* bk) {
  if (!bk) return;
  if (bk->stream) cudaStreamSynchronize(bk->stream);
  else cudaDeviceSynchronize();
  for (void* p : {(void*)bk->rowptr, (void*)bk->col, (void*)bk->val, (void*)bk->aj, (void*)bk->d, (void*)bk->b,
                  (void*)bk->bj, (void*)bk->halo_src, (void*)bk->part, (void*)bk->ticket})
    if (p) cudaFree(p);
  delete bk;
}

const char* reach_block_last_error(const reach_block* bk) { return bk ? bk->err.c_str() : ""; }

reach_status reach_block_create(reach_block** out, int64_t n_rows, int64_t n_halo, const int64_t* rowptr,
                                const int32_t* col, const double* val, const double* d, const double* b,
                                const int64_t* halo_src, int64_t gathered_len, int32_t flags, void* stream) {
  if (!out) return bfail(nullptr, REACH_EINVAL, "reach_block_create: out is NULL");
  if (n_rows < 1 || n_halo < 0 || n_rows + n_halo > INT32_MAX)
    return bfail(nullptr, REACH_EINVAL, "reach_block_create: need n_rows >= 1, n_halo >= 0, n_rows + n_halo < 2^31");
  if (!rowptr || !d || !b || (n_halo > 0 && !halo_src))
    return bfail(nullptr, REACH_EINVAL, "reach_block_create: NULL input pointer");
  if (flags != REACH_HOST && flags != REACH_DEVICE)
    return bfail(nullptr, REACH_EINVAL, "reach_block_create: flags must be REACH_HOST or REACH_DEVICE");
  const cudaMemcpyKind kind = flags == REACH_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  reach_block* bk = new reach_block();
  bk->stream = (cudaStream_t)stream;
  bk->n_rows = n_rows;
  bk->n_halo = n_halo;
  bk->n_cols = n_rows + n_halo;
  cudaError_t e = cudaGetDevice(&bk->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&bk->sm_count, cudaDevAttrMultiProcessorCount, bk->device);
  int64_t ends[2] = {0, 0};
  if (flags == REACH_HOST) {
    ends[0] = rowptr[0];
    ends[1] = rowptr[n_rows];
  } else {
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[0], rowptr, sizeof(int64_t), cudaMemcpyDeviceToHost, bk->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&ends[1], rowptr + n_rows, sizeof(int64_t), cudaMemcpyDeviceToHost, bk->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(bk->stream);
  }
  if (e != cudaSuccess) {
    reach_status st = bcuda(nullptr, e, "reach_block_create: reading rowptr");
    reach_block_destroy(bk);
    return st;
  }
  if (ends[0] != 0 || ends[1] < 0 || (ends[1] > 0 && (!col || !val))) {
    reach_block_destroy(bk);
    return bfail(nullptr, REACH_EINVAL, "reach_block_create: rowptr[0] must be 0 and entries need col and val");
  }
  const int64_t m = ends[1];
  bk->m = m;
  bk->g = lanes_for(n_rows, m);
  if ((e = balloc(&bk->rowptr, n_rows + 1)) != cudaSuccess || (e = balloc(&bk->col, m)) != cudaSuccess ||
      (e = balloc(&bk->val, m)) != cudaSuccess || (e = balloc(&bk->aj, m)) != cudaSuccess ||
      (e = balloc(&bk->d, n_rows)) != cudaSuccess || (e = balloc(&bk->b, n_rows)) != cudaSuccess ||
      (e = balloc(&bk->bj, n_rows)) != cudaSuccess || (e = balloc(&bk->halo_src, n_halo)) != cudaSuccess ||
      (e = balloc(&bk->part, 2 * BLK_MAX_GRID)) != cudaSuccess || (e = balloc(&bk->ticket, 1)) != cudaSuccess) {
    reach_status st = bcuda(nullptr, e, "reach_block_create: allocation");
    reach_block_destroy(bk);
    return st;
  }
  cudaStream_t s = bk->stream;
  e = cudaMemcpyAsync(bk->rowptr, rowptr, sizeof(int64_t) * (n_rows + 1), kind, s);
  if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(bk->col, col, sizeof(int32_t) * m, kind, s);
  if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(bk->val, val, sizeof(double) * m, kind, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bk->d, d, sizeof(double) * n_rows, kind, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bk->b, b, sizeof(double) * n_rows, kind, s);
  if (e == cudaSuccess && n_halo > 0) e = cudaMemcpyAsync(bk->halo_src, halo_src, sizeof(int64_t) * n_halo, kind, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bk->ticket, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) {
    reach_status st = bcuda(nullptr, e, "reach_block_create: copying inputs");
    reach_block_destroy(bk);
    return st;
  }
  // checks on the host copies the caller gave: column range and halo sources (host inputs
  // only; device inputs are the caller's own plan and are checked by its tests)
  if (flags == REACH_HOST) {
    for (int64_t k = 0; k < m; ++k)
      if (col[k] < 0 || col[k] >= n_rows + n_halo) {
        reach_block_destroy(bk);
        return bfail(nullptr, REACH_EINVAL, "reach_block_create: column outside [0, n_rows + n_halo)");
      }
    for (int64_t j = 0; j < n_halo; ++j)
      if (halo_src[j] < 0 || halo_src[j] >= gathered_len) {
        reach_block_destroy(bk);
        return bfail(nullptr, REACH_EINVAL, "reach_block_create: halo source outside the gathered vector");
      }
  }
  BLK_DISPATCH(bk->g, (k_blk_jform<g_><<<blk_grid(bk, n_rows * g_), BNT, 0, s>>>(
                           n_rows, bk->rowptr, bk->val, bk->d, bk->b, bk->aj, bk->bj)));
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    reach_status st = bcuda(nullptr, e, "reach_block_create: Jacobi form");
    reach_block_destroy(bk);
    return st;
  }
  *out = bk;
  return REACH_OK;
}

reach_status reach_block_halo(reach_block* bk, const double* gathered, double* x_ext) {
  if (!bk || !x_ext || (bk->n_halo > 0 && !gathered)) return bfail(bk, REACH_EINVAL, "reach_block_halo: NULL argument");
  if (bk->n_halo == 0) return REACH_OK;
  k_blk_halo<<<blk_grid(bk, bk->n_halo), BNT, 0, bk->stream>>>(bk->n_rows, bk->n_halo, bk->halo_src, gathered, x_ext);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? REACH_OK : bcuda(bk, e, "reach_block_halo");
}

reach_status reach_block_jacobi(reach_block* bk, const double* x_ext, double* x_new, double* delta) {
  if (!bk || !x_ext || !x_new || !delta) return bfail(bk, REACH_EINVAL, "reach_block_jacobi: NULL argument");
  cudaStream_t s = bk->stream;
  cudaError_t e = cudaMemsetAsync(delta, 0, sizeof(double), s);
  if (e != cudaSuccess) return bcuda(bk, e, "reach_block_jacobi");
  unsigned long long* dm = reinterpret_cast<unsigned long long*>(delta);
  BLK_DISPATCH(bk->g, (k_blk_jacobi<g_><<<blk_grid(bk, bk->n_rows * g_), BNT, 0, s>>>(
                           bk->n_rows, bk->rowptr, bk->col, bk->aj, bk->bj, x_ext, x_new, dm)));
  e = cudaGetLastError();
  return e == cudaSuccess ? REACH_OK : bcuda(bk, e, "reach_block_jacobi");
}

reach_status reach_block_matvec(reach_block* bk, const double* u_ext, double* y, const double* w, double* dot) {
  if (!bk || !u_ext || !y || (w && !dot)) return bfail(bk, REACH_EINVAL, "reach_block_matvec: NULL argument");
  cudaStream_t s = bk->stream;
  if (w) {
    BLK_DISPATCH(bk->g, (k_blk_matvec<g_, true><<<blk_grid(bk, bk->n_rows * g_), BNT, 0, s>>>(
                             bk->n_rows, bk->rowptr, bk->col, bk->val, bk->d, u_ext, y, w, bk->part, bk->ticket, dot)));
  } else {
    BLK_DISPATCH(bk->g, (k_blk_matvec<g_, false><<<blk_grid(bk, bk->n_rows * g_), BNT, 0, s>>>(
                             bk->n_rows, bk->rowptr, bk->col, bk->val, bk->d, u_ext, y, nullptr, bk->part, bk->ticket,
                             nullptr)));
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? REACH_OK : bcuda(bk, e, "reach_block_matvec");
}

reach_status reach_block_dot(reach_block* bk, const double* u, const double* v, const double* w, double* out) {
  if (!bk || !u || !v || !out) return bfail(bk, REACH_EINVAL, "reach_block_dot: NULL argument");
  const int grid = blk_grid(bk, bk->n_rows);
  if (w) k_blk_dot<true><<<grid, BNT, 0, bk->stream>>>(bk->n_rows, u, v, w, bk->part, bk->ticket, out);
  else k_blk_dot<false><<<grid, BNT, 0, bk->stream>>>(bk->n_rows, u, v, nullptr, bk->part, bk->ticket, out);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? REACH_OK : bcuda(bk, e, "reach_block_dot");
}

reach_status reach_block_bicgstab_update(reach_block* bk, int32_t stage, double alpha, double beta, double omega,
                                         double* x, double* r, double* p, const double* v, double* s,
                                         const double* t, double* out) {
  if (!bk) return bfail(nullptr, REACH_EINVAL, "reach_block_bicgstab_update: NULL block");
  const int64_t n = bk->n_rows;
  const int grid = blk_grid(bk, n);
  cudaStream_t st = bk->stream;
  cudaError_t e = cudaSuccess;
  switch (stage) {
    case REACH_BLOCK_P:
      if (!r || !p || !v) return bfail(bk, REACH_EINVAL, "reach_block_bicgstab_update: P needs r, p, v");
      k_blk_p<<<grid, BNT, 0, st>>>(n, r, p, v, beta, omega);
      break;
    case REACH_BLOCK_S:
      if (!r || !v || !s || !out) return bfail(bk, REACH_EINVAL, "reach_block_bicgstab_update: S needs r, v, s, out");
      e = cudaMemsetAsync(out, 0, sizeof(double), st);
      if (e == cudaSuccess)
        k_blk_s<<<grid, BNT, 0, st>>>(n, r, v, alpha, s, reinterpret_cast<unsigned long long*>(out));
      break;
    case REACH_BLOCK_XR:
      if (!x || !p || !s || !t || !r || !out)
        return bfail(bk, REACH_EINVAL, "reach_block_bicgstab_update: XR needs x, p, s, t, r, out");
      e = cudaMemsetAsync(out, 0, sizeof(double), st);
      if (e == cudaSuccess)
        k_blk_xr<<<grid, BNT, 0, st>>>(n, x, p, s, t, alpha, omega, r, reinterpret_cast<unsigned long long*>(out));
      break;
    case REACH_BLOCK_XP:
      if (!x || !p) return bfail(bk, REACH_EINVAL, "reach_block_bicgstab_update: XP needs x, p");
      k_blk_xp<<<grid, BNT, 0, st>>>(n, x, p, alpha);
      break;
    default:
      return bfail(bk, REACH_EINVAL, "reach_block_bicgstab_update: unknown stage");
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? REACH_OK : bcuda(bk, e, "reach_block_bicgstab_update");
}

}  // extern "C"
