// Iterative solvers for (I - A) x = b on S? (§2.3): Jacobi (§3.1) in FP64 and as
// FP32 sweeps with FP64 defect correction, and unpreconditioned BiCGStab (§3.2)
// with FP64 scalars kept on the device.  Every loop runs inside one CUDA graph
// with a conditional while node; the stopping rule is evaluated on the device.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <functional>
#include <mutex>
#include <string>
#include <unordered_map>

#include "common.cuh"
#include "internal.h"

namespace reach {

constexpr int NT = 256;

// ------------------------------------------------------------------ row dot products
// G lanes per row, lane-strided over the row.  V (G == 32 only): 16-byte loads of
// four column indices and the matching values, after a scalar head that aligns the
// start to four entries; the tail is scalar again.  Matrix data is streamed with
// evict-first loads; the gathered vector goes through the read-only cache.

// Column-index loads: int32, or uint16 when every column of the system fits (n? <= 65536).
RDEV int ld_idx(const int32_t* p) { return __ldcs(p); }
RDEV int ld_idx(const uint16_t* p) { return (int)__ldcs(reinterpret_cast<const unsigned short*>(p)); }
RDEV int4 ld_idx4(const int32_t* p) { return __ldcs(reinterpret_cast<const int4*>(p)); }
RDEV int4 ld_idx4(const uint16_t* p) {
  const ushort4 u = __ldcs(reinterpret_cast<const ushort4*>(p));
  return make_int4(u.x, u.y, u.z, u.w);
}

// init: the accumulator's starting value (a row's constant term, so that adding it costs
// no separate FP64 instruction).
template <int G, bool V, typename XF>
RDEV double dot64(int64_t lo, int64_t hi, int lane, const int32_t* __restrict__ ci,
                  const double* __restrict__ av, XF xf, double init = 0.0) {
  double s = init;
  if constexpr (V) {
    int64_t a = (lo + 3) & ~int64_t(3);
    if (a > hi) a = hi;
    const int64_t e = a + ((hi - a) & ~int64_t(3));
    if (lo + lane < a) s = fma(__ldcs(av + lo + lane), xf(__ldcs(ci + lo + lane)), s);
    // four independent FP64 accumulators: the narrow FP64 pipe of GB300 has a long
    // latency, and one dependent chain per lane would leave it waiting
    double s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int64_t k = a + 4 * lane; k < e; k += 4 * G) {
      const int4 c4 = __ldcs(reinterpret_cast<const int4*>(ci + k));
      const double2 v0 = __ldcs(reinterpret_cast<const double2*>(av + k));
      const double2 v1 = __ldcs(reinterpret_cast<const double2*>(av + k + 2));
      s = fma(v0.x, xf(c4.x), s);
      s1 = fma(v0.y, xf(c4.y), s1);
      s2 = fma(v1.x, xf(c4.z), s2);
      s3 = fma(v1.y, xf(c4.w), s3);
    }
    s = (s + s1) + (s2 + s3);
    if (e + lane < hi) s = fma(__ldcs(av + e + lane), xf(__ldcs(ci + e + lane)), s);
  } else {
    // B entries per lane per trip (4 with one lane per row, else 2), every load of a trip
    // issued before its first use: a short row costs one memory round trip per level
    // (index, gather), not one per entry.  One accumulator: a slot past the row end adds
    // 0 * 0, and no partial sums are combined -- an SM of GB300 completes two FP64 lanes
    // per clock, so every warp-wide FP64 instruction costs 16 clocks of it.
    constexpr int B = G == 1 ? 4 : 2;
    for (int64_t k = lo + lane; k < hi; k += B * G) {
      int32_t c[B];
      double v[B], xg[B];
#pragma unroll
      for (int u = 0; u < B; ++u) {
        const bool ok = k + u * G < hi;
        c[u] = ok ? __ldcs(ci + k + u * G) : 0;
        v[u] = ok ? __ldcs(av + k + u * G) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < B; ++u) xg[u] = k + u * G < hi ? xf(c[u]) : 0.0;
#pragma unroll
      for (int u = 0; u < B; ++u) s = fma(v[u], xg[u], s);
    }
  }
  return s;
}

// The FP64 dot of dot64 over either index width (16-bit columns when every column fits).
template <int G, bool V, typename IT>
RDEV double dot_jv(int64_t lo, int64_t hi, int lane, const IT* __restrict__ ci,
                   const double* __restrict__ av, const double* __restrict__ x, double init = 0.0) {
  double s = init;
  if constexpr (V) {
    int64_t a = (lo + 3) & ~int64_t(3);
    if (a > hi) a = hi;
    const int64_t e = a + ((hi - a) & ~int64_t(3));
    if (lo + lane < a) s = fma(__ldcs(av + lo + lane), __ldg(x + ld_idx(ci + lo + lane)), s);
    double s1 = 0.0, s2 = 0.0, s3 = 0.0;   // independent FP64 chains (see dot64)
    for (int64_t k = a + 4 * lane; k < e; k += 4 * G) {
      const int4 c4 = ld_idx4(ci + k);
      const double2 v0 = __ldcs(reinterpret_cast<const double2*>(av + k));
      const double2 v1 = __ldcs(reinterpret_cast<const double2*>(av + k + 2));
      s = fma(v0.x, __ldg(x + c4.x), s);
      s1 = fma(v0.y, __ldg(x + c4.y), s1);
      s2 = fma(v1.x, __ldg(x + c4.z), s2);
      s3 = fma(v1.y, __ldg(x + c4.w), s3);
    }
    s = (s + s1) + (s2 + s3);
    if (e + lane < hi) s = fma(__ldcs(av + e + lane), __ldg(x + ld_idx(ci + e + lane)), s);
  } else {
    constexpr int B = G == 1 ? 4 : 2;   // loads of a trip first, one accumulator (see dot64)
    for (int64_t k = lo + lane; k < hi; k += B * G) {
      int c[B];
      double v[B], xg[B];
#pragma unroll
      for (int u = 0; u < B; ++u) {
        const bool ok = k + u * G < hi;
        c[u] = ok ? ld_idx(ci + k + u * G) : 0;
        v[u] = ok ? __ldcs(av + k + u * G) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < B; ++u) xg[u] = k + u * G < hi ? __ldg(x + c[u]) : 0.0;
#pragma unroll
      for (int u = 0; u < B; ++u) s = fma(v[u], xg[u], s);
    }
  }
  return s;
}

// FP32 values, FP32 accumulation (inner sweeps of the mixed method).  XS: x lives in
// shared memory (plain loads) instead of global memory (read-only path).
template <int G, bool V, typename IT = int32_t, int U = 2, bool XS = false>
RDEV float dot32(int64_t lo, int64_t hi, int lane, const IT* __restrict__ ci,
                 const float* __restrict__ av, const float* __restrict__ x) {
  auto gx = [x](int j) { return XS ? x[j] : __ldg(x + j); };
  float s = 0.0f;
  if constexpr (V) {
    int64_t a = (lo + 3) & ~int64_t(3);
    if (a > hi) a = hi;
    const int64_t e = a + ((hi - a) & ~int64_t(3));
    if (lo + lane < a) s = fmaf(__ldcs(av + lo + lane), gx(ld_idx(ci + lo + lane)), s);
    // U quads per lane per trip, software-pipelined: the next trip's index and value
    // loads are issued before this trip's gathers, so HBM loads stay in flight while
    // the gathers of x (L1 / L2) complete.  Quads past the row end load as zeros.
    float acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] = 0.0f;
    int4 c4[U];
    float4 v4[U];
    auto load_trip = [&](int64_t k, int4 (&ci4)[U], float4 (&vv4)[U]) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t kk = k + 4 * G * u;
        if (kk < e) {
          ci4[u] = ld_idx4(ci + kk);
          vv4[u] = __ldcs(reinterpret_cast<const float4*>(av + kk));
        } else {
          ci4[u] = make_int4(0, 0, 0, 0);
          vv4[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
    };
    int64_t k = a + 4 * lane;
    load_trip(k, c4, v4);
    while (k < e) {
      const int64_t kn = k + 4 * G * U;
      int4 n4[U];
      float4 w4[U];
      load_trip(kn, n4, w4);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        acc[u] = fmaf(v4[u].x, gx(c4[u].x), acc[u]);
        acc[u] = fmaf(v4[u].y, gx(c4[u].y), acc[u]);
        acc[u] = fmaf(v4[u].z, gx(c4[u].z), acc[u]);
        acc[u] = fmaf(v4[u].w, gx(c4[u].w), acc[u]);
        c4[u] = n4[u];
        v4[u] = w4[u];
      }
      k = kn;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) s += acc[u];
    if (e + lane < hi) s = fmaf(__ldcs(av + e + lane), gx(ld_idx(ci + e + lane)), s);
  } else {
    // four entries per lane per trip, loads first (see dot64)
    float s1 = 0.0f;
    for (int64_t k = lo + lane; k < hi; k += 4 * G) {
      int c[4];
      float v[4], xg[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool ok = k + u * G < hi;
        c[u] = ok ? ld_idx(ci + k + u * G) : 0;
        v[u] = ok ? __ldcs(av + k + u * G) : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) xg[u] = k + u * G < hi ? __ldg(x + c[u]) : 0.0f;
      s = fmaf(v[0], xg[0], s);
      s1 = fmaf(v[1], xg[1], s1);
      s = fmaf(v[2], xg[2], s);
      s1 = fmaf(v[3], xg[3], s1);
    }
    s += s1;
  }
  return s;
}

RDEV double nan_to_inf(double v) { return v != v ? __longlong_as_double(0x7ff0000000000000LL) : v; }

// |v| as its bit pattern: non-negative doubles order like their bits, so a running
// max|x' - x| can use integer compares and keep the FP64 pipe for the sums.
RDEV unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}
RDEV unsigned long long umax64(unsigned long long a, unsigned long long b) { return a > b ? a : b; }
// Back to a double; NaN (bits above +inf) reads as +inf.
RDEV double bits_to_delta(unsigned long long b) {
  return __longlong_as_double((long long)(b > 0x7ff0000000000000ull ? 0x7ff0000000000000ull : b));
}

template <int NV, bool MAX>
RDEV void cta_to_slot(double v, unsigned long long* slot) {
  __shared__ double sh[32];
  double a[1] = {v};
  block_reduce<1, true>(a, sh);
  if (threadIdx.x == 0) atomic_max_nonneg(slot, nan_to_inf(a[0]));
}

// Last CTA of the grid reduces NS sums followed by NM maxima.
template <int NS, int NM>
RDEV bool last_cta_reduce(double (&mine)[NS + NM], double* part, unsigned* ticket,
                          double (&tot)[NS + NM]) {
  constexpr int NV = NS + NM;
  __shared__ double sh[NV * 32];
  __shared__ bool is_last;
  double bl[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) bl[j] = mine[j];
  {
    double s[NS > 0 ? NS : 1];
    double mx[NM > 0 ? NM : 1];
#pragma unroll
    for (int j = 0; j < NS; ++j) s[j] = bl[j];
#pragma unroll
    for (int j = 0; j < NM; ++j) mx[j] = bl[NS + j];
    if constexpr (NS > 0) block_reduce<NS, false>(reinterpret_cast<double(&)[NS]>(s), sh);
    if constexpr (NM > 0) block_reduce<NM, true>(reinterpret_cast<double(&)[NM]>(mx), sh);
#pragma unroll
    for (int j = 0; j < NS; ++j) bl[j] = s[j];
#pragma unroll
    for (int j = 0; j < NM; ++j) bl[NS + j] = mx[j];
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) part[j * gridDim.x + blockIdx.x] = bl[j];
    __threadfence();
    is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double s[NS > 0 ? NS : 1];
  double mx[NM > 0 ? NM : 1];
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    s[j] = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) s[j] += __ldcg(part + j * gridDim.x + b);
  }
#pragma unroll
  for (int j = 0; j < NM; ++j) {
    mx[j] = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
      mx[j] = fmax(mx[j], nan_to_inf(__ldcg(part + (NS + j) * gridDim.x + b)));
  }
  if constexpr (NS > 0) block_reduce<NS, false>(reinterpret_cast<double(&)[NS]>(s), sh);
  if constexpr (NM > 0) block_reduce<NM, true>(reinterpret_cast<double(&)[NM]>(mx), sh);
#pragma unroll
  for (int j = 0; j < NS; ++j) tot[j] = s[j];
#pragma unroll
  for (int j = 0; j < NM; ++j) tot[NS + j] = mx[j];
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// ------------------------------------------------------------------ Jacobi FP64 (§3.1)
// x'_i = (b_i + sum_{j != i} A_ij x_j) / d_i with d_i = 1 - A_ii: the paper's row
// update for M = I - A, double buffered; max|x' - x| is reduced into slot.  DELTA: only the
// sweep whose max|x' - x| the stopping test reads computes it (the last of each group of
// sweeps between checks); the others skip the FP64 difference and the reduction.

template <int G, bool V, bool DELTA = true>
__global__ void __launch_bounds__(NT) k_jacobi64(int64_t nq, const int64_t* __restrict__ rp,
                                                 const int32_t* __restrict__ ci,
                                                 const double* __restrict__ aj,
                                                 const double* __restrict__ bj,
                                                 const double* __restrict__ x,
                                                 double* __restrict__ xn, unsigned long long* slot, unsigned* ctr) {
  RowGroups rg = RowGroups::make<G>();
  unsigned long long mx = 0ull;
  auto xf = [x](int32_t j) { return __ldg(x + j); };
  for (int64_t i = row_begin<G>(rg, ctr); warp_has_row<G>(i, nq); i = row_next<G>(rg, ctr, i)) {
    double s = 0.0, bv = 0.0, xo = 0.0;
    // short rows: row-side loads issued ahead of the row's entries (long vector rows
    // would only hold the registers)
    if (!V && i < nq && rg.lane == 0) {
      bv = bj[i];
      if (DELTA) xo = x[i];
    }
    // short rows: the sum starts at bj_i in lane 0 (bv = 0 elsewhere), which saves the
    // separate FP64 add on a pipe that bounds these sweeps
    if (i < nq) s = dot64<G, V>(rp[i], rp[i + 1], rg.lane, ci, aj, xf, V ? 0.0 : bv);
    s = group_sum<G>(s);
    if (i < nq && rg.lane == 0) {
      if (V) {
        bv = bj[i];
        if (DELTA) xo = x[i];
      }
      // (b_i + sum A_ij x_j) / d_i in the Jacobi form
      const double xv = V ? bv + s : s;
      if (DELTA) mx = umax64(mx, abs_bits(xv - xo));
      xn[i] = xv;
    }
  }
  if (DELTA) cta_to_slot<1, true>(bits_to_delta(mx), slot);
}

// ------------------------------------------------------------------ certified error bound
// For M = I - A (§2.3) and any x, ||x* - x||_inf <= ||M^-1||_inf ||b - M x||_inf.  The
// residual kernel below returns, per row, an upper bound of the EXACT |b - M x|_i of the
// stored FP64 system: the computed |r_i| plus the rounding allowance gamma_D S_i, where
// S_i = |b_i| + |d_i x_i| + sum_j |A_ij x_j| (summed with upward rounding) and D the number
// of roundings any term passes through in this kernel's fixed order (ceil(len / G)
// sequential FMAs per lane, log2 G shuffle additions, then + b_i and - d_i x_i), with
// gamma_D = D u / (1 - D u), u = 2^-53, bounded above by D u (1 + 2 D u) with upward
// rounding (no division).


template <int G>
constexpr int log2_of() { return G <= 1 ? 0 : 1 + log2_of<G / 2>(); }

template <int G>
__global__ void __launch_bounds__(NT) k_resid_cert(int64_t nq, const int64_t* __restrict__ rp,
                                                   const int32_t* __restrict__ ci,
                                                   const double* __restrict__ av,
                                                   const double* __restrict__ b,
                                                   const double* __restrict__ d,
                                                   const double* __restrict__ x,
                                                   unsigned long long* slot_r, unsigned long long* slot_ub) {
  RowGroups rg = RowGroups::make<G>();
  unsigned long long mr = 0ull, mu = 0ull;
  for (int64_t i = rg.first; warp_has_row<G>(i, nq); i += rg.stride) {
    double s = 0.0, a = 0.0;
    int64_t lo = 0, hi = 0;
    if (i < nq) {
      lo = rp[i];
      hi = rp[i + 1];
      for (int64_t k = lo + rg.lane; k < hi; k += G) {
        const double v = __ldcs(av + k), xv = __ldg(x + __ldcs(ci + k));
        s = fma(v, xv, s);
        a = __fma_ru(fabs(v), fabs(xv), a);
      }
    }
    s = group_sum<G>(s);
    a = group_sum_ru<G>(a);
    if (i < nq && rg.lane == 0) {
      const double bi = b[i], di = d[i], xi = x[i];
      const double r = fma(-di, xi, bi + s);
      const double sum_abs = __dadd_ru(__dadd_ru(a, fabs(bi)), __dmul_ru(fabs(di), fabs(xi)));
      const double depth = (double)((hi - lo + G - 1) / G + log2_of<G>() + 2);
      const double du = depth * 0x1p-53;   // exact: an integer times a power of two
      // gamma = du / (1 - du) <= du (1 + 2 du) for du <= 1/2, without an FP64 division
      const double gam = __fma_ru(2.0 * du, du, du);
      const double ub = __dadd_ru(fabs(r), __dmul_ru(gam, sum_abs));
      mr = umax64(mr, abs_bits(r));
      mu = umax64(mu, abs_bits(ub));
    }
  }
  __shared__ double sh[64];
  double v[2] = {bits_to_delta(mr), bits_to_delta(mu)};
  block_reduce<2, true>(v, sh);
  if (threadIdx.x == 0) {
    atomic_max_nonneg(slot_r, nan_to_inf(v[0]));
    atomic_max_nonneg(slot_ub, nan_to_inf(v[1]));
  }
}


// Lower bound, per row, of (|M| w)_i in the sense needed by the norm bounds:
//   ABS:  |d_i| - sum_j |A_ij|          (w = 1: Varah's row-dominance margin)
//   else: d_i w_i - sum_j A_ij w_j      (M w for a chain's M-matrix, A >= 0)
// The subtracted sum is accumulated with upward rounding (an upper bound of the exact
// sum whatever the signs), the first term with downward rounding, the difference rounded
// down: a guaranteed lower bound of the exact value.  min over rows -> *kmin, and for
// !ABS max_i w_i -> *kmax, both as ordered keys.
template <int G, bool ABS>
__global__ void __launch_bounds__(NT) k_row_lower(int64_t nq, const int64_t* __restrict__ rp,
                                                  const int32_t* __restrict__ ci,
                                                  const double* __restrict__ av,
                                                  const double* __restrict__ d,
                                                  const double* __restrict__ w,
                                                  unsigned long long* kmin, unsigned long long* kmax) {
  RowGroups rg = RowGroups::make<G>();
  double lo_min = __longlong_as_double(0x7ff0000000000000LL), w_max = -lo_min;
  for (int64_t i = rg.first; warp_has_row<G>(i, nq); i += rg.stride) {
    double a = 0.0;
    if (i < nq)
      for (int64_t k = rp[i] + rg.lane; k < rp[i + 1]; k += G) {
        const double v = av[k];
        a = ABS ? __dadd_ru(a, fabs(v)) : __fma_ru(v, w[ci[k]], a);
      }
    a = group_sum_ru<G>(a);
    if (i < nq && rg.lane == 0) {
      const double first = ABS ? fabs(d[i]) : __dmul_rd(d[i], w[i]);
      const double lo = __dadd_rd(first, -a);
      lo_min = fmin(lo_min, lo != lo ? -__longlong_as_double(0x7ff0000000000000LL) : lo);
      if (!ABS) w_max = fmax(w_max, w[i]);
    }
  }
  // warp reductions and one atomic per warp: the values have either sign, which the
  // zero-padded block reduction does not handle
  lo_min = -warp_max(-lo_min);
  if (!ABS) w_max = warp_max(w_max);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(kmin, ordered_key(lo_min));
    if (!ABS) atomicMax(kmax, ordered_key(w_max));
  }
}

__global__ void k_fill_tau_rhs(int64_t nq, const double* __restrict__ d, double* __restrict__ b,
                               double* __restrict__ bj) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x) {
    b[i] = 1.0;
    bj[i] = 1.0 / d[i];
  }
}

__global__ void k_check(SolveState* st, int slot_idx, int sweeps, int reset_n) {
  if (st->done) return;
  const double dl = slot_value(&st->slot[slot_idx]);
  st->iter += sweeps;
  st->last = dl;
  if (dl < st->eps) {
    st->done = 1;
    st->status = REACH_OK;
  } else if (st->iter >= st->max_iter) {
    st->done = 1;
    st->status = REACH_ENOTCONV;
  }
  for (int j = 0; j < reset_n; ++j) {
    st->slot[j] = 0ull;
    st->rowctr[j] = 0u;
  }
}

__global__ void k_loop_ctl(SolveState* st, cudaGraphConditionalHandle h, int use_cond) {
  st->bodies += 1;
  if (!st->done && st->bodies >= st->max_bodies) {
    st->done = 1;
    st->status = REACH_ETIMEOUT;
  }
  if (use_cond) cudaGraphSetConditional(h, st->done ? 0u : 1u);
}

__global__ void k_finalize_resid(SolveState* st) {
  st->resid = slot_value(&st->slot[63]);
  st->resid_ub = slot_value(&st->slot[61]);
  st->slot[63] = 0ull;
  st->slot[61] = 0ull;
}

// ------------------------------------------------------------------ mixed precision
// Defect correction around the same Jacobi iteration, on the Jacobi form
// (Aj = D^-1 A, bj = D^-1 b): the FP64 residual step writes r = bj + Aj x - x (FP32),
// which is also the first correction sweep d_0; FP32 sweeps d <- r + Aj_hi d follow;
// then x += d in FP64.  max|r_i| is exactly the max|x' - x| of an FP64 Jacobi sweep
// from x, so the stopping rule matches.

// The FP64 residual step reads the FP64 Jacobi-form values: one FP64 FMA and one gather of x
// per entry, 10 (16-bit columns) or 12 bytes per entry.  Reading the FP32 pair hi + lo
// instead moves the same bytes but adds an FP32 product against an FP32 copy of x and the
// widening of hi, and was 1.31x slower on the dense benchmark system.
template <int G, bool V, typename IT>
__global__ void __launch_bounds__(NT) k_resid_jv(int64_t nq, const int64_t* __restrict__ rp,
                                                 const IT* __restrict__ ci, const double* __restrict__ av,
                                                 const double* __restrict__ bj, const double* __restrict__ x,
                                                 float* __restrict__ r32, float* __restrict__ dl0,
                                                 SolveState* st, int slot_idx, unsigned* ctr) {
  if (st->done) return;
  RowGroups rg = RowGroups::make<G>();
  unsigned long long mx = 0ull;
  for (int64_t i = row_begin<G>(rg, ctr); warp_has_row<G>(i, nq); i = row_next<G>(rg, ctr, i)) {
    double s = 0.0, bv = 0.0, xo = 0.0;
    if (!V && i < nq && rg.lane == 0) {  // short rows: row-side loads issued early
      bv = bj[i];
      xo = x[i];
    }
    if (i < nq) s = dot_jv<G, V, IT>(rp[i], rp[i + 1], rg.lane, ci, av, x, V ? 0.0 : bv);
    s = group_sum<G>(s);
    if (i < nq && rg.lane == 0) {
      if (V) {
        bv = bj[i];
        xo = x[i];
      }
      const double r = (V ? bv + s : s) - xo;   // bj_i + (Aj x)_i - x_i
      const float rf = __double2float_rn(r);
      r32[i] = rf;
      dl0[i] = rf;
      mx = umax64(mx, abs_bits(r));
    }
  }
  cta_to_slot<1, true>(bits_to_delta(mx), &st->slot[slot_idx]);
}

__global__ void k_check_mixed(SolveState* st, int slot_idx, int k) {
  if (st->done) return;
  const double dl = slot_value(&st->slot[slot_idx]);
  st->slot[slot_idx] = 0ull;
  st->refinements += 1;
  st->iter += 1;
  st->last = dl;
  if (dl < st->eps) {
    st->done = 1;
    st->status = REACH_OK;
  } else if (st->iter + (k - 1) > st->max_iter) {
    st->done = 1;
    st->status = REACH_ENOTCONV;
  } else {
    st->iter += k - 1;
  }
}

template <int G, bool V, typename IT, int U>
__global__ void __launch_bounds__(NT) k_sweep32(int64_t nq, const int64_t* __restrict__ rp,
                                                const IT* __restrict__ ci,
                                                const float* __restrict__ ah,
                                                const float* __restrict__ r32,
                                                const float* __restrict__ din,
                                                float* __restrict__ dout, const SolveState* st, unsigned* ctr) {
  if (st->done) return;
  RowGroups rg = RowGroups::make<G>();
  for (int64_t i = row_begin<G>(rg, ctr); warp_has_row<G>(i, nq); i = row_next<G>(rg, ctr, i)) {
    float s = 0.0f, rv = 0.0f;
    if (!V && i < nq && rg.lane == 0) rv = r32[i];  // short rows: issued early
    if (i < nq) s = dot32<G, V, IT, U>(rp[i], rp[i + 1], rg.lane, ci, ah, din);
    s = group_sum<G>(s);
    if (i < nq && rg.lane == 0) dout[i] = (V ? r32[i] : rv) + s;
  }
}

// The FP32 sweep with the correction vector staged in shared memory (layout 72): every
// CTA copies din (n? floats, at most SMX_MAX_ROWS) into shared memory once per launch, and
// a row's gathers then read shared memory instead of L1, whose tag lookups for 32 scattered
// addresses per warp instruction compete with the streamed matrix.  One CTA of 1024 threads
// per SM; a warp per row from the row counter, 16-byte loads of four 16-bit indices and four
// values, two quads per lane in flight.
constexpr int SMX_NT = 1024;
constexpr int64_t SMX_MAX_ROWS = 53248;   // 208 KB of FP32

__global__ void __launch_bounds__(SMX_NT, 1) k_sweep32_smem(int64_t nq, const int64_t* __restrict__ rp,
                                                            const uint16_t* __restrict__ ci,
                                                            const float* __restrict__ ah,
                                                            const float* __restrict__ r32,
                                                            const float* __restrict__ din, float* __restrict__ dout,
                                                            const SolveState* st, unsigned* ctr) {
  extern __shared__ float xs[];
  if (st->done) return;
  const int64_t n4 = nq >> 2;
  for (int64_t j = threadIdx.x; j < n4; j += blockDim.x)
    reinterpret_cast<float4*>(xs)[j] = __ldg(reinterpret_cast<const float4*>(din) + j);
  for (int64_t j = 4 * n4 + threadIdx.x; j < nq; j += blockDim.x) xs[j] = __ldg(din + j);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (int64_t i = warp_fetch_row(ctr); i < nq; i = warp_fetch_row(ctr)) {
    float s = dot32<32, true, uint16_t, 2, true>(rp[i], rp[i + 1], lane, ci, ah, xs);
    s = warp_sum(s);
    if (lane == 0) dout[i] = r32[i] + s;
  }
}

cudaError_t sweep32_smem(reach_ctx* c, const float* din, float* dout, cudaStream_t s, unsigned* ctr) {
  const size_t bytes = sizeof(float) * (size_t)c->n_q;
  // per device and cheap: set on every launch rather than cached in a static
  cudaError_t e = cudaFuncSetAttribute((const void*)k_sweep32_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(float) * SMX_MAX_ROWS));
  if (e != cudaSuccess) return e;
  k_sweep32_smem<<<c->sm_count, SMX_NT, bytes, s>>>(c->n_q, c->a_rowptr, c->a_col16, c->a_hi, c->r32, din, dout,
                                                   c->st, ctr);
  return cudaGetLastError();
}

// out_i = v_i / d_i (the right-hand side of a Jacobi form).
__global__ void k_div_d(int64_t nq, const double* __restrict__ v, const double* __restrict__ d,
                        double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = v[i] / d[i];
}

// x += delta in FP64, and the FP32 copy of x used by the next residual step.
// With dl == nullptr only the copy is refreshed (start of a solve).
__global__ void k_apply(int64_t nq, double* __restrict__ x, float* __restrict__ xf,
                        const float* __restrict__ dl, SolveState* st, int reset_n) {
  if (st->done) return;
  if (blockIdx.x == 0 && threadIdx.x < reset_n) st->rowctr[threadIdx.x] = 0u;  // counters of this body
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = dl ? x[i] + (double)dl[i] : x[i];
    x[i] = v;
    xf[i] = __double2float_rn(v);
  }
}

// ------------------------------------------------------------------ BiCGStab (§3.2)
// M = I - A, (M u)_i = d_i u_i - sum_{j != i} A_ij u_j.  Per iteration: p update;
// v = M p with q.v fused (a = y / q.v in the last CTA); t = M s with s = r - a v
// formed on the fly, t.s, t.t and max|s| fused (w = t.s / t.t); then x and r with
// q.r and max|r| fused (next y and beta).  All sums are fixed-order two-stage.

template <int G, bool V>
__global__ void __launch_bounds__(NT) k_bi_init(int64_t nq, const int64_t* __restrict__ rp,
                                                const int32_t* __restrict__ ci,
                                                const double* __restrict__ av,
                                                const double* __restrict__ b,
                                                const double* __restrict__ d,
                                                const double* __restrict__ x,
                                                double* __restrict__ r, double* __restrict__ q,
                                                double* __restrict__ p, double* __restrict__ v,
                                                double* part, unsigned* ticket, BiState* bi,
                                                SolveState* st) {
  RowGroups rg = RowGroups::make<G>();
  double acc[2] = {0.0, 0.0};
  auto xf = [x](int32_t j) { return __ldg(x + j); };
  for (int64_t i = rg.first; warp_has_row<G>(i, nq); i += rg.stride) {
    double s = 0.0;
    if (i < nq) s = dot64<G, V>(rp[i], rp[i + 1], rg.lane, ci, av, xf);
    s = group_sum<G>(s);
    if (i < nq && rg.lane == 0) {
      const double ri = b[i] - (d[i] * x[i] - s);
      r[i] = ri;
      q[i] = ri;
      p[i] = 0.0;
      v[i] = 0.0;
      acc[0] = fma(ri, ri, acc[0]);
      acc[1] = fmax(acc[1], nan_to_inf(fabs(ri)));
    }
  }
  double tot[2];
  if (last_cta_reduce<1, 1>(acc, part, ticket, tot) && threadIdx.x == 0) {
    bi->y = tot[0];
    bi->yprev = 1.0;
    bi->a = 1.0;
    bi->w = 1.0;
    bi->beta = 0.0;
    bi->s_done = 0;
    bi->restarted = 0;
    bi->restart = 0;
    bi->skip = 0;
    bi->rr = tot[0];
    bi->rnorm = tot[1];
    st->last = tot[1];
    if (tot[1] < st->eps) {
      st->done = 1;
      st->status = REACH_OK;
    }
  }
}

// p = r + beta (p - w v).  After a breakdown the iteration restarts from the current
// residual: q = r, p = r, v = 0 (y = r.r was set by the CTA that detected it).
__global__ void k_bi_p(int64_t nq, const double* __restrict__ r, double* __restrict__ p,
                       double* __restrict__ v, double* __restrict__ q, BiState* bi,
                       SolveState* st) {
  if (st->done) return;
  const double beta = bi->beta, w = bi->w;
  const int rs = bi->restart;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    bi->skip = 0;
    st->rowctr[0] = 0u;   // row counters of k_bi_v and k_bi_t
    st->rowctr[1] = 0u;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = r[i];
    if (rs) {
      q[i] = ri;
      p[i] = ri;
      v[i] = 0.0;
    } else {
      p[i] = ri + beta * (p[i] - w * v[i]);
    }
  }
}

// A breakdown restarts once (q = r); a second one ends the solve with EBREAKDOWN.
RDEV bool bi_restart_or_fail(BiState* bi, SolveState* st) {
  if (bi->restarted) {
    st->done = 1;
    st->status = REACH_EBREAKDOWN;
    return false;
  }
  bi->restarted = 1;
  bi->restart = 1;
  bi->y = bi->rr;
  return true;
}

// After v = M p and q.v: a = y / q.v, or a breakdown restart.
RDEV void bi_v_done(const double (&tot)[1], BiState* bi, SolveState* st) {
  bi->qv = tot[0];
  bi->restart = 0;
  if (tot[0] == 0.0 || !(fabs(tot[0]) <= DBL_MAX)) {
    if (bi_restart_or_fail(bi, st)) bi->skip = 1;
  } else {
    bi->a = bi->y / tot[0];
  }
}

// After t = M s with t.s, t.t and max|s|: finish with x += a p when max|s| < eps, else
// w = t.s / t.t.
RDEV void bi_t_done(const double (&tot)[3], BiState* bi, SolveState* st) {
  bi->ts = tot[0];
  bi->tt = tot[1];
  bi->snorm = tot[2];
  if (tot[2] < st->eps) {
    bi->s_done = 1;
  } else if (tot[1] == 0.0) {
    st->done = 1;
    st->status = REACH_EBREAKDOWN;
  } else {
    bi->w = tot[0] / tot[1];
  }
}

template <int G, bool V>
__global__ void __launch_bounds__(NT) k_bi_v(int64_t nq, const int64_t* __restrict__ rp,
                                             const int32_t* __restrict__ ci,
                                             const double* __restrict__ av,
                                             const double* __restrict__ d,
                                             const double* __restrict__ p,
                                             const double* __restrict__ q, double* __restrict__ v,
                                             double* part, unsigned* ticket, BiState* bi,
                                             SolveState* st, unsigned* ctr) {
  if (st->done) return;
  RowGroups rg = RowGroups::make<G>();
  double acc[1] = {0.0};
  auto pf = [p](int32_t j) { return __ldg(p + j); };
  for (int64_t i = row_begin<G>(rg, ctr); warp_has_row<G>(i, nq); i = row_next<G>(rg, ctr, i)) {
    double s = 0.0;
    if (i < nq) s = dot64<G, V>(rp[i], rp[i + 1], rg.lane, ci, av, pf);
    s = group_sum<G>(s);
    if (i < nq && rg.lane == 0) {
      const double vi = d[i] * p[i] - s;
      v[i] = vi;
      acc[0] = fma(q[i], vi, acc[0]);
    }
  }
  double tot[1];
  if (last_cta_reduce<1, 0>(acc, part, ticket, tot) && threadIdx.x == 0) bi_v_done(tot, bi, st);
}

// v = M p from y = A p of the entry-balanced product: v_i = d_i p_i - y_i, q.v fused.
__global__ void __launch_bounds__(NT) k_bi_v_ew(int64_t nq, const double* __restrict__ d,
                                                const double* __restrict__ p, const double* __restrict__ y,
                                                const double* __restrict__ q, double* __restrict__ v,
                                                double* part, unsigned* ticket, BiState* bi, SolveState* st) {
  if (st->done) return;
  double acc[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double vi = d[i] * p[i] - y[i];
    v[i] = vi;
    acc[0] = fma(q[i], vi, acc[0]);
  }
  double tot[1];
  if (last_cta_reduce<1, 0>(acc, part, ticket, tot) && threadIdx.x == 0) bi_v_done(tot, bi, st);
}

// s = r - a v (elementwise; formed once here instead of at every gather of the next
// product, which doubled that product's FP64 work).
__global__ void k_bi_s(int64_t nq, const double* __restrict__ r, const double* __restrict__ v,
                       double* __restrict__ s, const BiState* bi, const SolveState* st) {
  if (st->done || bi->skip) return;
  const double a = bi->a;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq;
       i += (int64_t)gridDim.x * blockDim.x)
    s[i] = r[i] - a * v[i];
}

template <int G, bool V>
__global__ void __launch_bounds__(NT) k_bi_t(int64_t nq, const int64_t* __restrict__ rp,
                                             const int32_t* __restrict__ ci,
                                             const double* __restrict__ av,
                                             const double* __restrict__ d,
                                             const double* __restrict__ sv, double* __restrict__ t,
                                             double* part, unsigned* ticket, BiState* bi,
                                             SolveState* st, unsigned* ctr) {
  if (st->done || bi->skip) return;
  RowGroups rg = RowGroups::make<G>();
  double acc[3] = {0.0, 0.0, 0.0};
  auto sf = [sv](int32_t j) { return __ldg(sv + j); };
  for (int64_t i = row_begin<G>(rg, ctr); warp_has_row<G>(i, nq); i = row_next<G>(rg, ctr, i)) {
    double s = 0.0;
    if (i < nq) s = dot64<G, V>(rp[i], rp[i + 1], rg.lane, ci, av, sf);
    s = group_sum<G>(s);
    if (i < nq && rg.lane == 0) {
      const double si = sv[i];
      const double ti = d[i] * si - s;
      t[i] = ti;
      acc[0] = fma(ti, si, acc[0]);
      acc[1] = fma(ti, ti, acc[1]);
      acc[2] = fmax(acc[2], nan_to_inf(fabs(si)));
    }
  }
  double tot[3];
  if (last_cta_reduce<2, 1>(acc, part, ticket, tot) && threadIdx.x == 0) bi_t_done(tot, bi, st);
}

// t = M s from y = A s of the entry-balanced product: t_i = d_i s_i - y_i, with t.s, t.t
// and max|s| fused.
__global__ void __launch_bounds__(NT) k_bi_t_ew(int64_t nq, const double* __restrict__ d,
                                                const double* __restrict__ sv, const double* __restrict__ y,
                                                double* __restrict__ t, double* part, unsigned* ticket,
                                                BiState* bi, SolveState* st) {
  if (st->done || bi->skip) return;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double si = sv[i];
    const double ti = d[i] * si - y[i];
    t[i] = ti;
    acc[0] = fma(ti, si, acc[0]);
    acc[1] = fma(ti, ti, acc[1]);
    acc[2] = fmax(acc[2], nan_to_inf(fabs(si)));
  }
  double tot[3];
  if (last_cta_reduce<2, 1>(acc, part, ticket, tot) && threadIdx.x == 0) bi_t_done(tot, bi, st);
}

__global__ void __launch_bounds__(NT) k_bi_x(int64_t nq, double* __restrict__ x,
                                             const double* __restrict__ p,
                                             const double* __restrict__ s,
                                             const double* __restrict__ t, double* __restrict__ r,
                                             const double* __restrict__ q, double* part,
                                             unsigned* ticket, BiState* bi, SolveState* st) {
  if (st->done || bi->skip) return;
  const double a = bi->a, w = bi->w;
  const int s_done = bi->s_done;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (s_done) {
      x[i] += a * p[i];
    } else {
      x[i] += a * p[i] + w * s[i];
      const double ri = s[i] - w * t[i];
      r[i] = ri;
      acc[0] = fma(q[i], ri, acc[0]);
      acc[1] = fma(ri, ri, acc[1]);
      acc[2] = fmax(acc[2], nan_to_inf(fabs(ri)));
    }
  }
  double tot[3];
  if (last_cta_reduce<2, 1>(acc, part, ticket, tot) && threadIdx.x == 0) {
    st->iter += 1;
    if (s_done) {
      st->last = bi->snorm;
      st->done = 1;
      st->status = REACH_OK;
      return;
    }
    bi->rnorm = tot[2];
    bi->rr = tot[1];
    st->last = tot[2];
    bi->yprev = bi->y;
    bi->y = tot[0];
    if (tot[2] < st->eps) {
      st->done = 1;
      st->status = REACH_OK;
    } else if (st->iter >= st->max_iter) {
      st->done = 1;
      st->status = REACH_ENOTCONV;
    } else if (bi->y == 0.0 || w == 0.0 || !(fabs(bi->y) <= DBL_MAX)) {
      bi_restart_or_fail(bi, st);
    } else {
      bi->beta = (bi->y / bi->yprev) * (a / w);
    }
  }
}

// ------------------------------------------------------------------ host side

struct Lay {
  int g;
  bool vec;
  bool seg = false;     // entry-balanced tiles (segscan.cu) instead of a row mapping
  bool tma = false;     // FP32 sweep with rows staged by bulk copies (tma.cu); others as 64
  bool smx = false;     // FP32 sweep with the correction vector in shared memory; others as 64
};

constexpr int LAY_SEG = 128;
constexpr int LAY_VEC16 = 48;   // half a warp per row with 16-byte loads
constexpr int LAY_TMA = 80;
constexpr int LAY_SMX = 72;

static Lay lay_of(int code) {
  if (code == LAY_SEG) return Lay{32, true, true};
  if (code == LAY_TMA) return Lay{32, true, false, true};
  if (code == LAY_SMX) return Lay{32, true, false, false, true};
  if (code == LAY_VEC16) return Lay{16, true};
  return code >= 64 ? Lay{32, true} : Lay{code, false};
}

// Row mapping of `method`'s kernels: the autotuned choice if there is one, else the
// REACH_LANES override, else lanes from the mean row length (warp + 16-byte loads from 96).
// Lanes per row of the solver kernels when nothing is tuned, from the mean row length:
// one lane up to 6 entries (a model checker's state spaces), then G such that a lane
// takes about 3 to 6 entries (two per trip).  Measured: one lane is 1.9x faster than two
// on 2.4 entries per row and 2.3x faster than four on 4.9; four lanes win on 16.
static int solver_group(int64_t rows, int64_t nnz) {
  const double mean = rows > 0 ? (double)nnz / (double)rows : 0.0;
  if (mean <= 6.0) return 1;
  if (mean <= 12.0) return 2;
  if (mean <= 24.0) return 4;
  if (mean <= 48.0) return 8;
  if (mean <= 96.0) return 16;
  return 32;
}

static Lay layout(reach_ctx* c, int64_t rows, int64_t nnz, int method = 0) {
  if (method >= 0 && method < 3 && c->tune.gm[method] > 0) return lay_of(c->tune.gm[method]);
  if (c->tune.g > 0) {
    Lay L = lay_of(c->tune.g);
    // the shared-memory sweep needs 16-bit indices and a vector that fits: else as 64
    if (L.smx && (!c->a_col16 || c->n_q > SMX_MAX_ROWS)) L.smx = false;
    return L;
  }
  const int g = solver_group(rows, nnz);
  const bool vec = g == 32 && rows > 0 && nnz / rows >= 96;
  return {g, vec};
}

// Row mapping for a kernel that has no entry-balanced form (the reported FP64 residual,
// the start of BiCGStab): the method's mapping, or -- when the method runs on
// entry-balanced tiles, which the autotuner picks for a few very long rows -- a warp per
// row with 16-byte loads, so those rows are not left to a few lanes.  The transposed
// system (method -1) takes the default mapping from its mean row length.
static Lay row_layout(reach_ctx* c, int method) {
  const Lay L = layout(c, c->n_q, c->m_q, method);
  if (!L.seg) return L;
  if (method >= 0) return Lay{32, true};
  const int g = solver_group(c->n_q, c->m_q);
  return {g, g == 32 && c->n_q > 0 && c->m_q / c->n_q >= 96};
}

#define LAY_DISPATCH(L, FN, ...)                          \
  do {                                                    \
    if ((L).vec && (L).g == 16) FN<16, true>(__VA_ARGS__); \
    else if ((L).vec) FN<32, true>(__VA_ARGS__);          \
    else switch ((L).g) {                                 \
        case 1: FN<1, false>(__VA_ARGS__); break;         \
        case 2: FN<2, false>(__VA_ARGS__); break;         \
        case 4: FN<4, false>(__VA_ARGS__); break;         \
        case 8: FN<8, false>(__VA_ARGS__); break;         \
        case 16: FN<16, false>(__VA_ARGS__); break;       \
        default: FN<32, false>(__VA_ARGS__); break;       \
      }                                                   \
  } while (0)

struct Sys {
  int64_t nq;
  const int64_t* rp;
  const int32_t* ci;
  const double* av;
  const double* b;
};

template <int G, bool V>
static void l_jacobi(reach_ctx* c, const Sys& y, const double* x, double* xn, unsigned long long* slot,
                     cudaStream_t s, unsigned* ctr = nullptr) {
  const int grid = grid_rows(c, (const void*)k_jacobi64<G, V>, NT, G, y.nq, G == 32 && ctr);
  k_jacobi64<G, V><<<grid, NT, 0, s>>>(y.nq, y.rp, y.ci, y.av, y.b, x, xn, slot, G == 32 ? ctr : nullptr);
}

// A sweep whose max|x' - x| nobody reads.
template <int G, bool V>
static void l_jacobi_nd(reach_ctx* c, const Sys& y, const double* x, double* xn, unsigned long long* slot,
                        cudaStream_t s, unsigned* ctr = nullptr) {
  const int grid = grid_rows(c, (const void*)k_jacobi64<G, V, false>, NT, G, y.nq, G == 32 && ctr);
  k_jacobi64<G, V, false><<<grid, NT, 0, s>>>(y.nq, y.rp, y.ci, y.av, y.b, x, xn, slot, G == 32 ? ctr : nullptr);
}

// The reported residual: max|b - M x| and its certified upper bound (k_resid_cert, one
// accumulator per lane so that the rounding depth is known; V layouts use a warp per row).
template <int G, bool V>
static void l_resid(reach_ctx* c, const Sys& y, const double* x, cudaStream_t s) {
  const int grid = grid_rows(c, (const void*)k_resid_cert<G>, NT, G, y.nq);
  k_resid_cert<G><<<grid, NT, 0, s>>>(y.nq, y.rp, y.ci, y.av, y.b, c->d, x, &c->st->slot[63], &c->st->slot[61]);
}

// The mixed method's FP64 residual on the Jacobi form (16-bit column indices whenever every
// column fits).
template <int G, bool V>
static void l_resid_mixed(reach_ctx* c, int slot, cudaStream_t s, unsigned* ctr = nullptr) {
  unsigned* cr = G == 32 ? ctr : nullptr;
  if (c->a_col16) {
    const int grid = grid_rows(c, (const void*)k_resid_jv<G, V, uint16_t>, NT, G, c->n_q, cr != nullptr);
    k_resid_jv<G, V, uint16_t><<<grid, NT, 0, s>>>(c->n_q, c->a_rowptr, c->a_col16, c->a_jv, c->bj, c->x,
                                                   c->r32, c->dl[1], c->st, slot, cr);
  } else {
    const int grid = grid_rows(c, (const void*)k_resid_jv<G, V, int32_t>, NT, G, c->n_q, cr != nullptr);
    k_resid_jv<G, V, int32_t><<<grid, NT, 0, s>>>(c->n_q, c->a_rowptr, c->a_col, c->a_jv, c->bj, c->x,
                                                  c->r32, c->dl[1], c->st, slot, cr);
  }
}

template <int G, bool V, int U>
static void l_sweep32_u(reach_ctx* c, const float* din, float* dout, cudaStream_t s, unsigned* cr) {
  if (c->a_col16) {   // 16-bit column indices whenever every column fits
    const int grid = grid_rows(c, (const void*)k_sweep32<G, V, uint16_t, U>, NT, G, c->n_q, cr != nullptr);
    k_sweep32<G, V, uint16_t, U><<<grid, NT, 0, s>>>(c->n_q, c->a_rowptr, c->a_col16, c->a_hi, c->r32,
                                                     din, dout, c->st, cr);
  } else {
    const int grid = grid_rows(c, (const void*)k_sweep32<G, V, int32_t, U>, NT, G, c->n_q, cr != nullptr);
    k_sweep32<G, V, int32_t, U><<<grid, NT, 0, s>>>(c->n_q, c->a_rowptr, c->a_col, c->a_hi, c->r32,
                                                    din, dout, c->st, cr);
  }
}

// FP32 sweep; with warp-per-row vector loads the quads per trip (2 or 4) come from the
// layout code (64 or 66).
template <int G, bool V>
static void l_sweep32(reach_ctx* c, const float* din, float* dout, cudaStream_t s, unsigned* ctr = nullptr) {
  unsigned* cr = G == 32 ? ctr : nullptr;
  if constexpr (V) {
    if (c->tune.sweep_u == 4) {
      l_sweep32_u<G, V, 4>(c, din, dout, s, cr);
      return;
    }
  }
  l_sweep32_u<G, V, 2>(c, din, dout, s, cr);
}

// BiCGStab launchers on a system y (rows, values with diagonal c->d, right-hand side y.b):
// the chain's system, or its transpose for the adjoint solve.
template <int G, bool V>
static void l_bi_init(reach_ctx* c, const Sys& y, const double* x, cudaStream_t s) {
  const int grid = grid_rows(c, (const void*)k_bi_init<G, V>, NT, G, y.nq);
  k_bi_init<G, V><<<grid, NT, 0, s>>>(y.nq, y.rp, y.ci, y.av, y.b, c->d, x, c->vr, c->vq, c->vp, c->vv, c->part,
                                      c->ticket, c->bi, c->st);
}

template <int G, bool V>
static void l_bi_v(reach_ctx* c, const Sys& y, cudaStream_t s) {
  unsigned* cr = G == 32 ? &c->st->rowctr[0] : nullptr;
  const int grid = grid_rows(c, (const void*)k_bi_v<G, V>, NT, G, y.nq, cr != nullptr);
  k_bi_v<G, V><<<grid, NT, 0, s>>>(y.nq, y.rp, y.ci, y.av, c->d, c->vp, c->vq, c->vv, c->part, c->ticket, c->bi,
                                   c->st, cr);
}

template <int G, bool V>
static void l_bi_t(reach_ctx* c, const Sys& y, cudaStream_t s) {
  unsigned* cr = G == 32 ? &c->st->rowctr[1] : nullptr;
  const int grid = grid_rows(c, (const void*)k_bi_t<G, V>, NT, G, y.nq, cr != nullptr);
  k_bi_t<G, V><<<grid, NT, 0, s>>>(y.nq, y.rp, y.ci, y.av, c->d, c->vs, c->vt, c->part, c->ticket, c->bi, c->st,
                                   cr);
}

static int ew_grid(reach_ctx* c, const void* k, int64_t n) { return grid_for(c, k, NT, n); }

// Runs `body` inside a conditional while node until SolveState::done (device
// loops), or relaunches it from the host and polls `done` (host loops).  Graphs
// are cached in slot `gs` under `key`; the stopping parameters live in SolveState.
cudaError_t run_loop(reach_ctx* c, cudaGraphExec_t& exec, int64_t& exec_key, int64_t key,
                     const std::function<void(cudaStream_t, cudaGraphConditionalHandle, int)>& body) {
  cudaError_t e = cudaSuccess;
  if (!c->device_loops) {
    int32_t done = 0;
    while (!done) {
      body(c->stream, cudaGraphConditionalHandle(), 0);
      k_loop_ctl<<<1, 1, 0, c->stream>>>(c->st, cudaGraphConditionalHandle(), 0);
      e = cudaMemcpyAsync(&done, &c->st->done, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
  }
  if (exec == nullptr || exec_key != key) {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    cudaGraph_t graph = nullptr;
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
      cudaGraph_t bg = np.conditional.phGraph_out[0];
      e = cudaStreamBeginCaptureToGraph(c->cap, bg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
      if (e == cudaSuccess) {
        body(c->cap, h, 1);
        k_loop_ctl<<<1, 1, 0, c->cap>>>(c->st, h, 1);
        e = cudaStreamEndCapture(c->cap, &bg);
      }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      exec = nullptr;
      return e;
    }
    exec_key = key;
  }
  return cudaGraphLaunch(exec, c->stream);
}

static int64_t shape_key(reach_ctx* c, const Lay& L, int k) {
  return (c->n_q * 1000003LL + c->m_q) * 131 + L.g * 7 + (L.vec ? 1 : 0) + (L.seg ? 3 : 0) + (L.tma ? 5 : 0) +
         (L.smx ? 11 : 0) +
         1000LL * k +
         100000LL * c->tune.sweep_u;
}

cudaError_t solve_jacobi64(reach_ctx* c, const double* x0q, bool transposed) {
  if (!transposed && layout(c, c->n_q, c->m_q, REACH_JACOBI_FP64).seg) return solve_jacobi_seg(c, x0q);
  cudaStream_t s = c->stream;
  const int64_t nq = c->n_q;
  double* xa = transposed ? c->vr : c->x;
  double* xb = transposed ? c->vq : c->x2;
  if (x0q) cudaMemcpyAsync(xa, x0q, sizeof(double) * nq, cudaMemcpyDeviceToDevice, s);
  else cudaMemsetAsync(xa, 0, sizeof(double) * nq, s);
  // the sweep runs on the Jacobi form; the final residual on the system itself
  if (transposed)
    k_div_d<<<ew_grid(c, (const void*)k_div_d, nq), NT, 0, s>>>(nq, c->vp, c->d, c->vv);
  Sys y = transposed ? Sys{nq, c->at_rowptr, c->at_col, c->at_jv, c->vv}
                     : Sys{nq, c->a_rowptr, c->a_col, c->a_jv, c->bj};
  Sys yr = transposed ? Sys{nq, c->at_rowptr, c->at_col, c->at_val, c->vp}
                      : Sys{nq, c->a_rowptr, c->a_col, c->a_val, c->b};
  const Lay L = transposed ? row_layout(c, -1) : layout(c, nq, c->m_q, REACH_JACOBI_FP64);
  const int k = c->tune.k;
  if (!transposed && small_system(c, REACH_JACOBI_FP64)) {
    // the whole iteration in one launch on a thread-block cluster (small.cu)
    cudaError_t e = solve_small(c, REACH_JACOBI_FP64, k);
    if (e == cudaSuccess) {
      LAY_DISPATCH(L, l_resid, c, yr, xa, s);
      k_finalize_resid<<<1, 1, 0, s>>>(c->st);
      return cudaGetLastError();
    }
    if (e != cudaErrorNotSupported) return e;
  }
  const int gs = transposed ? 3 : 0;
  cudaError_t e = run_loop(c, c->g_exec[gs], c->g_key[gs], shape_key(c, L, k),
                           [&](cudaStream_t cs, cudaGraphConditionalHandle, int) {
                             for (int j = 0; j < k; ++j) {
                               const double* xi = (j & 1) ? xb : xa;
                               double* xo = (j & 1) ? xa : xb;
                               // the check reads the last sweep's max|x' - x| only
                               if (j == k - 1)
                                 LAY_DISPATCH(L, l_jacobi, c, y, xi, xo, &c->st->slot[j], cs, &c->st->rowctr[j]);
                               else
                                 LAY_DISPATCH(L, l_jacobi_nd, c, y, xi, xo, &c->st->slot[j], cs, &c->st->rowctr[j]);
                             }
                             k_check<<<1, 1, 0, cs>>>(c->st, k - 1, k, k);
                           });
  if (e != cudaSuccess) return e;
  LAY_DISPATCH(L, l_resid, c, yr, xa, s);
  k_finalize_resid<<<1, 1, 0, s>>>(c->st);
  return cudaGetLastError();
}

cudaError_t solve_mixed(reach_ctx* c, const double* x0q) {
  cudaStream_t s = c->stream;
  const int64_t nq = c->n_q;
  cudaError_t e = split_hilo(c);
  if (e != cudaSuccess) return e;
  if (x0q) cudaMemcpyAsync(c->x, x0q, sizeof(double) * nq, cudaMemcpyDeviceToDevice, s);
  else cudaMemsetAsync(c->x, 0, sizeof(double) * nq, s);
  if (small_system(c, REACH_JACOBI_MIXED)) {
    // the whole iteration in one launch on a thread-block cluster (small.cu)
    e = solve_small(c, REACH_JACOBI_MIXED, c->tune.k);
    if (e == cudaSuccess) {
      Sys y{nq, c->a_rowptr, c->a_col, c->a_val, c->b};
      const Lay LR = row_layout(c, REACH_JACOBI_MIXED);
      LAY_DISPATCH(LR, l_resid, c, y, c->x, s);
      k_finalize_resid<<<1, 1, 0, s>>>(c->st);
      return cudaGetLastError();
    }
    if (e != cudaErrorNotSupported) return e;
  }
  k_apply<<<ew_grid(c, (const void*)k_apply, nq), NT, 0, s>>>(nq, c->x, c->xf, nullptr, c->st, 0);
  const Lay L = layout(c, nq, c->m_q, REACH_JACOBI_MIXED);
  if (L.seg && (e = seg_plan(c)) != cudaSuccess) return e;
  const int k = c->tune.k;
  e = run_loop(c, c->g_exec[1], c->g_key[1], shape_key(c, L, k), [&](cudaStream_t cs, cudaGraphConditionalHandle, int) {
    if (L.seg) seg_resid_hilo(c, &c->st->slot[0], cs);
    else LAY_DISPATCH(L, l_resid_mixed, c, 0, cs, &c->st->rowctr[0]);
    k_check_mixed<<<1, 1, 0, cs>>>(c->st, 0, k);
    // k - 1 FP32 sweeps: dl[1] -> dl[0] -> dl[1] ... ; k even, so the last lands in dl[0]
    for (int j = 1; j < k; ++j) {
      const float* din = (j & 1) ? c->dl[1] : c->dl[0];
      float* dout = (j & 1) ? c->dl[0] : c->dl[1];
      if (L.seg) seg_sweep32(c, din, dout, cs);
      else if (L.tma) sweep32_tma(c, din, dout, cs, &c->st->rowctr[j]);
      else if (L.smx) sweep32_smem(c, din, dout, cs, &c->st->rowctr[j]);
      else LAY_DISPATCH(L, l_sweep32, c, din, dout, cs, &c->st->rowctr[j]);
    }
    k_apply<<<ew_grid(c, (const void*)k_apply, nq), NT, 0, cs>>>(nq, c->x, c->xf, c->dl[0], c->st, k);
  });
  if (e != cudaSuccess) return e;
  Sys y{nq, c->a_rowptr, c->a_col, c->a_val, c->b};
  const Lay LR = row_layout(c, REACH_JACOBI_MIXED);
  LAY_DISPATCH(LR, l_resid, c, y, c->x, s);
  k_finalize_resid<<<1, 1, 0, s>>>(c->st);
  return cudaGetLastError();
}

// FP64 max|b - (I - A) x| of the final iterate into SolveState::resid.
cudaError_t residual_report(reach_ctx* c, const double* xq) {
  const Lay L = row_layout(c, REACH_JACOBI_FP64);
  Sys y{c->n_q, c->a_rowptr, c->a_col, c->a_val, c->b};
  LAY_DISPATCH(L, l_resid, c, y, xq, c->stream);
  k_finalize_resid<<<1, 1, 0, c->stream>>>(c->st);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ norm bounds (host side)

static double key_to_double(unsigned long long k) {
  const unsigned long long u = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  double v;
  std::memcpy(&v, &u, sizeof(v));
  return v;
}

// Launches k_row_lower over the system (or its transpose) and reads back the minimum
// lower bound and (for w) the largest w_i.  Synchronises the context stream.
static cudaError_t row_lower(reach_ctx* c, bool transposed, const double* w, double* lo_min, double* w_max) {
  const int64_t nq = c->n_q;
  const int64_t* rp = transposed ? c->at_rowptr : c->a_rowptr;
  const int32_t* ci = transposed ? c->at_col : c->a_col;
  const double* av = transposed ? c->at_val : c->a_val;
  cudaStream_t s = c->stream;
  unsigned long long keys[2] = {~0ull, 0ull};
  cudaError_t e = cudaMemcpyAsync(c->keys, keys, sizeof(keys), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  const int g = solver_group(nq, c->m_q);   // the transpose has the same entries
#define KL(G)                                                                                            \
  do {                                                                                                   \
    if (w) {                                                                                             \
      const int grid = grid_rows(c, (const void*)k_row_lower<G, false>, NT, G, nq);                     \
      k_row_lower<G, false><<<grid, NT, 0, s>>>(nq, rp, ci, av, c->d, w, c->keys, c->keys + 1);          \
    } else {                                                                                             \
      const int grid = grid_rows(c, (const void*)k_row_lower<G, true>, NT, G, nq);                       \
      k_row_lower<G, true><<<grid, NT, 0, s>>>(nq, rp, ci, av, c->d, nullptr, c->keys, c->keys + 1);     \
    }                                                                                                    \
  } while (0)
  switch (g) {
    case 1: KL(1); break;
    case 2: KL(2); break;
    case 4: KL(4); break;
    case 8: KL(8); break;
    case 16: KL(16); break;
    default: KL(32); break;
  }
#undef KL
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(keys, c->keys, sizeof(keys), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  const double lo = key_to_double(keys[0]);
  *lo_min = lo == lo ? lo : -INFINITY;
  if (w_max) {
    const double wm = key_to_double(keys[1]);
    *w_max = wm == wm ? wm : INFINITY;
  }
  return cudaSuccess;
}

// ||M^-1||_inf <= 1 / min_i (|d_i| - sum_j |A_ij|) when that margin is positive (Varah);
// +inf otherwise.  Over the rows of the transpose, the same bound for ||M^-T||_inf.
cudaError_t varah_norm_bound(reach_ctx* c, bool transposed, double* kinv) {
  if (c->n_q == 0) {
    *kinv = 0.0;
    return cudaSuccess;
  }
  double margin = 0.0;
  cudaError_t e;
  if (!transposed && c->varah_key) {   // reduced by the extraction
    unsigned long long k = 0ull;
    e = cudaMemcpyAsync(&k, c->keys + VARAH_KEY, sizeof(k), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return e;
    const double lo = key_to_double(k);
    margin = lo == lo ? lo : -INFINITY;
  } else if ((e = row_lower(c, transposed, nullptr, &margin, nullptr)) != cudaSuccess) {
    return e;
  }
  *kinv = margin > 0.0 ? std::nextafter(1.0 / margin, INFINITY) : INFINITY;
  return cudaSuccess;
}

// The right-hand side of (I - A) tau = 1 in place of b (and 1 / d in place of bj), the
// system's own saved in c->tau_save; tau_rhs_end puts them back.
cudaError_t tau_rhs_begin(reach_ctx* c) {
  const int64_t nq = c->n_q;
  cudaStream_t s = c->stream;
  cudaError_t e = cudaMemcpyAsync(c->tau_save, c->b, sizeof(double) * nq, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->tau_save + nq, c->bj, sizeof(double) * nq, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  k_fill_tau_rhs<<<ew_grid(c, (const void*)k_fill_tau_rhs, nq), NT, 0, s>>>(nq, c->d, c->b, c->bj);
  return cudaGetLastError();
}

cudaError_t tau_rhs_end(reach_ctx* c) {
  const int64_t nq = c->n_q;
  cudaStream_t s = c->stream;
  cudaError_t e = cudaMemcpyAsync(c->b, c->tau_save, sizeof(double) * nq, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->bj, c->tau_save + nq, sizeof(double) * nq, cudaMemcpyDeviceToDevice, s);
  return e;
}

// From an approximate tau' (any vector): c = min_i (M tau')_i, bounded from below with
// directed rounding; if c > 0 then ||M^-1||_inf <= max_i tau'_i / c for the chain's
// M-matrix (M^-1 >= 0 entrywise, so tau = M^-1 1 <= tau' / c).  +inf otherwise.
cudaError_t tau_norm_bound(reach_ctx* c, const double* tau, double* kinv) {
  double cmin = 0.0, tmax = 0.0;
  const cudaError_t e = row_lower(c, false, tau, &cmin, &tmax);
  if (e != cudaSuccess) return e;
  *kinv = (cmin > 0.0 && tmax > 0.0 && std::isfinite(tmax)) ? std::nextafter(tmax / cmin, INFINITY) : INFINITY;
  return cudaSuccess;
}

// BiCGStab iterations on the system y from x (x holds the start), the loop graph cached
// in slot gs.  Entry-balanced products (LS.seg) serve the chain's own system only.
static cudaError_t bicgstab_loop(reach_ctx* c, const Sys& y, double* x, const Lay& LS, const Lay& L, int gs) {
  cudaStream_t s = c->stream;
  const int64_t nq = y.nq;
  cudaError_t e = cudaSuccess;
  if (LS.seg && (e = seg_plan(c)) != cudaSuccess) return e;
  LAY_DISPATCH(L, l_bi_init, c, y, x, s);
  // entry-balanced products write y = A u into x2 (free during BiCGStab); the M u epilogue
  // with its fused dots is then elementwise
  e = run_loop(c, c->g_exec[gs], c->g_key[gs], shape_key(c, LS, 1) * 2 + (gs == 2 ? 0 : 1),
               [&](cudaStream_t cs, cudaGraphConditionalHandle, int) {
    k_bi_p<<<ew_grid(c, (const void*)k_bi_p, nq), NT, 0, cs>>>(nq, c->vr, c->vp, c->vv, c->vq, c->bi, c->st);
    if (LS.seg) {
      seg_spmv64(c, c->vp, c->x2, cs);
      k_bi_v_ew<<<ew_grid(c, (const void*)k_bi_v_ew, nq), NT, 0, cs>>>(nq, c->d, c->vp, c->x2, c->vq, c->vv,
                                                                       c->part, c->ticket, c->bi, c->st);
    } else {
      LAY_DISPATCH(L, l_bi_v, c, y, cs);
    }
    k_bi_s<<<ew_grid(c, (const void*)k_bi_s, nq), NT, 0, cs>>>(nq, c->vr, c->vv, c->vs, c->bi, c->st);
    if (LS.seg) {
      seg_spmv64(c, c->vs, c->x2, cs);
      k_bi_t_ew<<<ew_grid(c, (const void*)k_bi_t_ew, nq), NT, 0, cs>>>(nq, c->d, c->vs, c->x2, c->vt, c->part,
                                                                       c->ticket, c->bi, c->st);
    } else {
      LAY_DISPATCH(L, l_bi_t, c, y, cs);
    }
    k_bi_x<<<ew_grid(c, (const void*)k_bi_x, nq), NT, 0, cs>>>(nq, x, c->vp, c->vs, c->vt, c->vr, c->vq,
                                                               c->part, c->ticket, c->bi, c->st);
  });
  if (e != cudaSuccess) return e;
  LAY_DISPATCH(L, l_resid, c, y, x, s);
  k_finalize_resid<<<1, 1, 0, s>>>(c->st);
  return cudaGetLastError();
}

cudaError_t solve_bicgstab(reach_ctx* c, const double* x0q) {
  cudaStream_t s = c->stream;
  const int64_t nq = c->n_q;
  if (x0q) cudaMemcpyAsync(c->x, x0q, sizeof(double) * nq, cudaMemcpyDeviceToDevice, s);
  else cudaMemsetAsync(c->x, 0, sizeof(double) * nq, s);
  const Lay LS = layout(c, nq, c->m_q, REACH_BICGSTAB_FP64);
  const Lay L = row_layout(c, REACH_BICGSTAB_FP64);
  Sys y{nq, c->a_rowptr, c->a_col, c->a_val, c->b};
  return bicgstab_loop(c, y, c->x, LS, L, 2);
}

// The adjoint system (I - A)^T y = e with BiCGStab (§3.2 on the transpose): row j of the
// transpose holds A_ij, the diagonal is the same d, the right-hand side e is in c->at_b;
// the solution goes to c->x2, from y = 0.
cudaError_t solve_bicgstab_transposed(reach_ctx* c) {
  const int64_t nq = c->n_q;
  cudaMemsetAsync(c->x2, 0, sizeof(double) * nq, c->stream);
  const Lay L = row_layout(c, -1);
  Sys y{nq, c->at_rowptr, c->at_col, c->at_val, c->at_b};
  return bicgstab_loop(c, y, c->x2, L, L, 8);
}

void launch_check_mixed(cudaStream_t s, SolveState* st, int slot, int k) {
  k_check_mixed<<<1, 1, 0, s>>>(st, slot, k);
}

void launch_finalize_resid(cudaStream_t s, SolveState* st) { k_finalize_resid<<<1, 1, 0, s>>>(st); }

// ------------------------------------------------------------------ full-state vectors

__global__ void k_scatter(int64_t n, const uint8_t* __restrict__ cls, const int64_t* __restrict__ qidx,
                          const double* __restrict__ xq, double* __restrict__ full) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t k = cls[s];
    full[s] = k == CLS_S1 ? 1.0 : (k == CLS_S0 ? 0.0 : xq[qidx[s]]);
  }
}

__global__ void k_gather(int64_t nq, const int64_t* __restrict__ qstate, const double* __restrict__ full,
                         double* __restrict__ xq) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq;
       i += (int64_t)gridDim.x * blockDim.x)
    xq[i] = full[qstate[i]];
}

cudaError_t scatter_full(reach_ctx* c, const double* xq, double* full) {
  k_scatter<<<ew_grid(c, (const void*)k_scatter, c->n), NT, 0, c->stream>>>(c->n, c->cls, c->qidx, xq, full);
  return cudaGetLastError();
}

cudaError_t gather_q(reach_ctx* c, const double* full, double* xq) {
  if (c->n_q == 0) return cudaSuccess;
  k_gather<<<ew_grid(c, (const void*)k_gather, c->n_q), NT, 0, c->stream>>>(c->n_q, c->qstate, full, xq);
  return cudaGetLastError();
}

// d x_init / d P(s, s') = y_s * x_s' for rows s in S?, 0 elsewhere (input order).
template <int G>
__global__ void k_grad(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                       const uint8_t* __restrict__ cls, const int64_t* __restrict__ qidx,
                       const double* __restrict__ y, const double* __restrict__ xfull,
                       double* __restrict__ g) {
  RowGroups rg = RowGroups::make<G>();
  for (int64_t s = rg.first; s < n; s += rg.stride) {
    const bool q = cls[s] == CLS_SQ;
    const double ys = q ? y[qidx[s]] : 0.0;
    for (int64_t k = rp[s] + rg.lane; k < rp[s + 1]; k += G) g[k] = q ? ys * xfull[col[k]] : 0.0;
  }
}

cudaError_t grad_entries(reach_ctx* c, const double* yq, double* grad) {
  const int g = pick_group(c->n, c->m);
#define KG(G) k_grad<G><<<grid_for(c, (const void*)k_grad<G>, NT, c->n * G), NT, 0, c->stream>>>( \
      c->n, c->rowptr, c->col, c->cls, c->qidx, yq, c->xfull, grad)
  switch (g) {
    case 2: KG(2); break;
    case 4: KG(4); break;
    case 8: KG(8); break;
    case 16: KG(16); break;
    default: KG(32); break;
  }
#undef KG
  return cudaGetLastError();
}

// ------------------------------------------------------------------ autotuner
// Times each row mapping (lanes per row 2..32, or a warp with 16-byte loads) for the
// kernel that dominates `method` on the current system and keeps the fastest.  For FP64
// Jacobi it also picks the sweeps between checks k from the measured sweep time t and
// the check cost c (about the time of two tiny launches): minimising N t + (N / k) c +
// (k / 2) t for N = 1000 sweeps gives k = sqrt(2 N c / t), rounded to an even number.
cudaError_t autotune(reach_ctx* c, int method, int* chosen, float* best_ms) {
  if (c->n_q == 0) {
    *chosen = 0;
    return cudaSuccess;
  }
  cudaError_t e = cudaSuccess;
  if (method == REACH_JACOBI_MIXED) {
    e = split_hilo(c);
    if (e != cudaSuccess) return e;
    // a defined x for the residual candidates (its values do not change their time)
    cudaMemsetAsync(c->x, 0, sizeof(double) * c->n_q, c->stream);
    cudaMemsetAsync(c->xf, 0, sizeof(float) * c->n_q, c->stream);
  }
  // process-wide cache: contexts over the same system shape reuse the measurement
  static std::mutex cache_mu;
  static std::unordered_map<std::string, std::pair<int, float>> cache;
  const std::string key = std::to_string(c->n_q) + "/" + std::to_string(c->m_q) + "/" + std::to_string(method);
  {
    std::lock_guard<std::mutex> lk(cache_mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      const int pick = it->second.first;
      const float best = it->second.second;
      c->tune.gm[method] = pick;
      if (method == REACH_JACOBI_MIXED) c->tune.sweep_u = pick == 66 ? 4 : 2;
      if (method == REACH_JACOBI_FP64) {
        const double check_ms = 0.006, sweeps = 1000.0;
        int k = (int)std::lround(std::sqrt(2.0 * sweeps * check_ms / std::max(1e-4, (double)best)));
        c->tune.k_auto = std::max(2, std::min(62, k + (k & 1)));
      }
      *chosen = pick;
      *best_ms = best;
      return cudaSuccess;
    }
  }
  // a fresh solve state: a finished solve leaves `done` set, and the solve kernels
  // return at once when it is
  {
    SolveState hs;
    std::memset(&hs, 0, sizeof(hs));
    hs.eps = 1e-300;
    hs.max_iter = 1;
    hs.max_bodies = 1;
    e = cudaMemcpyAsync(c->st, &hs, sizeof(hs), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return e;
  }
  // 66: warp + vector loads with four quads per trip (FP32 sweep only); 128: entry-balanced
  // tiles (FP64 Jacobi and the FP32 sweep), which wins when a few rows are very long
  // (LAY_TMA, the FP32 sweep staged by bulk copies, is not a candidate: it measured 1.7x
  // slower than 64 on the dense system, with each row's first segments arriving cold)
  // (LAY_SMX, the FP32 sweep with its vector in shared memory, is opt-in too: on the dense
  // system it measured within 1 % of 64, so the L1 gathers are not what limits that sweep)
  const int codes[10] = {1, 2, 4, 8, 16, 32, LAY_VEC16, 64, 66, LAY_SEG};
  const double mean = (double)c->m_q / (double)c->n_q;
  Sys y{c->n_q, c->a_rowptr, c->a_col, c->a_jv, c->bj};   // Jacobi form (the FP64 sweep)
  cudaStream_t s = c->stream;
  float best = 1e30f;
  int pick = 0;
  for (int code : codes) {
    const Lay L = lay_of(code);
    if (code == 66 && method != REACH_JACOBI_MIXED) continue;
    if (L.smx && (method != REACH_JACOBI_MIXED || !c->a_col16 || c->n_q > SMX_MAX_ROWS)) continue;
    if (L.seg && (e = seg_plan(c)) != cudaSuccess) return e;
    if (L.vec && !L.seg && mean < 16) continue;  // nothing to vectorise
    if (!L.vec && L.g > 4 * mean + 4) continue;  // mostly idle lanes
    if (!L.vec && L.g == 1 && mean > 8) continue;  // one lane walking long rows
    if (method == REACH_JACOBI_MIXED) c->tune.sweep_u = code == 66 ? 4 : 2;
    unsigned* ctr = &c->st->rowctr[0];
    // the mixed method also times its FP64 residual step (same mapping), which runs once
    // per 16 sweeps: a mapping that speeds up the sweep but slows the residual more loses
    float total = 0.f, total_r = 0.f;
    const int parts = method == REACH_JACOBI_MIXED ? 2 : 1;
    for (int part = 0; part < parts; ++part) {
      for (int rep = 0; rep < 4; ++rep) {
        cudaMemsetAsync(ctr, 0, sizeof(unsigned), s);
        cudaMemsetAsync(&c->st->done, 0, sizeof(int32_t), s);   // a candidate must never see a finished state
        e = cudaEventRecord(c->ev0, s);
        if (part == 1 && L.seg) {
          seg_resid_hilo(c, &c->st->slot[62], s);
        } else if (part == 1) {
          LAY_DISPATCH(L, l_resid_mixed, c, 62, s, ctr);
        } else if (L.tma) {
          e = sweep32_tma(c, c->dl[0], c->dl[1], s, ctr);
          if (e != cudaSuccess) return e;
        } else if (L.smx) {
          e = sweep32_smem(c, c->dl[0], c->dl[1], s, ctr);
          if (e != cudaSuccess) return e;
        } else if (L.seg && method == REACH_JACOBI_MIXED) {
          seg_sweep32(c, c->dl[0], c->dl[1], s);
        } else if (L.seg && method == REACH_BICGSTAB_FP64) {
          seg_spmv64(c, c->b, c->x2, s);
          k_bi_v_ew<<<ew_grid(c, (const void*)k_bi_v_ew, c->n_q), NT, 0, s>>>(c->n_q, c->d, c->b, c->x2, c->b,
                                                                             c->vv, c->part, c->ticket, c->bi,
                                                                             c->st);
        } else if (L.seg) {
          seg_sweep(c, c->x, c->x2, &c->st->slot[62], s);
        } else if (method == REACH_JACOBI_MIXED) {
          LAY_DISPATCH(L, l_sweep32, c, c->dl[0], c->dl[1], s, ctr);
        } else {
          LAY_DISPATCH(L, l_jacobi, c, y, c->x, c->x2, &c->st->slot[62], s, ctr);
        }
        if (e == cudaSuccess) e = cudaEventRecord(c->ev1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(c->ev1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        if (e != cudaSuccess) return e;
        if (rep > 0) (part ? total_r : total) += ms;   // first launch is a warm-up
      }
    }
    const float avg = parts == 2 ? (15.f * total + total_r) / (16.f * 3.f) : total / 3.f;
    if (avg < best) {
      best = avg;
      pick = code;
    }
  }
  if (method == REACH_JACOBI_MIXED) c->tune.sweep_u = pick == 66 ? 4 : 2;
  {
    std::lock_guard<std::mutex> lk(cache_mu);
    cache[key] = {pick, best};
  }
  c->tune.gm[method] = pick;
  if (method == REACH_JACOBI_FP64) {
    const double check_ms = 0.006, sweeps = 1000.0;
    int k = (int)std::lround(std::sqrt(2.0 * sweeps * check_ms / std::max(1e-4, (double)best)));
    k = std::max(2, std::min(62, k + (k & 1)));
    c->tune.k_auto = k;
  }
  *chosen = pick;
  *best_ms = best;
  return cudaSuccess;
}

// Average device time of `launches` back-to-back launches of one solver kernel on the
// context stream, in the layout and row order the solves use (CUDA events on that
// stream).  kernel: 0 FP64 Jacobi sweep, 1 FP32 sweep, 2 FP64 hi+lo residual,
// 3 BiCGStab product v = M p.  The kernels only touch solve workspace.
cudaError_t time_kernel(reach_ctx* c, int kernel, int launches, float* avg_ms) {
  *avg_ms = 0.f;
  if (c->n_q == 0 || launches < 1) return cudaSuccess;
  cudaStream_t s = c->stream;
  cudaError_t e = cudaSuccess;
  if (kernel == 1 || kernel == 2) {
    e = split_hilo(c);
    if (e != cudaSuccess) return e;
    k_apply<<<ew_grid(c, (const void*)k_apply, c->n_q), NT, 0, s>>>(c->n_q, c->x, c->xf, nullptr, c->st, 0);
  }
  const int method = kernel == 0 ? REACH_JACOBI_FP64 : kernel == 3 ? REACH_BICGSTAB_FP64 : REACH_JACOBI_MIXED;
  const Lay L = layout(c, c->n_q, c->m_q, method);
  if (L.seg && (e = seg_plan(c)) != cudaSuccess) return e;
  Sys y{c->n_q, c->a_rowptr, c->a_col, c->a_jv, c->bj};   // Jacobi form (the FP64 sweep)
  Sys ya{c->n_q, c->a_rowptr, c->a_col, c->a_val, c->b};  // the system itself (BiCGStab)
  SolveState hs;
  std::memset(&hs, 0, sizeof(hs));
  hs.eps = 1e-300;
  hs.max_iter = 1;
  hs.max_bodies = 1;
  e = cudaMemcpyAsync(c->st, &hs, sizeof(hs), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  if (kernel == 3) {   // a non-zero shadow vector, so q.v never reads as a breakdown
    e = cudaMemcpyAsync(c->vq, c->b, sizeof(double) * c->n_q, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  auto one = [&](int) {
    unsigned* ctr = &c->st->rowctr[0];
    cudaMemsetAsync(ctr, 0, sizeof(unsigned), s);   // fresh row counter for every launch
    cudaMemsetAsync(&c->st->done, 0, sizeof(int32_t), s);
    if (L.seg && kernel == 0) seg_sweep(c, c->x, c->x2, &c->st->slot[0], s);
    else if (L.seg && kernel == 1) seg_sweep32(c, c->dl[0], c->dl[1], s);
    else if (L.tma && kernel == 1) {
      const cudaError_t le = sweep32_tma(c, c->dl[0], c->dl[1], s, ctr);
      if (le != cudaSuccess) e = le;
    } else if (L.smx && kernel == 1) {
      const cudaError_t le = sweep32_smem(c, c->dl[0], c->dl[1], s, ctr);
      if (le != cudaSuccess) e = le;
    } else if (L.seg && kernel == 2) seg_resid_hilo(c, &c->st->slot[0], s);
    else if (L.seg && kernel == 3) {
      seg_spmv64(c, c->vp, c->x2, s);
      k_bi_v_ew<<<ew_grid(c, (const void*)k_bi_v_ew, c->n_q), NT, 0, s>>>(c->n_q, c->d, c->vp, c->x2, c->vq, c->vv,
                                                                         c->part, c->ticket, c->bi, c->st);
    }
    else if (kernel == 0) LAY_DISPATCH(L, l_jacobi, c, y, c->x, c->x2, &c->st->slot[0], s, ctr);
    else if (kernel == 1) LAY_DISPATCH(L, l_sweep32, c, c->dl[0], c->dl[1], s, ctr);
    else if (kernel == 2) LAY_DISPATCH(L, l_resid_mixed, c, 0, s, ctr);
    else LAY_DISPATCH(L, l_bi_v, c, ya, s);
  };
  one(0);  // warm-up
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(c->ev0, s);
  for (int j = 1; j <= launches && e == cudaSuccess; ++j) one(j);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(c->ev1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  if (e == cudaSuccess) e = cudaGetLastError();
  *avg_ms = ms / (float)launches;
  return e;
}

}  // namespace reach
