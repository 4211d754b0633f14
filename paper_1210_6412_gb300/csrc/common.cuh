// Device helpers shared by the solver kernels: warp / block reductions, the
// "last CTA finishes the reduction" pattern, and the row-group mapping used by
// every CSR kernel (G lanes of a warp own one row; G in {2,4,8,16,32}).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define RDEV __device__ __forceinline__

namespace reach {

constexpr unsigned FULL = 0xffffffffu;

template <int G, typename T>
RDEV T group_sum(T v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

template <typename T>
RDEV T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, o));
  return v;
}

template <typename T>
RDEV T warp_sum(T v) { return group_sum<32>(v); }

// Sum over a group of G lanes with every addition rounded upward: an upper bound of the
// exact sum of the lanes' values.
template <int G>
RDEV double group_sum_ru(double v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = __dadd_ru(v, __shfl_xor_sync(FULL, v, o));
  return v;
}

// Order-preserving map of doubles onto unsigned integers (for atomicMin / atomicMax of
// values of either sign).
RDEV unsigned long long ordered_key(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// Block-wide reduction of NV doubles (sum or max).  Result valid in thread 0.
// `sh` needs NV * 32 doubles.  Fixed order, so the result is deterministic.
template <int NV, bool MAX>
RDEV void block_reduce(double (&v)[NV], double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) v[j] = MAX ? warp_max(v[j]) : warp_sum(v[j]);
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) sh[j * 32 + w] = v[j];
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double t = lane < nw ? sh[j * 32 + lane] : 0.0;
      v[j] = MAX ? warp_max(t) : warp_sum(t);
    }
  }
  __syncthreads();
}

// FP32 -> FP64 widening with integer arithmetic only.  On GB300 the conversion
// instruction shares the (narrow) FP64 pipe, while this bit rearrangement runs on the
// integer units.  Exact for finite normal numbers and zero; FP32 subnormals (below
// 1.2e-38) become signed zero.  Inputs are finite (validated matrix values split into
// FP32 hi + lo).  No branch or select: those compiled into per-element control flow.
RDEV double widen(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  const uint32_t nz = (e + 255u) >> 8;              // 1 unless zero / subnormal, without a predicate
  const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
  const uint64_t ex = (uint64_t)((e + 896u) * nz);
  const uint64_t mant = (uint64_t)((u & 0x7fffffu) * nz) << 29;
  return __longlong_as_double((long long)(sign | (ex << 52) | mant));
}

// Max of non-negative doubles through the integer order of their bit patterns.
RDEV void atomic_max_nonneg(unsigned long long* slot, double v) {
  if (v > 0.0) atomicMax(slot, (unsigned long long)__double_as_longlong(v));
}
RDEV double slot_value(const unsigned long long* slot) {
  return __longlong_as_double((long long)__ldcg(slot));
}

// Deterministic grid reduction: every CTA stores its partials (NV doubles) in
// part[NV * gridDim.x]; the CTA that arrives last sums them in a fixed order.
// Returns true in every thread of the last CTA, with tot[] valid in thread 0.
// No CTA waits on another, so this cannot hang.
template <int NV>
RDEV bool last_cta_sum(const double (&mine)[NV], double* part, unsigned* ticket,
                       double (&tot)[NV], double* sh) {
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) part[j * gridDim.x + blockIdx.x] = mine[j];
    __threadfence();
    unsigned t = atomicAdd(ticket, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double s = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) s += __ldcg(part + j * gridDim.x + b);
    tot[j] = s;
  }
  block_reduce<NV, false>(tot, sh);
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// Warp-uniform iteration over rows with G lanes per row: every lane of a warp
// runs the same number of trips, so group shuffles are always convergent.
struct RowGroups {
  int64_t first, stride;  // in units of rows
  int lane;               // lane within the group
  template <int G>
  RDEV static RowGroups make() {
    RowGroups r;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    r.first = gtid / G;
    r.stride = (int64_t)gridDim.x * blockDim.x / G;
    r.lane = threadIdx.x & (G - 1);
    return r;
  }
};

// Row loop bound that is equal for all lanes of a warp: the row of lane 0 of the
// warp decides whether the warp runs another trip.
template <int G>
RDEV bool warp_has_row(int64_t row, int64_t nrows) {
  const int64_t warp_first = row - ((threadIdx.x & 31) / G);
  return warp_first < nrows;
}

// Row order of a kernel.  Static: groups take rows first, first + stride, ...
// Dynamic (warp per row, ctr != nullptr): each warp takes the next row from a
// counter in device memory, so warps that drew short rows take more of them and all
// SMs stay busy until the last rows (the counter must be 0 at launch).
RDEV int64_t warp_fetch_row(unsigned* ctr) {
  unsigned r = 0;
  if ((threadIdx.x & 31) == 0) r = atomicAdd(ctr, 1u);
  return (int64_t)__shfl_sync(FULL, r, 0);
}
template <int G>
RDEV int64_t row_begin(const RowGroups& rg, unsigned* ctr) {
  if constexpr (G == 32) {
    if (ctr) return warp_fetch_row(ctr);
  }
  return rg.first;
}
template <int G>
RDEV int64_t row_next(const RowGroups& rg, unsigned* ctr, int64_t i) {
  if constexpr (G == 32) {
    if (ctr) return warp_fetch_row(ctr);
  }
  return i + rg.stride;
}

}  // namespace reach
