// Parametric chains: P_e = softmax over the out-edges of a row of
// theta[class_e] + offset_e, and the chain rule from dx_init/dP to dx_init/dtheta.
#include <cfloat>
#include <string>

#include "common.cuh"
#include "internal.h"

namespace reach {

template <int G>
RDEV double group_max(double v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, o));
  return v;
}

// Logit of entry k; a class outside [0, nc) yields NaN, which reach_create rejects.
RDEV double logit(const int32_t* __restrict__ cls, const double* __restrict__ off,
                  const double* __restrict__ theta, int nc, int64_t k) {
  const int32_t c = cls[k];
  return (unsigned)c < (unsigned)nc ? theta[c] + off[k] : __longlong_as_double(0x7ff8000000000000LL);
}

template <int G>
__global__ void k_softmax(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ cls,
                          const double* __restrict__ off, const double* __restrict__ theta, int nc,
                          double* __restrict__ p) {
  RowGroups rg = RowGroups::make<G>();
  for (int64_t s = rg.first; warp_has_row<G>(s, n); s += rg.stride) {
    const bool act = s < n;
    const int64_t lo = act ? rp[s] : 0, hi = act ? rp[s + 1] : 0;
    double mx = -DBL_MAX;
    for (int64_t k = lo + rg.lane; k < hi; k += G) mx = fmax(mx, logit(cls, off, theta, nc, k));
    mx = group_max<G>(mx);
    double sum = 0.0;
    for (int64_t k = lo + rg.lane; k < hi; k += G) sum += exp(logit(cls, off, theta, nc, k) - mx);
    sum = group_sum<G>(sum);
    for (int64_t k = lo + rg.lane; k < hi; k += G) p[k] = exp(logit(cls, off, theta, nc, k) - mx) / sum;
  }
}

// Per-CTA class bins: bins[blockIdx.x * C + c] = sum over this CTA's rows of
// dl_f = P_f (g_f - sum_e P_e g_e) for edges f of class c.
template <int G>
__global__ void k_softmax_grad(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ cls,
                               const double* __restrict__ p, const double* __restrict__ gp, int nc,
                               double* __restrict__ bins) {
  extern __shared__ double sb[];
  for (int j = threadIdx.x; j < nc; j += blockDim.x) sb[j] = 0.0;
  __syncthreads();
  RowGroups rg = RowGroups::make<G>();
  for (int64_t s = rg.first; warp_has_row<G>(s, n); s += rg.stride) {
    const bool act = s < n;
    const int64_t lo = act ? rp[s] : 0, hi = act ? rp[s + 1] : 0;
    double inner = 0.0;
    for (int64_t k = lo + rg.lane; k < hi; k += G) inner = fma(p[k], gp[k], inner);
    inner = group_sum<G>(inner);
    for (int64_t k = lo + rg.lane; k < hi; k += G) {
      const int32_t c = cls[k];
      if ((unsigned)c < (unsigned)nc) atomicAdd(sb + c, p[k] * (gp[k] - inner));
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nc; j += blockDim.x) bins[(int64_t)blockIdx.x * nc + j] = sb[j];
}

__global__ void k_bins_sum(int nb, int nc, const double* __restrict__ bins, double* __restrict__ out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nc; j += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += bins[(int64_t)b * nc + j];
    out[j] = s;
  }
}

}  // namespace reach

using namespace reach;

namespace {
int sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}
}  // namespace

extern "C" {

reach_status reach_param_probs(int64_t n, int64_t m, const int64_t* rowptr, const int32_t* cls,
                               const double* offset, const double* theta, int32_t n_classes,
                               double* p_out, void* stream) {
  if (n < 1 || m < 1 || !rowptr || !cls || !offset || !theta || !p_out || n_classes < 1) {
    set_err(nullptr, "reach_param_probs: bad arguments");
    return REACH_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int g = pick_group(n, m);
  const int grid = sms() * 8;
#define SM(G) k_softmax<G><<<grid, 256, 0, s>>>(n, rowptr, cls, offset, theta, n_classes, p_out)
  switch (g) {
    case 2: SM(2); break;
    case 4: SM(4); break;
    case 8: SM(8); break;
    case 16: SM(16); break;
    default: SM(32); break;
  }
#undef SM
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_err(nullptr, std::string("reach_param_probs: ") + cudaGetErrorString(e));
    return REACH_ECUDA;
  }
  return REACH_OK;
}

reach_status reach_param_grad_theta(int64_t n, int64_t m, const int64_t* rowptr, const int32_t* cls,
                                    const double* p, const double* g_p, int32_t n_classes,
                                    double* g_theta, void* stream) {
  if (n < 1 || m < 1 || !rowptr || !cls || !p || !g_p || !g_theta || n_classes < 1 || n_classes > 4096) {
    set_err(nullptr, "reach_param_grad_theta: bad arguments (n_classes must be in [1, 4096])");
    return REACH_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = sms() * 4;
  double* bins = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&bins, sizeof(double) * (size_t)grid * n_classes, s);
  if (e != cudaSuccess) {
    set_err(nullptr, std::string("reach_param_grad_theta: ") + cudaGetErrorString(e));
    return REACH_ENOMEM;
  }
  const size_t shm = sizeof(double) * (size_t)n_classes;
  const int g = pick_group(n, m);
#define SG(G) k_softmax_grad<G><<<grid, 256, shm, s>>>(n, rowptr, cls, p, g_p, n_classes, bins)
  switch (g) {
    case 2: SG(2); break;
    case 4: SG(4); break;
    case 8: SG(8); break;
    case 16: SG(16); break;
    default: SG(32); break;
  }
#undef SG
  k_bins_sum<<<(n_classes + 127) / 128, 128, 0, s>>>(grid, n_classes, bins, g_theta);
  cudaFreeAsync(bins, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_err(nullptr, std::string("reach_param_grad_theta: ") + cudaGetErrorString(e));
    return REACH_ECUDA;
  }
  return REACH_OK;
}

}  // extern "C"
