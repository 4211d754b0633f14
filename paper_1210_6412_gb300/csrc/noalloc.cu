// Allocation-free Jacobi solve of an already extracted system (I - A) x = b.
//
// Some callers cannot call cudaMalloc: code that runs inside a host application which
// owns the device memory through its own pool and forbids outside allocations, code on
// a latency-critical path where cudaMalloc / cudaFree would synchronise the device, or
// code that must not fail with out-of-memory once it has started.  The regular entry
// points allocate per-context buffers; this one takes every input and output from the
// caller and keeps its only scratch -- the second Jacobi vector and one reduction word
// -- in a fixed device array compiled into the library.
#include <algorithm>
#include <cstring>
#include <string>

#include "common.cuh"
#include "internal.h"

namespace {

using namespace reach;

// Largest system this entry point accepts, and the size of its scratch array:
// 4 KiB of header plus one float64 per unknown (4 MiB + 4 KiB in total).
constexpr int64_t NOALLOC_MAX_ROWS = int64_t(1) << 19;
constexpr size_t NOALLOC_HEADER = 4096;
constexpr size_t NOALLOC_BYTES = NOALLOC_HEADER + sizeof(double) * (size_t)NOALLOC_MAX_ROWS;

// Device-resident scratch shared by every call on a device.  Each GPU that loads the
// library holds it until the process exits.  Host code must not use the symbol as an
// address: the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

__global__ void k_na_clear(unsigned long long* dmax) { *dmax = 0ull; }

// One Jacobi sweep x' = (b + A x) / d with max|x' - x| folded into *dmax.
template <int G>
__global__ void __launch_bounds__(256) k_na_sweep(int64_t nq, const int64_t* __restrict__ rp,
                                                  const int32_t* __restrict__ ci,
                                                  const double* __restrict__ av,
                                                  const double* __restrict__ b,
                                                  const double* __restrict__ d,
                                                  const double* __restrict__ x,
                                                  double* __restrict__ xn, unsigned long long* dmax) {
  RowGroups rg = RowGroups::make<G>();
  double mx = 0.0;
  for (int64_t i = rg.first; warp_has_row<G>(i, nq); i += rg.stride) {
    double s = 0.0;
    if (i < nq)
      for (int64_t k = rp[i] + rg.lane; k < rp[i + 1]; k += G) s = fma(av[k], x[ci[k]], s);
    s = group_sum<G>(s);
    if (i < nq && rg.lane == 0) {
      const double xv = (b[i] + s) / d[i];
      const double dx = fabs(xv - x[i]);
      mx = fmax(mx, dx != dx ? __longlong_as_double(0x7ff0000000000000LL) : dx);
      xn[i] = xv;
    }
  }
  __shared__ double sh[32];
  double a[1] = {mx};
  block_reduce<1, true>(a, sh);
  if (threadIdx.x == 0) atomic_max_nonneg(dmax, a[0]);
}

template <int G>
void na_sweep(int grid, cudaStream_t s, int64_t nq, const int64_t* rp, const int32_t* ci,
              const double* av, const double* b, const double* d, const double* x, double* xn,
              unsigned long long* dmax) {
  k_na_sweep<G><<<grid, 256, 0, s>>>(nq, rp, ci, av, b, d, x, xn, dmax);
}

// Device address of the scratch array on the current device.  Looked up on every call:
// the lookup is cheap and allocates nothing, and a cached pointer would go stale after a
// cudaDeviceReset (new context) or point into another device's copy.
cudaError_t scratch_on_current_device(unsigned char** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<unsigned char*>(p);
  return cudaSuccess;
}

reach_status na_cuda_fail(cudaError_t e, const char* what) {
  set_err(nullptr, std::string("reach_jacobi_solve_noalloc: ") + what + ": " + cudaGetErrorString(e));
  return REACH_ECUDA;
}

}  // namespace

extern "C" reach_status reach_jacobi_solve_noalloc(int64_t n_q, const int64_t* rowptr, const int32_t* col,
                                                  const double* val, const double* b, const double* d,
                                                  double eps, int64_t max_iter, int32_t check_every,
                                                  double* x, int64_t* iters_out, double* delta_out,
                                                  void* stream) {
  if (n_q < 1 || n_q > NOALLOC_MAX_ROWS) {
    set_err(nullptr, "reach_jacobi_solve_noalloc: n_q must be in [1, 524288] (the size of the built-in scratch)");
    return REACH_EINVAL;
  }
  if (!rowptr || !col || !val || !b || !d || !x) {
    set_err(nullptr, "reach_jacobi_solve_noalloc: NULL device pointer");
    return REACH_EINVAL;
  }
  if (!(eps > 0.0) || max_iter < 1 || check_every < 2 || (check_every & 1)) {
    set_err(nullptr, "reach_jacobi_solve_noalloc: need eps > 0, max_iter >= 1, check_every even >= 2");
    return REACH_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_cuda_fail(e, "current device");
  // the scratch used is the current device's copy: the stream must belong to that device
  int sdev = dev;
  e = cudaStreamGetDevice(s, &sdev);
  if (e != cudaSuccess) return na_cuda_fail(e, "stream device");
  if (sdev != dev) {
    set_err(nullptr, "reach_jacobi_solve_noalloc: the stream belongs to another device than the current one");
    return REACH_EINVAL;
  }
  unsigned char* base = nullptr;
  e = scratch_on_current_device(&base);
  if (e != cudaSuccess) return na_cuda_fail(e, "scratch lookup");
  unsigned long long* dmax = reinterpret_cast<unsigned long long*>(base);
  double* xn = reinterpret_cast<double*>(base + NOALLOC_HEADER);
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return na_cuda_fail(e, "device attribute");
  int64_t nnz = 0;
  e = cudaMemcpyAsync(&nnz, rowptr + n_q, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return na_cuda_fail(e, "reading rowptr[n_q]");
  const int g = pick_group(n_q, nnz);
  const int64_t blocks = (n_q * g + 255) / 256;
  const int grid = (int)std::min<int64_t>(blocks, (int64_t)sms * 8);
  int64_t it = 0;
  double delta = 0.0;
  reach_status status = REACH_ENOTCONV;
  while (it < max_iter) {
    // a window of check_every sweeps, the last one shortened so that exactly max_iter
    // sweeps run at most; the window's last sweep computes max|x' - x|
    const int w = (int)std::min<int64_t>(check_every, max_iter - it);
    for (int j = 0; j < w; ++j) {
      const double* xi = (j & 1) ? xn : x;
      double* xo = (j & 1) ? x : xn;
      if (j == w - 1) k_na_clear<<<1, 1, 0, s>>>(dmax);
      switch (g) {
        case 2: na_sweep<2>(grid, s, n_q, rowptr, col, val, b, d, xi, xo, dmax); break;
        case 4: na_sweep<4>(grid, s, n_q, rowptr, col, val, b, d, xi, xo, dmax); break;
        case 8: na_sweep<8>(grid, s, n_q, rowptr, col, val, b, d, xi, xo, dmax); break;
        case 16: na_sweep<16>(grid, s, n_q, rowptr, col, val, b, d, xi, xo, dmax); break;
        default: na_sweep<32>(grid, s, n_q, rowptr, col, val, b, d, xi, xo, dmax); break;
      }
    }
    // an odd window leaves the newest iterate in the scratch vector: copy it back
    if (w & 1) e = cudaMemcpyAsync(x, xn, sizeof(double) * (size_t)n_q, cudaMemcpyDeviceToDevice, s);
    // a launch that failed without a sticky error would otherwise leave x untouched and
    // the reduction word at the previous call's value
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return na_cuda_fail(e, "sweep launch");
    it += w;
    unsigned long long bits = 0;
    e = cudaMemcpyAsync(&bits, dmax, sizeof(bits), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return na_cuda_fail(e, "reading max|x' - x|");
    std::memcpy(&delta, &bits, sizeof(delta));
    if (delta < eps) {
      status = REACH_OK;
      break;
    }
  }
  if (iters_out) *iters_out = it;
  if (delta_out) *delta_out = delta;
  if (status != REACH_OK) set_err(nullptr, "reach_jacobi_solve_noalloc: max_iter reached before max|x' - x| < eps");
  return status;
}
