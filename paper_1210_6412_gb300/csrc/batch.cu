// Batched multi-RHS reachability: K <= 8 goal sets over one chain (typically the
// block-diagonal union of many independent chains).  Each right-hand side j has
// its own partition S=0_j / S=1_j / S?_j (§2.2); one pass over the matrix serves all
// K of them.  The partition is a bit-parallel fixed point (bit j of a state's byte
// belongs to goal set j).  The solve is the masked Jacobi iteration on the full P:
//   x_j[s] = (sum_{s' != s} P(s,s') x_j[s']) / (1 - P(s,s))   for s in S?_j,
// with x_j fixed to 1 on S=1_j and 0 on S=0_j, which is the system of §2.3 for each j
// (b enters through the fixed ones).  It runs as FP32 sweeps with an FP64 residual and
// correction every k sweeps, all inside one conditional-while CUDA graph.
#include <cstring>
#include <string>

#include "common.cuh"
#include "internal.h"

using namespace reach;

struct reach_batch {
  reach_ctx* base = nullptr;   // holds P, validation, the all-rows extraction, scratch
  int k = 0;
  uint8_t* gbits = nullptr;    // bit j: goal of set j
  uint8_t* rbits = nullptr;    // bit j: can reach GS_j
  uint8_t* bbits = nullptr;    // bit j: reaches S=0_j along a path avoiding GS_j
  uint8_t* sq = nullptr;       // bit j: in S?_j
  uint8_t* one = nullptr;      // bit j: in S=1_j
  double* X = nullptr;         // [n][8] FP64
  float* R = nullptr;          // [n][8] FP32 residual
  float* D[2] = {nullptr, nullptr};  // [n][8] FP32 corrections
  unsigned* changed = nullptr;
  bool have_classes = false;
  cudaGraphExec_t g_exec[3] = {nullptr, nullptr, nullptr};
  int64_t g_key[3] = {-1, -1, -1};
  int64_t passes[2] = {0, 0};
};

namespace reach {

constexpr int BT = 256;

__global__ void k_goal_bits(int64_t n, int k, const uint8_t* __restrict__ goals, uint8_t* __restrict__ g) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    unsigned b = 0;
    for (int j = 0; j < k; ++j) b |= (goals[(int64_t)j * n + s] != 0 ? 1u : 0u) << j;
    g[s] = (uint8_t)b;
  }
}

template <int G>
RDEV unsigned group_or(unsigned v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v |= __shfl_xor_sync(FULL, v, o);
  return v;
}

// One pull pass of a backward-reachability fixed point, all K sets at once:
// bits[s] |= allow(s) & OR over successors s' (P(s,s') > 0) of bits[s'].
// allow(s) = ~block[s] (block = goal bits for the S=1 search, none for S=0).
// Updates land in place; the fixed point is monotone, so stale reads only delay it.
template <int G>
__global__ void k_pull_or(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                          const double* __restrict__ val, uint8_t* bits, const uint8_t* __restrict__ block,
                          unsigned kmask, unsigned* changed) {
  RowGroups rg = RowGroups::make<G>();
  bool any = false;
  for (int64_t s = rg.first; warp_has_row<G>(s, n); s += rg.stride) {
    unsigned acc = 0;
    if (s < n) {
      for (int64_t k = rp[s] + rg.lane; k < rp[s + 1]; k += G)
        if (val[k] > 0.0) acc |= *(volatile const uint8_t*)(bits + col[k]);
    }
    acc = group_or<G>(acc);
    if (s < n && rg.lane == 0) {
      const unsigned allow = block ? (~(unsigned)block[s] & kmask) : kmask;
      const unsigned old = bits[s];
      const unsigned add = acc & allow & ~old;
      if (add) {
        bits[s] = (uint8_t)(old | add);
        any = true;
      }
    }
  }
  if (any) *changed = 1u;
}

__global__ void k_fix_ctl(unsigned* changed, int64_t* passes, int64_t max_passes,
                          cudaGraphConditionalHandle h, int use_cond) {
  const unsigned c = *changed;
  *changed = 0u;
  *passes += 1;
  const bool more = c != 0u && *passes < max_passes;
  if (use_cond) cudaGraphSetConditional(h, more ? 1u : 0u);
}

__global__ void k_batch_classes(int64_t n, int mode, unsigned kmask, const uint8_t* __restrict__ g,
                                const uint8_t* __restrict__ r, const uint8_t* __restrict__ bb,
                                uint8_t* __restrict__ sq, uint8_t* __restrict__ one,
                                double* __restrict__ X) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    const unsigned s0 = ~(unsigned)r[s] & kmask;
    const unsigned s1 = mode == REACH_PROB01 ? (~(unsigned)bb[s] & kmask) : ((unsigned)g[s] & kmask);
    const unsigned q = kmask & ~s0 & ~s1;
    sq[s] = (uint8_t)q;
    one[s] = (uint8_t)s1;
#pragma unroll
    for (int j = 0; j < 8; ++j) X[s * 8 + j] = (s1 >> j) & 1u ? 1.0 : 0.0;
  }
}

__global__ void k_not_bits(int64_t n, const uint8_t* __restrict__ src, uint8_t* __restrict__ dst,
                           unsigned kmask) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x)
    dst[s] = (uint8_t)(~(unsigned)src[s] & kmask);
}

// x_j = 1 on S=1_j, 0 elsewhere (the iteration starts from 0 on S?_j).
__global__ void k_batch_init_x(int64_t n, const uint8_t* __restrict__ one, double* __restrict__ X) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * 8;
       i += (int64_t)gridDim.x * blockDim.x)
    X[i] = (one[i >> 3] >> (i & 7)) & 1u ? 1.0 : 0.0;
}

// Row mapping of the multi-RHS kernels: a group of lanes owns a row and each lane owns
// some of the right-hand sides, so every lane walks the whole row and no cross-lane
// reduction is needed (which matters most in FP64, whose pipe is narrow).

// FP64 residual of every right-hand side on the Jacobi form (values A_sj / d_s, read in
// FP64): r_j = sum_{s'} Aj(s,s') x_j[s'] - x_j[s] on S?_j, 0 elsewhere; r_j is also the
// first correction.  REPORT: only max|d_s r_j| (the residual of the system itself) into
// the slot, after the loop.  Two lanes own a row, lane h the right-hand sides 4h .. 4h+3,
// gathering two double2 of the 64-byte row of X per entry.
template <bool REPORT>
__global__ void __launch_bounds__(BT) k_bresid(int64_t n, const int64_t* __restrict__ rp,
                                               const int32_t* __restrict__ ci, const double* __restrict__ aj,
                                               const double* __restrict__ d, const uint8_t* __restrict__ sq,
                                               const double* __restrict__ X, float* __restrict__ R,
                                               float* __restrict__ D1, SolveState* st, int slot) {
  if (!REPORT && st->done) return;
  RowGroups rg = RowGroups::make<2>();
  const int h = rg.lane;                    // right-hand sides 4h .. 4h+3
  double mx = 0.0;
  for (int64_t s = rg.first; s < n; s += rg.stride) {
    const int64_t hi = rp[s + 1];
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t k = rp[s]; k < hi; ++k) {
      const double v = __ldcs(aj + k);
      const double2* xr = reinterpret_cast<const double2*>(X + (int64_t)__ldcs(ci + k) * 8 + 4 * h);
      const double2 t0 = __ldg(xr), t1 = __ldg(xr + 1);
      a[0] = fma(v, t0.x, a[0]);
      a[1] = fma(v, t0.y, a[1]);
      a[2] = fma(v, t1.x, a[2]);
      a[3] = fma(v, t1.y, a[3]);
    }
    const unsigned m = sq[s] >> (4 * h);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t o = s * 8 + 4 * h + q;
      const double r = ((m >> q) & 1u) ? a[q] - X[o] : 0.0;
      if (REPORT) {
        mx = fmax(mx, fabs(d[s] * r));
      } else {
        const float rf = __double2float_rn(r);
        R[o] = rf;
        D1[o] = rf;
        mx = fmax(mx, fabs(r));
      }
    }
  }
  __shared__ double sh[32];
  double a[1] = {mx != mx ? __longlong_as_double(0x7ff0000000000000LL) : mx};
  block_reduce<1, true>(a, sh);
  if (threadIdx.x == 0) atomic_max_nonneg(&st->slot[slot], a[0]);
}

// FP32 correction sweep of every right-hand side on the Jacobi form:
// D'_j = R_j + sum_{s'} Aj_hi(s,s') D_j[s'] on S?_j, 0 elsewhere.  Here 8 lanes own a row,
// lane j the right-hand side j, so the 8 lanes gather one 32-byte row of D together.  (Two
// lanes with a float4 each ran at the same speed but doubled the DRAM traffic: more rows
// in flight per warp spread the gathers over more of D and L2 kept less of it.)
__global__ void __launch_bounds__(BT) k_bsweep(int64_t n, const int64_t* __restrict__ rp,
                                               const int32_t* __restrict__ ci, const float* __restrict__ ah,
                                               const uint8_t* __restrict__ sq, const float* __restrict__ R,
                                               const float* __restrict__ Din, float* __restrict__ Dout,
                                               const SolveState* st) {
  if (st->done) return;
  RowGroups rg = RowGroups::make<8>();
  const int j = rg.lane;
  for (int64_t s = rg.first; s < n; s += rg.stride) {
    const int64_t hi = rp[s + 1];
    int64_t k = rp[s];
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
    for (; k + 3 < hi; k += 4) {
      const int32_t c0 = __ldcs(ci + k), c1 = __ldcs(ci + k + 1), c2 = __ldcs(ci + k + 2), c3 = __ldcs(ci + k + 3);
      const float v0 = __ldcs(ah + k), v1 = __ldcs(ah + k + 1), v2 = __ldcs(ah + k + 2), v3 = __ldcs(ah + k + 3);
      a0 = fmaf(v0, __ldg(Din + (int64_t)c0 * 8 + j), a0);
      a1 = fmaf(v1, __ldg(Din + (int64_t)c1 * 8 + j), a1);
      a2 = fmaf(v2, __ldg(Din + (int64_t)c2 * 8 + j), a2);
      a3 = fmaf(v3, __ldg(Din + (int64_t)c3 * 8 + j), a3);
    }
    for (; k < hi; ++k) a0 = fmaf(__ldcs(ah + k), __ldg(Din + (int64_t)__ldcs(ci + k) * 8 + j), a0);
    const bool q = (sq[s] >> j) & 1u;
    Dout[s * 8 + j] = q ? R[s * 8 + j] + ((a0 + a1) + (a2 + a3)) : 0.0f;
  }
}

__global__ void k_bapply(int64_t total, double* __restrict__ X, const float* __restrict__ D,
                         const SolveState* st) {
  if (st->done) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x)
    X[i] += (double)D[i];
}

__global__ void k_bout(int64_t n, int k, const double* __restrict__ X, double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * k;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = i / n, s = i - j * n;
    out[i] = X[s * 8 + j];
  }
}

__global__ void k_bclasses_out(int64_t n, int k, const uint8_t* __restrict__ sq, const uint8_t* __restrict__ one,
                               uint8_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * k;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = i / n, s = i - j * n;
    out[i] = ((sq[s] >> j) & 1u) ? CLS_SQ : (((one[s] >> j) & 1u) ? CLS_S1 : CLS_S0);
  }
}

#define G_DISPATCH(g, FN, ...)             \
  do {                                     \
    switch (g) {                           \
      case 2: FN<2>(__VA_ARGS__); break;   \
      case 4: FN<4>(__VA_ARGS__); break;   \
      case 8: FN<8>(__VA_ARGS__); break;   \
      case 16: FN<16>(__VA_ARGS__); break; \
      default: FN<32>(__VA_ARGS__); break; \
    }                                      \
  } while (0)

template <int G>
static void l_pull(reach_batch* b, uint8_t* bits, const uint8_t* block, cudaStream_t s) {
  reach_ctx* c = b->base;
  const int grid = grid_rows(c, (const void*)k_pull_or<G>, BT, G, c->n);
  k_pull_or<G><<<grid, BT, 0, s>>>(c->n, c->rowptr, c->col, c->val, bits, block, (1u << b->k) - 1u,
                                   b->changed);
}

static void l_bresid(reach_batch* b, bool report, cudaStream_t s) {
  reach_ctx* c = b->base;
  if (report) {
    const int grid = grid_rows(c, (const void*)k_bresid<true>, BT, 2, c->n);
    k_bresid<true><<<grid, BT, 0, s>>>(c->n, c->a_rowptr, c->a_col, c->a_jv, c->d, b->sq, b->X, b->R, b->D[1],
                                       c->st, 63);
  } else {
    const int grid = grid_rows(c, (const void*)k_bresid<false>, BT, 2, c->n);
    k_bresid<false><<<grid, BT, 0, s>>>(c->n, c->a_rowptr, c->a_col, c->a_jv, c->d, b->sq, b->X, b->R, b->D[1],
                                        c->st, 0);
  }
}

static void l_bsweep(reach_batch* b, const float* din, float* dout, cudaStream_t s) {
  reach_ctx* c = b->base;
  const int grid = grid_rows(c, (const void*)k_bsweep, BT, 8, c->n);
  k_bsweep<<<grid, BT, 0, s>>>(c->n, c->a_rowptr, c->a_col, c->a_hi, b->sq, b->R, din, dout, c->st);
}

// Runs one backward fixed point to completion (conditional-while graph or host loop).
static cudaError_t fixed_point(reach_batch* b, int slot, uint8_t* bits, const uint8_t* block) {
  reach_ctx* c = b->base;
  cudaStream_t s = c->stream;
  const int g = pick_group(c->n, c->m);
  const int64_t max_passes = c->n + 2;
  int64_t* passes = reinterpret_cast<int64_t*>(c->bfs);
  cudaMemsetAsync(b->changed, 0, sizeof(unsigned), s);
  cudaMemsetAsync(passes, 0, sizeof(int64_t), s);
  cudaError_t e = cudaSuccess;
  if (!c->device_loops) {
    for (int64_t it = 0; it < max_passes; ++it) {
      G_DISPATCH(g, l_pull, b, bits, block, s);
      unsigned ch = 0;
      e = cudaMemcpyAsync(&ch, b->changed, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(b->changed, 0, sizeof(unsigned), s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return e;
      b->passes[slot] = it + 1;
      if (!ch) break;
    }
    return cudaGetLastError();
  }
  const int64_t key = c->n * 64 + g * 2 + (block ? 1 : 0);
  if (b->g_exec[slot] == nullptr || b->g_key[slot] != key) {
    if (b->g_exec[slot]) cudaGraphExecDestroy(b->g_exec[slot]);
    b->g_exec[slot] = nullptr;
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
        G_DISPATCH(g, l_pull, b, bits, block, c->cap);
        k_fix_ctl<<<1, 1, 0, c->cap>>>(b->changed, passes, max_passes, h, 1);
        e = cudaStreamEndCapture(c->cap, &bg);
      }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->g_exec[slot], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      b->g_exec[slot] = nullptr;
      return e;
    }
    b->g_key[slot] = key;
  }
  e = cudaGraphLaunch(b->g_exec[slot], s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&b->passes[slot], passes, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace reach

namespace {

// Batch errors are reported through reach_last_error(NULL) (the calling thread's message).
reach_status bfail(reach_batch* b, reach_status s, const std::string& m) {
  if (b && b->base) set_err(b->base, m);
  set_err(nullptr, m);
  return s;
}

reach_status bcuda(reach_batch* b, cudaError_t e, const char* where) {
  bfail(b, REACH_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? REACH_ENOMEM : REACH_ECUDA;
}

template <typename T>
cudaError_t balloc(T** p, int64_t count) {
  *p = nullptr;
  const char* v = std::getenv("REACH_FAULT_ENOMEM");
  if (v && v[0] == '1') return cudaErrorMemoryAllocation;
  return cudaMalloc((void**)p, sizeof(T) * (size_t)(count > 0 ? count : 1));
}

template <typename T>
void bfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

}  // namespace

extern "C" {

void reach_batch_destroy(reach_batch* b) {
  if (!b) return;
  if (b->base && b->base->stream) cudaStreamSynchronize(b->base->stream);
  else cudaDeviceSynchronize();
  for (int i = 0; i < 3; ++i)
    if (b->g_exec[i]) cudaGraphExecDestroy(b->g_exec[i]);
  bfree(b->gbits); bfree(b->rbits); bfree(b->bbits); bfree(b->sq); bfree(b->one);
  bfree(b->X); bfree(b->R); bfree(b->D[0]); bfree(b->D[1]); bfree(b->changed);
  reach_destroy(b->base);
  delete b;
}

reach_status reach_batch_create(reach_batch** out, int64_t n, int64_t m, const int64_t* rowptr,
                                const int32_t* col, const double* val, int32_t k, const uint8_t* goals,
                                int32_t flags, void* stream) {
  if (!out) return bfail(nullptr, REACH_EINVAL, "reach_batch_create: out is NULL");
  if (k < 1 || k > 8) return bfail(nullptr, REACH_EINVAL, "reach_batch_create: k must be in [1, 8]");
  if (!goals) return bfail(nullptr, REACH_EINVAL, "reach_batch_create: goals is NULL");
  // the base context validates P; its own goal mask is the first goal set
  reach_ctx* base = nullptr;
  reach_status st = reach_create(&base, n, m, rowptr, col, val, goals, flags, stream);
  if (st != REACH_OK) return st;
  reach_batch* b = new reach_batch();
  b->base = base;
  b->k = k;
  cudaStream_t s = base->stream;
  cudaError_t e;
  uint8_t* gdev = nullptr;
  if ((e = balloc(&b->gbits, n)) != cudaSuccess || (e = balloc(&b->rbits, n)) != cudaSuccess ||
      (e = balloc(&b->bbits, n)) != cudaSuccess || (e = balloc(&b->sq, n)) != cudaSuccess ||
      (e = balloc(&b->one, n)) != cudaSuccess || (e = balloc(&b->changed, 1)) != cudaSuccess ||
      (flags == REACH_HOST && (e = balloc(&gdev, n * k)) != cudaSuccess)) {
    reach_status r = bcuda(b, e, "reach_batch_create: allocation");
    std::string msg = base->err;
    bfree(gdev);
    reach_batch_destroy(b);
    set_err(nullptr, msg);
    return r;
  }
  const uint8_t* gsrc = goals;
  if (flags == REACH_HOST) {
    e = cudaMemcpyAsync(gdev, goals, (size_t)(n * k), cudaMemcpyHostToDevice, s);
    gsrc = gdev;
  } else {
    e = cudaSuccess;
  }
  if (e == cudaSuccess) {
    k_goal_bits<<<grid_for(base, (const void*)k_goal_bits, BT, n), BT, 0, s>>>(n, k, gsrc, b->gbits);
    e = cudaStreamSynchronize(s);
  }
  bfree(gdev);
  if (e != cudaSuccess) {
    reach_status r = bcuda(b, e, "reach_batch_create");
    std::string msg = base->err;
    reach_batch_destroy(b);
    set_err(nullptr, msg);
    return r;
  }
  *out = b;
  return REACH_OK;
}

reach_status reach_batch_precompute(reach_batch* b, int32_t mode) {
  if (!b) return bfail(nullptr, REACH_EINVAL, "reach_batch_precompute: NULL batch");
  if (mode != REACH_PROB01 && mode != REACH_PROB0_ONLY)
    return bfail(b, REACH_EINVAL, "reach_batch_precompute: unknown mode");
  reach_ctx* c = b->base;
  cudaStream_t s = c->stream;
  const int64_t n = c->n;
  const unsigned kmask = (1u << b->k) - 1u;
  b->have_classes = false;
  cudaError_t e = cudaSuccess;
  // system rows for every state, FP32 hi/lo split (once per batch)
  if (!c->a_rowptr) {
    e = extract_all_rows(c);
    // the batch has no b (the goal sets enter through X); its Jacobi form divides rows by
    // d_s, and absorbing rows (d_s = 0) have no off-diagonal entries to divide
    if (e == cudaSuccess) e = cudaMemsetAsync(c->b, 0, sizeof(double) * (size_t)c->n_q, s);
    if (e == cudaSuccess) e = build_jacobi_form(c);
    if (e == cudaSuccess) e = split_hilo(c);
    if (e != cudaSuccess) return bcuda(b, e, "reach_batch_precompute: extraction");
  }
  if (!b->X) {
    if ((e = balloc(&b->X, n * 8)) != cudaSuccess || (e = balloc(&b->R, n * 8)) != cudaSuccess ||
        (e = balloc(&b->D[0], n * 8)) != cudaSuccess || (e = balloc(&b->D[1], n * 8)) != cudaSuccess)
      return bcuda(b, e, "reach_batch_precompute: workspace");
  }
  e = cudaEventRecord(c->ev0, s);
  // S=0_j: complement of the states that reach GS_j (§2.2)
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->rbits, b->gbits, n, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = fixed_point(b, 0, b->rbits, nullptr);
  // S=1_j: complement of the states that reach S=0_j without meeting GS_j
  if (e == cudaSuccess && mode == REACH_PROB01) {
    k_not_bits<<<grid_for(c, (const void*)k_not_bits, BT, n), BT, 0, s>>>(n, b->rbits, b->bbits, kmask);
    e = fixed_point(b, 1, b->bbits, b->gbits);
  }
  if (e == cudaSuccess) {
    k_batch_classes<<<grid_for(c, (const void*)k_batch_classes, BT, n), BT, 0, s>>>(
        n, mode, kmask, b->gbits, b->rbits, b->bbits, b->sq, b->one, b->X);
    e = cudaEventRecord(c->ev1, s);
  }
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventSynchronize(c->ev1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  if (e != cudaSuccess) return bcuda(b, e, "reach_batch_precompute");
  c->ms_precompute = ms;
  b->have_classes = true;
  return REACH_OK;
}

reach_status reach_batch_get_classes(reach_batch* b, uint8_t* cls, int32_t flags) {
  if (!b) return bfail(nullptr, REACH_EINVAL, "reach_batch_get_classes: NULL batch");
  if (!b->have_classes) return bfail(b, REACH_ESTATE, "reach_batch_get_classes: call reach_batch_precompute first");
  if (!cls || (flags != REACH_HOST && flags != REACH_DEVICE))
    return bfail(b, REACH_EINVAL, "reach_batch_get_classes: bad output");
  reach_ctx* c = b->base;
  cudaStream_t s = c->stream;
  const int64_t total = c->n * b->k;
  uint8_t* dst = cls;
  cudaError_t e = cudaSuccess;
  if (flags == REACH_HOST) e = balloc(&dst, total);
  if (e == cudaSuccess) {
    k_bclasses_out<<<grid_for(c, (const void*)k_bclasses_out, BT, total), BT, 0, s>>>(c->n, b->k, b->sq, b->one, dst);
    if (flags == REACH_HOST) e = cudaMemcpyAsync(cls, dst, (size_t)total, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (flags == REACH_HOST) bfree(dst);
  return e == cudaSuccess ? REACH_OK : bcuda(b, e, "reach_batch_get_classes");
}

reach_status reach_batch_solve(reach_batch* b, double eps, int64_t max_iter, int32_t refine_k,
                               double* x_out, int32_t flags, reach_info* info) {
  if (!b) return bfail(nullptr, REACH_EINVAL, "reach_batch_solve: NULL batch");
  if (!b->have_classes) return bfail(b, REACH_ESTATE, "reach_batch_solve: call reach_batch_precompute first");
  if (!(eps > 0.0) || max_iter < 1) return bfail(b, REACH_EINVAL, "reach_batch_solve: bad eps or max_iter");
  if (refine_k == 0) refine_k = 16;
  if (refine_k < 2 || refine_k > 62 || (refine_k & 1))
    return bfail(b, REACH_EINVAL, "reach_batch_solve: refine_k must be even in [2, 62]");
  if (!x_out || (flags != REACH_HOST && flags != REACH_DEVICE))
    return bfail(b, REACH_EINVAL, "reach_batch_solve: bad output");
  reach_ctx* c = b->base;
  cudaStream_t s = c->stream;
  const int64_t n = c->n;
  SolveState hs;
  std::memset(&hs, 0, sizeof(hs));
  hs.eps = eps;
  hs.max_iter = max_iter;
  hs.status = REACH_ENOTCONV;
  hs.max_bodies = max_iter / refine_k + 4;
  cudaError_t e = cudaMemcpyAsync(c->st, &hs, sizeof(hs), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  double* xdev = x_out;
  if (e == cudaSuccess && flags == REACH_HOST) e = balloc(&xdev, n * b->k);
  if (e != cudaSuccess) return bcuda(b, e, "reach_batch_solve");
  const int g = pick_group(n, c->m_q);
  const int kref = refine_k;
  k_batch_init_x<<<grid_for(c, (const void*)k_batch_init_x, BT, n * 8), BT, 0, s>>>(n, b->one, b->X);
  e = cudaEventRecord(c->ev0, s);
  if (e == cudaSuccess) {
    const int64_t key = (n * 1000003LL + c->m_q) * 64 + g * 4 + kref * 1000;
    e = run_loop(c, b->g_exec[2], b->g_key[2], key, [&](cudaStream_t cs, cudaGraphConditionalHandle, int) {
      l_bresid(b, false, cs);
      launch_check_mixed(cs, c->st, 0, kref);
      // kref - 1 FP32 sweeps: D[1] -> D[0] -> ...; kref even, so the last lands in D[0]
      for (int j = 1; j < kref; ++j) {
        const float* din = (j & 1) ? b->D[1] : b->D[0];
        float* dout = (j & 1) ? b->D[0] : b->D[1];
        l_bsweep(b, din, dout, cs);
      }
      k_bapply<<<grid_for(c, (const void*)k_bapply, BT, n * 8), BT, 0, cs>>>(n * 8, b->X, b->D[0], c->st);
    });
  }
  if (e == cudaSuccess) {
    l_bresid(b, true, s);
    launch_finalize_resid(s, c->st);
    k_bout<<<grid_for(c, (const void*)k_bout, BT, n * b->k), BT, 0, s>>>(n, b->k, b->X, xdev);
    e = cudaEventRecord(c->ev1, s);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, c->st, sizeof(hs), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && flags == REACH_HOST)
    e = cudaMemcpyAsync(x_out, xdev, sizeof(double) * (size_t)(n * b->k), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  if (flags == REACH_HOST) bfree(xdev);
  if (e != cudaSuccess) return bcuda(b, e, "reach_batch_solve");
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iters = hs.iter;
    info->n_q = n;
    info->m_q = c->m_q;
    info->last_delta = hs.last;
    info->resid_inf = hs.resid;
    info->ms_precompute = c->ms_precompute;
    info->ms_solve = ms;
    info->bytes_moved = (double)hs.refinements * ((double)c->m_q * 12.0 + (double)n * 150.0) +
                        (double)(hs.iter - hs.refinements) * ((double)c->m_q * 8.0 + (double)n * 80.0);
    info->status = hs.status;
    info->refinements = hs.refinements;
  }
  if (hs.status != REACH_OK) bfail(b, REACH_ENOTCONV, "reach_batch_solve: max_iter reached before the stopping rule held");
  return (reach_status)hs.status;
}

}  // extern "C"
