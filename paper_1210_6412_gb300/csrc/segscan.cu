// FP64 Jacobi sweep balanced over stored entries instead of rows: a segmented
// reduction over the flat entry array of A (the related work the paper cites runs the
// Jacobi iteration on a backward segmented scan; the forward segmented reduction used
// here yields the same row sums).  Every CTA processes one tile of SEG_T consecutive
// entries whatever the row lengths, so a matrix with a few very long rows keeps every
// SM busy, where a row-per-warp mapping would leave one warp with a whole long row.
//
// The sweep runs on the Jacobi form (Aj = D^-1 A, bj = D^-1 b: x' = bj + Aj x).
// Per sweep: k_seg_sweep reads each entry once, finishes every row whose entries lie in
// one tile, and leaves for each tile the sum before its first row end (head) and after
// its last row end (tail); k_seg_fix completes the rows that span tiles by adding those
// partial sums in tile order and also handles rows without entries.  All sums are in a
// fixed order, so the sweep is deterministic.
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "internal.h"

namespace reach {

constexpr int SEG_NT = 256;
constexpr int SEG_ITEMS = 16;   // stored entries per thread (a multiple of 4, at most 32)
constexpr int64_t SEG_T = SEG_NT * SEG_ITEMS;   // entries per tile

struct SegPlan {
  int64_t ntiles = 0;
  int64_t n_span = 0;      // rows whose entries span more than one tile
  int64_t n_empty = 0;     // rows without entries
  uint32_t* endbits = nullptr;    // bit k: entry k is the last of its row
  int64_t* tile_row0 = nullptr;   // nonempty-row index of the row holding the tile's first entry
  int64_t* nonempty = nullptr;    // nonempty-row index -> row
  int64_t* span = nullptr;        // rows spanning tiles
  int64_t* empty = nullptr;       // rows without entries
  double* head = nullptr;         // per tile
  double* tail = nullptr;         // per tile
  int64_t* total = nullptr;       // one scan total
};

// ---- plan construction (once per system)

__global__ void k_seg_marks(int64_t nq, const int64_t* __restrict__ rp, uint32_t* endbits,
                            uint8_t* nonempty_flag, uint8_t* span_flag, uint8_t* empty_flag) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nq;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lo = rp[r], hi = rp[r + 1];
    const bool ne = hi > lo;
    nonempty_flag[r] = ne;
    empty_flag[r] = !ne;
    span_flag[r] = ne && (lo / SEG_T) != ((hi - 1) / SEG_T);
    if (ne) atomicOr(endbits + ((hi - 1) >> 5), 1u << ((hi - 1) & 31));
  }
}

__global__ void k_seg_compact(int64_t nq, const uint8_t* __restrict__ flag, const int64_t* __restrict__ pos,
                              int64_t* __restrict__ out) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nq;
       r += (int64_t)gridDim.x * blockDim.x)
    if (flag[r]) out[pos[r]] = r;
}

// Row holding entry t*SEG_T (binary search in rp), as a nonempty-row index.
__global__ void k_seg_tile_rows(int64_t nq, int64_t ntiles, const int64_t* __restrict__ rp,
                                const int64_t* __restrict__ ne_pos, int64_t* __restrict__ tile_row0) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntiles;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = t * SEG_T;
    int64_t lo = 0, hi = nq;                 // last r with rp[r] <= k
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (rp[mid] <= k) lo = mid;
      else hi = mid;
    }
    while (lo < nq && rp[lo + 1] <= k) ++lo;  // skip empty rows sitting at k
    tile_row0[t] = ne_pos[lo];
  }
}

// ---- the sweep

// Inclusive segmented sum across the CTA: (v, f) then (w, g) -> (g ? w : v + w, f | g).
template <typename V>
RDEV void seg_scan_cta(V& v, int& f, V* shv, int* shf) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const V pv = __shfl_up_sync(FULL, v, o);
    const int pf = __shfl_up_sync(FULL, f, o);
    if (lane >= o && !f) v += pv;
    if (lane >= o) f |= pf;
  }
  if (lane == 31) {
    shv[w] = v;
    shf[w] = f;
  }
  __syncthreads();
  if (w == 0) {
    V a = lane < (SEG_NT / 32) ? shv[lane] : V(0);
    int af = lane < (SEG_NT / 32) ? shf[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const V pv = __shfl_up_sync(FULL, a, o);
      const int pf = __shfl_up_sync(FULL, af, o);
      if (lane >= o && !af) a += pv;
      if (lane >= o) af |= pf;
    }
    if (lane < SEG_NT / 32) {
      shv[lane] = a;
      shf[lane] = af;
    }
  }
  __syncthreads();
  if (w > 0 && !f) v += shv[w - 1];
  if (w > 0) f |= shf[w - 1];
  __syncthreads();
}

// The three sweeps that run entry-balanced: how a stored entry adds into a running row
// sum (one FMA in the accumulation type, so a sum costs one FP64 instruction per entry
// in the FP64 sweeps), and what a finished row sum becomes.  finish() returns the row's
// contribution to the stopping quantity (0 for the FP32 sweep, which has none).
struct OpJac64 {          // FP64 Jacobi on the Jacobi form: x' = bj + Aj x, max|x' - x|
  using V = double;
  struct Q { double2 a, b; };
  static constexpr bool DELTA = true;
  const double* av;
  const double* x;
  const double* bj;
  double* xn;
  RDEV Q load4(int64_t k) const {
    return {__ldcs(reinterpret_cast<const double2*>(av + k)), __ldcs(reinterpret_cast<const double2*>(av + k + 2))};
  }
  RDEV V acc(V run, const Q& q, int u, int c) const {
    const double v = u == 0 ? q.a.x : u == 1 ? q.a.y : u == 2 ? q.b.x : q.b.y;
    return fma(v, __ldg(x + c), run);
  }
  RDEV V acc1(V run, int64_t k, int c) const { return fma(__ldcs(av + k), __ldg(x + c), run); }
  RDEV double finish(int64_t r, V s) const {
    const double xv = bj[r] + s;
    xn[r] = xv;
    return fabs(xv - x[r]);
  }
};

struct OpSpmv64 {         // y = A u with the system's own values (the products of BiCGStab)
  using V = double;
  struct Q { double2 a, b; };
  static constexpr bool DELTA = false;
  const double* av;
  const double* u;
  double* y;
  RDEV Q load4(int64_t k) const {
    return {__ldcs(reinterpret_cast<const double2*>(av + k)), __ldcs(reinterpret_cast<const double2*>(av + k + 2))};
  }
  RDEV V acc(V run, const Q& q, int i, int c) const {
    const double v = i == 0 ? q.a.x : i == 1 ? q.a.y : i == 2 ? q.b.x : q.b.y;
    return fma(v, __ldg(u + c), run);
  }
  RDEV V acc1(V run, int64_t k, int c) const { return fma(__ldcs(av + k), __ldg(u + c), run); }
  RDEV double finish(int64_t r, V s) const {
    y[r] = s;
    return 0.0;
  }
};

struct OpSweep32 {        // FP32 correction sweep of the mixed method: d' = r + Aj_hi d
  using V = float;
  using Q = float4;
  static constexpr bool DELTA = false;
  const float* ah;
  const float* din;
  const float* r32;
  float* dout;
  RDEV Q load4(int64_t k) const { return __ldcs(reinterpret_cast<const float4*>(ah + k)); }
  RDEV V acc(V run, const Q& q, int u, int c) const {
    const float v = u == 0 ? q.x : u == 1 ? q.y : u == 2 ? q.z : q.w;
    return fmaf(v, __ldg(din + c), run);
  }
  RDEV V acc1(V run, int64_t k, int c) const { return fmaf(__ldcs(ah + k), __ldg(din + c), run); }
  RDEV double finish(int64_t r, V s) const {
    dout[r] = r32[r] + s;
    return 0.0;
  }
};

struct OpResidHilo {      // FP64 residual of the mixed method: r = bj + Aj x - x, values hi + lo
  using V = double;
  struct Q { float4 h, l; };
  static constexpr bool DELTA = true;
  const float* ah;
  const float* al;
  const double* x;
  const float* xf;
  const double* bj;
  float* r32;
  float* dl0;
  // hi * x in FP64 (the FMA, with the integer widening), lo * x in FP32 (lo is below
  // 2^-24 of the value) and widened, added to the running sum in FP64
  RDEV V one(V run, float h, float l, int c) const { return fma(widen(h), __ldg(x + c), run + widen(l * __ldg(xf + c))); }
  RDEV Q load4(int64_t k) const {
    return {__ldcs(reinterpret_cast<const float4*>(ah + k)), __ldcs(reinterpret_cast<const float4*>(al + k))};
  }
  RDEV V acc(V run, const Q& q, int u, int c) const {
    const float h = u == 0 ? q.h.x : u == 1 ? q.h.y : u == 2 ? q.h.z : q.h.w;
    const float l = u == 0 ? q.l.x : u == 1 ? q.l.y : u == 2 ? q.l.z : q.l.w;
    return one(run, h, l, c);
  }
  RDEV V acc1(V run, int64_t k, int c) const { return one(run, __ldcs(ah + k), __ldcs(al + k), c); }
  RDEV double finish(int64_t r, V s) const {
    const double rv = bj[r] + s - x[r];
    const float rf = __double2float_rn(rv);
    r32[r] = rf;
    dl0[r] = rf;
    return fabs(rv);
  }
};

RDEV void delta_to_slot(double mx, unsigned long long* slot) {
  __shared__ double sh[32];
  double a[1] = {mx != mx ? __longlong_as_double(0x7ff0000000000000LL) : mx};
  block_reduce<1, true>(a, sh);
  if (threadIdx.x == 0) atomic_max_nonneg(slot, a[0]);
}

template <class Op>
__global__ void __launch_bounds__(SEG_NT) k_seg_sweep(int64_t mq, int64_t ntiles, const int64_t* __restrict__ rp,
                                                      const int32_t* __restrict__ ci, Op op,
                                                      const uint32_t* __restrict__ endbits,
                                                      const int64_t* __restrict__ tile_row0,
                                                      const int64_t* __restrict__ nonempty,
                                                      typename Op::V* __restrict__ head,
                                                      typename Op::V* __restrict__ tail,
                                                      unsigned long long* slot) {
  using V = typename Op::V;
  __shared__ V shv[SEG_NT / 32];
  __shared__ int shf[SEG_NT / 32];
  __shared__ int shc[SEG_NT / 32];
  __shared__ V lastv[SEG_NT / 32];
  double mx = 0.0;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t base = t * SEG_T + (int64_t)threadIdx.x * SEG_ITEMS;
    // this thread's row-end flags
    unsigned flags = 0;
    const bool full = base + SEG_ITEMS <= mq;
    if (full) {
      flags = (__ldg(endbits + (base >> 5)) >> (base & 31)) & ((1u << SEG_ITEMS) - 1u);
    } else {
#pragma unroll
      for (int j = 0; j < SEG_ITEMS; ++j) {
        const int64_t k = base + j;
        if (k < mq && ((__ldg(endbits + (k >> 5)) >> (k & 31)) & 1u)) flags |= 1u << j;
      }
    }
    const int cnt = __popc(flags);
    // row index (among non-empty rows) of this thread's first entry: tile start + row ends before it
    int excl = cnt;
    {
      const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int pv = __shfl_up_sync(FULL, excl, o);
        if (lane >= o) excl += pv;
      }
      if (lane == 31) shc[w] = excl;
      __syncthreads();
      int off = 0;
      for (int j = 0; j < w; ++j) off += shc[j];
      excl += off - cnt;
      __syncthreads();
    }
    // running sums over this thread's entries: head (up to the first row end), whole rows
    // inside, tail
    V head_v = V(0), run = V(0);
    int seen = 0;
    const int64_t row0 = tile_row0[t] + excl;    // nonempty index of this thread's first row
    auto row_end = [&](int j) {
      if ((flags >> j) & 1u) {
        if (seen == 0) {
          head_v = run;                          // completed below, after the carry-in
        } else {
          const int64_t r = nonempty[row0 + seen];   // row entirely inside this thread
          mx = fmax(mx, op.finish(r, run));
        }
        ++seen;
        run = V(0);
      }
    };
    if (full) {
#pragma unroll
      for (int q = 0; q < SEG_ITEMS / 4; ++q) {
        const int4 c4 = __ldcs(reinterpret_cast<const int4*>(ci + base + 4 * q));
        const typename Op::Q v4 = op.load4(base + 4 * q);
        run = op.acc(run, v4, 0, c4.x);
        row_end(4 * q);
        run = op.acc(run, v4, 1, c4.y);
        row_end(4 * q + 1);
        run = op.acc(run, v4, 2, c4.z);
        row_end(4 * q + 2);
        run = op.acc(run, v4, 3, c4.w);
        row_end(4 * q + 3);
      }
    } else {
#pragma unroll
      for (int j = 0; j < SEG_ITEMS; ++j) {
        const int64_t k = base + j;
        if (k < mq) run = op.acc1(run, k, __ldcs(ci + k));
        row_end(j);
      }
    }
    // Segmented scan over threads: value = this thread's tail, a segment starts at every
    // thread with a row end.  The exclusive result is the part of this thread's first row
    // that lies in earlier threads of the tile.
    int f = cnt ? 1 : 0;
    V incl = run;
    seg_scan_cta<V>(incl, f, shv, shf);
    V carry = __shfl_up_sync(FULL, incl, 1);
    {
      const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
      if (lane == 31) lastv[w] = incl;
      __syncthreads();
      if (lane == 0) carry = w > 0 ? lastv[w - 1] : V(0);
      __syncthreads();
    }
    if (cnt) {
      const V first_total = carry + head_v;
      const int64_t r = nonempty[row0];
      if (rp[r] >= t * SEG_T) {                  // the row starts inside this tile: complete
        mx = fmax(mx, op.finish(r, first_total));
      } else {                                   // started in an earlier tile: finished by k_seg_fix
        head[t] = first_total;
      }
    }
    // the tile's last thread publishes what follows the tile's last row end
    if (threadIdx.x == SEG_NT - 1) tail[t] = incl;
    __syncthreads();
  }
  if constexpr (Op::DELTA) delta_to_slot(mx, slot);
}

// Rows spanning tiles: tail of the first tile + whole middle tiles + head of the last
// tile, in tile order.  Threads past the spanning rows handle rows without entries.
template <class Op>
__global__ void k_seg_fix(int64_t n_span, int64_t n_empty, const int64_t* __restrict__ span,
                          const int64_t* __restrict__ empty, const int64_t* __restrict__ rp, Op op,
                          const typename Op::V* __restrict__ head, const typename Op::V* __restrict__ tail,
                          unsigned long long* slot) {
  using V = typename Op::V;
  double mx = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_span + n_empty;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t r;
    V s = V(0);
    if (i < n_span) {
      r = span[i];
      const int64_t t0 = rp[r] / SEG_T, t1 = (rp[r + 1] - 1) / SEG_T;
      s = tail[t0];
      for (int64_t t = t0 + 1; t < t1; ++t) s += tail[t];
      s += head[t1];
    } else {
      r = empty[i - n_span];
    }
    mx = fmax(mx, op.finish(r, s));
  }
  if constexpr (Op::DELTA) delta_to_slot(mx, slot);
}

__global__ void k_seg_check(SolveState* st, int slot_idx, int sweeps, int reset_n) {
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
  for (int j = 0; j < reset_n; ++j) st->slot[j] = 0ull;
}

// ---- host side

template <typename T>
static cudaError_t salloc(T** p, int64_t n) {
  return cudaMalloc((void**)p, sizeof(T) * (size_t)(n > 0 ? n : 1));
}

void seg_free(reach_ctx* c) {
  SegPlan* sp = static_cast<SegPlan*>(c->seg);
  if (!sp) return;
  cudaFree(sp->endbits);
  cudaFree(sp->tile_row0);
  cudaFree(sp->nonempty);
  cudaFree(sp->span);
  cudaFree(sp->empty);
  cudaFree(sp->head);
  cudaFree(sp->tail);
  cudaFree(sp->total);
  delete sp;
  c->seg = nullptr;
}

// Tile plan of the current system: row-end bits, the row of each tile's first entry,
// the rows spanning tiles and the rows without entries.
cudaError_t seg_plan(reach_ctx* c) {
  if (c->seg) return cudaSuccess;
  cudaStream_t s = c->stream;
  const int64_t nq = c->n_q, mq = c->m_q;
  SegPlan* sp = new SegPlan();
  c->seg = sp;
  sp->ntiles = (mq + SEG_T - 1) / SEG_T;
  const int64_t words = (mq + 31) / 32 + 1;
  uint8_t *fne = nullptr, *fspan = nullptr, *fempty = nullptr;
  int64_t *pne = nullptr, *pspan = nullptr, *pempty = nullptr;
  cudaError_t e;
  if ((e = salloc(&sp->endbits, words)) != cudaSuccess || (e = salloc(&sp->tile_row0, sp->ntiles)) != cudaSuccess ||
      (e = salloc(&sp->head, sp->ntiles)) != cudaSuccess || (e = salloc(&sp->tail, sp->ntiles)) != cudaSuccess ||
      (e = salloc(&sp->total, 1)) != cudaSuccess ||
      (e = salloc(&fne, nq)) != cudaSuccess || (e = salloc(&fspan, nq)) != cudaSuccess ||
      (e = salloc(&fempty, nq)) != cudaSuccess || (e = salloc(&pne, nq + 1)) != cudaSuccess ||
      (e = salloc(&pspan, nq + 1)) != cudaSuccess || (e = salloc(&pempty, nq + 1)) != cudaSuccess) {
    cudaFree(fne); cudaFree(fspan); cudaFree(fempty); cudaFree(pne); cudaFree(pspan); cudaFree(pempty);
    seg_free(c);
    return e;
  }
  cudaMemsetAsync(sp->endbits, 0, sizeof(uint32_t) * words, s);
  const int g = grid_for(c, (const void*)k_seg_marks, 256, nq);
  k_seg_marks<<<g, 256, 0, s>>>(nq, c->a_rowptr, sp->endbits, fne, fspan, fempty);
  int64_t counts[3] = {0, 0, 0};
  int64_t* tot = sp->total;     // scan totals (never the solve state: a solve may be under way)
  e = exclusive_scan_u8(c, fne, pne, nq, tot);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&counts[0], tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = exclusive_scan_u8(c, fspan, pspan, nq, tot);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&counts[1], tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = exclusive_scan_u8(c, fempty, pempty, nq, tot);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&counts[2], tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) {
    sp->n_span = counts[1];
    sp->n_empty = counts[2];
    if ((e = salloc(&sp->nonempty, counts[0])) == cudaSuccess && (e = salloc(&sp->span, counts[1])) == cudaSuccess &&
        (e = salloc(&sp->empty, counts[2])) == cudaSuccess) {
      k_seg_compact<<<g, 256, 0, s>>>(nq, fne, pne, sp->nonempty);
      k_seg_compact<<<g, 256, 0, s>>>(nq, fspan, pspan, sp->span);
      k_seg_compact<<<g, 256, 0, s>>>(nq, fempty, pempty, sp->empty);
      if (sp->ntiles > 0)
        k_seg_tile_rows<<<grid_for(c, (const void*)k_seg_tile_rows, 256, sp->ntiles), 256, 0, s>>>(
            nq, sp->ntiles, c->a_rowptr, pne, sp->tile_row0);
      e = cudaStreamSynchronize(s);
    }
  }
  cudaFree(fne); cudaFree(fspan); cudaFree(fempty); cudaFree(pne); cudaFree(pspan); cudaFree(pempty);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) seg_free(c);
  return e;
}

template <class Op>
static void seg_run(reach_ctx* c, const Op& op, unsigned long long* slot, cudaStream_t s) {
  SegPlan* sp = static_cast<SegPlan*>(c->seg);
  using V = typename Op::V;
  V* head = reinterpret_cast<V*>(sp->head);
  V* tail = reinterpret_cast<V*>(sp->tail);
  if (sp->ntiles > 0) {
    const int grid =
        (int)std::min<int64_t>(sp->ntiles, grid_for(c, (const void*)k_seg_sweep<Op>, SEG_NT, INT64_MAX / 2));
    k_seg_sweep<Op><<<grid, SEG_NT, 0, s>>>(c->m_q, sp->ntiles, c->a_rowptr, c->a_col, op, sp->endbits,
                                             sp->tile_row0, sp->nonempty, head, tail, slot);
  }
  const int64_t rest = sp->n_span + sp->n_empty;
  if (rest > 0)
    k_seg_fix<Op><<<grid_for(c, (const void*)k_seg_fix<Op>, 256, rest), 256, 0, s>>>(
        sp->n_span, sp->n_empty, sp->span, sp->empty, c->a_rowptr, op, head, tail, slot);
}

void seg_sweep(reach_ctx* c, const double* x, double* xn, unsigned long long* slot, cudaStream_t s) {
  seg_run(c, OpJac64{c->a_jv, x, c->bj, xn}, slot, s);
}

// Entry-balanced forms of the mixed method's two kernels (FP32 sweep, FP64 residual).
void seg_sweep32(reach_ctx* c, const float* din, float* dout, cudaStream_t s) {
  seg_run(c, OpSweep32{c->a_hi, din, c->r32, dout}, nullptr, s);
}

void seg_spmv64(reach_ctx* c, const double* u, double* y, cudaStream_t s) {
  seg_run(c, OpSpmv64{c->a_val, u, y}, nullptr, s);
}

void seg_resid_hilo(reach_ctx* c, unsigned long long* slot, cudaStream_t s) {
  seg_run(c, OpResidHilo{c->a_hi, c->a_lo, c->x, c->xf, c->bj, c->r32, c->dl[1]}, slot, s);
}

// FP64 Jacobi (§3.1) with the entry-balanced sweep: same iteration and stopping rule as
// REACH_JACOBI_FP64, different work distribution (and summation order).
cudaError_t solve_jacobi_seg(reach_ctx* c, const double* x0q) {
  cudaStream_t s = c->stream;
  const int64_t nq = c->n_q;
  cudaError_t e = seg_plan(c);
  if (e != cudaSuccess) return e;
  if (x0q) cudaMemcpyAsync(c->x, x0q, sizeof(double) * nq, cudaMemcpyDeviceToDevice, s);
  else cudaMemsetAsync(c->x, 0, sizeof(double) * nq, s);
  const int k = c->tune.k;
  const int64_t key = (nq * 1000003LL + c->m_q) * 131 + 1000LL * k + 77;
  e = run_loop(c, c->g_exec[4], c->g_key[4], key, [&](cudaStream_t cs, cudaGraphConditionalHandle, int) {
    for (int j = 0; j < k; ++j) {
      const double* xi = (j & 1) ? c->x2 : c->x;
      double* xo = (j & 1) ? c->x : c->x2;
      seg_sweep(c, xi, xo, &c->st->slot[j], cs);
    }
    k_seg_check<<<1, 1, 0, cs>>>(c->st, k - 1, k, k);
  });
  if (e != cudaSuccess) return e;
  return residual_report(c, c->x);
}

}  // namespace reach
