// Batched multi-RHS reachability: K <= 8 goal sets over one chain (typically the
// block-diagonal union of many independent chains).  Each right-hand side j has
// its own partition S=0_j / S=1_j / S?_j (§2.2); one pass over the matrix serves all
// K of them.  The partition is a bit-parallel fixed point (bit j of a state's byte
// belongs to goal set j).  The solve is the masked Jacobi iteration on the full P:
//   x_j[s] = (sum_{s' != s} P(s,s') x_j[s']) / (1 - P(s,s))   for s in S?_j,
// with x_j fixed to 1 on S=1_j and 0 on S=0_j, which is the system of §2.3 for each j
// (b enters through the fixed ones).  It runs as FP32 sweeps with an FP64 residual and
// correction every k sweeps, all inside one conditional-while CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

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
  // Chains of the block-diagonal union (one chain [0, n) until reach_batch_set_chains).
  // Chain lists cut each chain into chunks of BCH rows: list 0 holds every chain, list 1
  // the chains still iterating in the current solve.
  int32_t n_chains = 0;
  int64_t chunks_all = 0;      // chunks of list 0
  int64_t* coff = nullptr;     // [n_chains + 1] first state of each chain
  int32_t* lid[2] = {nullptr, nullptr};   // chain ids of each list
  int64_t* lpre[2] = {nullptr, nullptr};  // chunk prefix of each list, [n_chains + 1]
  int64_t* lhdr = nullptr;     // {chains, chunks} of list 0, then of list 1
  unsigned long long* cmax = nullptr;     // per chain: bits of max |r| of a residual step
  double* clast = nullptr;     // per chain: last FP64 Jacobi step
  int64_t* citer = nullptr;    // per chain: sweeps at which it stopped (-1: not yet)
  double* work = nullptr;      // rows and entries processed: residual steps, then sweeps
  int sweep_variant = 0;       // FP32 sweep: BSW_Q (default), BSW_LANES8, BSW_Q_HINT, BSW_Q_PIPE, BSW_Q_HINT_PIPE
  int tuned_k = 0;             // refinement period from reach_batch_autotune (0 = none)
  cudaGraphExec_t g_exec[3] = {nullptr, nullptr, nullptr};
  int64_t g_key[3] = {-1, -1, -1};
  int64_t passes[2] = {0, 0};
};

namespace reach {

constexpr int BT = 256;
// FP32 sweep variants of the batch (autotuner candidates)
enum { BSW_Q = 0, BSW_LANES8 = 1, BSW_Q_HINT = 2, BSW_Q_PIPE = 3, BSW_Q_HINT_PIPE = 4, BSW_COUNT = 5 };

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
// reduction is needed (which matters most in FP64, whose pipe is narrow).  Rows are dealt
// by chain lists: chunk q of a list is BCH rows of one chain, warp w takes chunks w, w + W,
// ... (W warps in the grid), so a converged chain costs nothing and a warp's per-chain
// maximum needs one atomic per chunk at most.  At any moment the grid works on a window of
// W * BCH consecutive rows, which keeps the gathers of that window's chains in L2.

constexpr int BCH = 32;

struct ChainList {
  const int64_t* hdr;   // {chains, chunks}
  const int32_t* id;    // chain ids (ascending)
  const int64_t* pre;   // chunk prefix over the list, [chains + 1]
  const int64_t* coff;  // chain offsets
};

// A warp's walk over its chunks.  q only grows, so the list position moves forward: one
// probe of the next boundary, and a binary search over the rest when q jumped past it.
struct ChunkWalk {
  int32_t t = 0;
  RDEV void rows(const ChainList& L, int32_t nl, int64_t q, int64_t& r0, int64_t& r1, int32_t& c) {
    if (L.pre[t + 1] <= q) {
      int32_t lo = t + 1, hi = nl;  // pre[lo] <= q < pre[hi]
      while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (L.pre[mid] <= q) lo = mid;
        else hi = mid;
      }
      t = lo;
    }
    c = L.id[t];
    r0 = L.coff[c] + (q - L.pre[t]) * BCH;
    r1 = min(r0 + (int64_t)BCH, L.coff[c + 1]);
  }
};

RDEV unsigned long long bits_abs(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}

// Warp max of |r| bit patterns into a slot; NaN (bits above +inf) is stored as +inf.
RDEV void warp_flush_max(unsigned long long* slot, unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(FULL, v, o);
    v = y > v ? y : v;
  }
  if ((threadIdx.x & 31) == 0 && v != 0ull) atomicMax(slot, v < 0x7ff0000000000000ull ? v : 0x7ff0000000000000ull);
}

// FP64 residual of every right-hand side on the Jacobi form (values A_sj / d_s, read in
// FP64): r_j = sum_{s'} Aj(s,s') x_j[s'] - x_j[s] on S?_j, 0 elsewhere; r_j is also the
// first correction.  Per chain of the list, max|r_j| goes to cmax[chain].  REPORT: only
// max|d_s r_j| (the residual of the system itself) over the list, into st->slot[slot].
// Two lanes own a row, lane h the right-hand sides 4h .. 4h+3, gathering two double2 of
// the 64-byte row of X per entry.
template <bool REPORT>
__global__ void __launch_bounds__(BT) k_bresid(ChainList L, const int64_t* __restrict__ rp,
                                               const int32_t* __restrict__ ci, const double* __restrict__ aj,
                                               const double* __restrict__ d, const uint8_t* __restrict__ sq,
                                               const double* __restrict__ X, float* __restrict__ R,
                                               float* __restrict__ D1, SolveState* st, int slot,
                                               unsigned long long* cmax) {
  if (!REPORT && st->done) return;
  const int lane = threadIdx.x & 31;
  const int h = lane & 1;      // right-hand sides 4h .. 4h+3
  const int grp = lane >> 1;   // 16 rows of a chunk at a time
  const int64_t nw = (int64_t)gridDim.x * (BT / 32);
  const int32_t nl = (int32_t)L.hdr[0];
  const int64_t nch = L.hdr[1];
  ChunkWalk walk;
  unsigned long long mx = 0ull;
  int32_t cur = -1;
  for (int64_t q = (int64_t)blockIdx.x * (BT / 32) + (threadIdx.x >> 5); q < nch; q += nw) {
    int64_t r0, r1;
    int32_t c;
    walk.rows(L, nl, q, r0, r1, c);
    if (!REPORT && c != cur) {  // warp-uniform: the warp shares the chunk
      if (cur >= 0) warp_flush_max(cmax + cur, mx);
      cur = c;
      mx = 0ull;
    }
    for (int64_t s = r0 + grp; s < r1; s += 16) {
      const int64_t hi = rp[s + 1];
      double a[4] = {0.0, 0.0, 0.0, 0.0};
      // two entries per trip, both entries' loads issued before the first use
      for (int64_t k = rp[s]; k < hi; k += 2) {
        const bool o1 = k + 1 < hi;
        const double v = __ldcs(aj + k), w = o1 ? __ldcs(aj + k + 1) : 0.0;
        const int32_t c0 = __ldcs(ci + k), c1 = o1 ? __ldcs(ci + k + 1) : 0;
        const double2* xr = reinterpret_cast<const double2*>(X + (int64_t)c0 * 8 + 4 * h);
        const double2* yr = reinterpret_cast<const double2*>(X + (int64_t)c1 * 8 + 4 * h);
        const double2 t0 = __ldg(xr), t1 = __ldg(xr + 1);
        double2 u0 = make_double2(0.0, 0.0), u1 = make_double2(0.0, 0.0);
        if (o1) {
          u0 = __ldg(yr);
          u1 = __ldg(yr + 1);
        }
        a[0] = fma(v, t0.x, a[0]);
        a[1] = fma(v, t0.y, a[1]);
        a[2] = fma(v, t1.x, a[2]);
        a[3] = fma(v, t1.y, a[3]);
        if (o1) {
          a[0] = fma(w, u0.x, a[0]);
          a[1] = fma(w, u0.y, a[1]);
          a[2] = fma(w, u1.x, a[2]);
          a[3] = fma(w, u1.y, a[3]);
        }
      }
      const unsigned m = sq[s] >> (4 * h);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t o = s * 8 + 4 * h + u;
        const double r = ((m >> u) & 1u) ? a[u] - X[o] : 0.0;
        if (REPORT) {
          const unsigned long long b = bits_abs(d[s] * r);
          mx = b > mx ? b : mx;
        } else {
          const float rf = __double2float_rn(r);
          __stcs(R + o, rf);
          __stcs(D1 + o, rf);
          const unsigned long long b = bits_abs(r);
          mx = b > mx ? b : mx;
        }
      }
    }
  }
  if (REPORT) warp_flush_max(&st->slot[slot], mx);
  else if (cur >= 0) warp_flush_max(cmax + cur, mx);
}

// FP32 correction sweep of every right-hand side on the Jacobi form:
// D'_j = R_j + sum_{s'} Aj_hi(s,s') D_j[s'] on S?_j, 0 elsewhere.  Here 8 lanes own a row,
// lane j the right-hand side j, so the 8 lanes gather one 32-byte row of D together.  The
// default is k_bsweep_q below (two lanes per row), 1.5x faster on 64 chains: the gathers
// are latency-bound, and it keeps four times as many rows in flight per warp.
__global__ void __launch_bounds__(BT) k_bsweep(ChainList L, const int64_t* __restrict__ rp,
                                               const int32_t* __restrict__ ci, const float* __restrict__ ah,
                                               const uint8_t* __restrict__ sq, const float* __restrict__ R,
                                               const float* __restrict__ Din, float* __restrict__ Dout,
                                               const SolveState* st) {
  if (st->done) return;
  const int lane = threadIdx.x & 31;
  const int j = lane & 7;      // right-hand side of this lane
  const int grp = lane >> 3;   // 4 rows of a chunk at a time
  const int64_t nw = (int64_t)gridDim.x * (BT / 32);
  const int32_t nl = (int32_t)L.hdr[0];
  const int64_t nch = L.hdr[1];
  ChunkWalk walk;
  for (int64_t q = (int64_t)blockIdx.x * (BT / 32) + (threadIdx.x >> 5); q < nch; q += nw) {
    int64_t r0, r1;
    int32_t c;
    walk.rows(L, nl, q, r0, r1, c);
    for (int64_t s = r0 + grp; s < r1; s += 4) {
      const int64_t hi = rp[s + 1];
      int64_t k = rp[s];
      float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
      // eight entries per trip, every index and value load before the gathers: a row of
      // the batch (2 to 32 entries) takes one to four round trips
      for (; k < hi; k += 8) {
        int32_t c[8];
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const bool ok = k + u < hi;
          c[u] = ok ? __ldcs(ci + k + u) : 0;
          v[u] = ok ? __ldcs(ah + k + u) : 0.0f;
        }
        float g[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) g[u] = k + u < hi ? __ldg(Din + (int64_t)c[u] * 8 + j) : 0.0f;
        a0 = fmaf(v[0], g[0], a0);
        a1 = fmaf(v[1], g[1], a1);
        a2 = fmaf(v[2], g[2], a2);
        a3 = fmaf(v[3], g[3], a3);
        a0 = fmaf(v[4], g[4], a0);
        a1 = fmaf(v[5], g[5], a1);
        a2 = fmaf(v[6], g[6], a2);
        a3 = fmaf(v[7], g[7], a3);
      }
      // R and the new D are streamed (evict-first): L2 keeps the gathered D of the chains
      // in the window instead
      const bool qj = (sq[s] >> j) & 1u;
      __stcs(Dout + s * 8 + j, qj ? __ldcs(R + s * 8 + j) + ((a0 + a1) + (a2 + a3)) : 0.0f);
    }
  }
}

// L2 policy for the gathers of D: evict-last, so that the gathered D of the chains in the
// window outlives the matrix, R and D' streams (those are loaded and stored evict-first).
RDEV uint64_t l2_evict_last_policy() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

template <bool HINT>
RDEV float4 gather4(const float* p, uint64_t pol) {
  if constexpr (HINT) {
    float4 r;
    asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
        : "l"(p), "l"(pol));
    return r;
  } else {
    return __ldg(reinterpret_cast<const float4*>(p));
  }
}

// The same sweep with two lanes per row: lane h owns the right-hand sides 4h .. 4h+3 and
// gathers them as one 16-byte load per entry, so a warp has 16 rows in flight instead of 4.
// HINT: the gathers carry the evict-last L2 policy.  PIPE: the index and value loads of a
// row's next trip of four entries are issued before this trip's gathers complete, so the
// two dependent memory round trips of a trip overlap with the previous trip's.
template <bool HINT, bool PIPE>
__global__ void __launch_bounds__(BT) k_bsweep_q(ChainList L, const int64_t* __restrict__ rp,
                                                 const int32_t* __restrict__ ci, const float* __restrict__ ah,
                                                 const uint8_t* __restrict__ sq, const float* __restrict__ R,
                                                 const float* __restrict__ Din, float* __restrict__ Dout,
                                                 const SolveState* st) {
  if (st->done) return;
  const int lane = threadIdx.x & 31;
  const int h = lane & 1;      // right-hand sides 4h .. 4h+3
  const int grp = lane >> 1;   // 16 rows of a chunk at a time
  const int64_t nw = (int64_t)gridDim.x * (BT / 32);
  const int32_t nl = (int32_t)L.hdr[0];
  const int64_t nch = L.hdr[1];
  const uint64_t pol = HINT ? l2_evict_last_policy() : 0ull;
  ChunkWalk walk;
  for (int64_t q = (int64_t)blockIdx.x * (BT / 32) + (threadIdx.x >> 5); q < nch; q += nw) {
    int64_t r0, r1;
    int32_t c;
    walk.rows(L, nl, q, r0, r1, c);
    for (int64_t s = r0 + grp; s < r1; s += 16) {
      const int64_t hi = rp[s + 1];
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
      int32_t cc[4];
      float v[4];
      auto load = [&](int64_t k) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const bool ok = k + u < hi;
          cc[u] = ok ? __ldcs(ci + k + u) : 0;
          v[u] = ok ? __ldcs(ah + k + u) : 0.0f;
        }
      };
      int64_t k = rp[s];
      if (PIPE) load(k);
      for (; k < hi; k += 4) {
        if (!PIPE) load(k);
        float4 g[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          g[u] = k + u < hi ? gather4<HINT>(Din + (int64_t)cc[u] * 8 + 4 * h, pol) : make_float4(0.f, 0.f, 0.f, 0.f);
        float vv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) vv[u] = v[u];
        if (PIPE) load(k + 4);     // slots past the row end load nothing
#pragma unroll
        for (int u = 0; u < 4; u += 2) {
          a.x = fmaf(vv[u], g[u].x, a.x);
          a.y = fmaf(vv[u], g[u].y, a.y);
          a.z = fmaf(vv[u], g[u].z, a.z);
          a.w = fmaf(vv[u], g[u].w, a.w);
          b.x = fmaf(vv[u + 1], g[u + 1].x, b.x);
          b.y = fmaf(vv[u + 1], g[u + 1].y, b.y);
          b.z = fmaf(vv[u + 1], g[u + 1].z, b.z);
          b.w = fmaf(vv[u + 1], g[u + 1].w, b.w);
        }
      }
      const unsigned m = sq[s] >> (4 * h);
      const float4 r4 = __ldcs(reinterpret_cast<const float4*>(R + s * 8 + 4 * h));
      float4 o;
      o.x = (m & 1u) ? r4.x + (a.x + b.x) : 0.0f;
      o.y = (m & 2u) ? r4.y + (a.y + b.y) : 0.0f;
      o.z = (m & 4u) ? r4.z + (a.z + b.z) : 0.0f;
      o.w = (m & 8u) ? r4.w + (a.w + b.w) : 0.0f;
      __stcs(reinterpret_cast<float4*>(Dout + s * 8 + 4 * h), o);
    }
  }
}

// X += D over the rows of the list's chains.
__global__ void k_bapply(ChainList L, double* __restrict__ X, const float* __restrict__ D,
                         const SolveState* st) {
  if (st->done) return;
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
  const int32_t nl = (int32_t)L.hdr[0];
  const int64_t nch = L.hdr[1];
  ChunkWalk walk;
  for (int64_t q = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); q < nch; q += nw) {
    int64_t r0, r1;
    int32_t c;
    walk.rows(L, nl, q, r0, r1, c);
    for (int64_t i = r0 * 8 + lane; i < r1 * 8; i += 32) X[i] += (double)D[i];
  }
}

// Block-wide exclusive scan (blockDim.x a multiple of 32, at most 1024); *total gets the
// block's sum.  sh: 32 entries of shared memory.
template <typename T>
RDEV T block_excl_scan(T v, T* total, T* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  T inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) sh[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T t = lane < nwarp ? sh[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(FULL, t, o);
      if (lane >= o) t += y;
    }
    sh[lane] = t;
  }
  __syncthreads();
  *total = sh[nwarp - 1];
  const T ex = inc - v + (wid > 0 ? sh[wid - 1] : T(0));
  __syncthreads();
  return ex;
}

// Stopping rule per chain, after a residual step over list 1 (one CTA of CTL_NT threads):
// a chain whose largest step max|r_j| is below eps stops (its sweep count is recorded)
// and leaves the list; the others are compacted in place with their chunk prefix.  The
// solve ends when the list is empty (or max_iter is reached, as in the mixed method).
// work[] accumulates the rows and entries of the residual steps ({0, 1}) and of the
// k - 1 sweeps that follow ({2, 3}).
constexpr int CTL_NT = 1024;
__global__ void __launch_bounds__(CTL_NT) k_bchain_ctl(SolveState* st, int64_t* hdr1, int32_t* id, int64_t* pre,
                                                     const int64_t* __restrict__ coff,
                                                     const int64_t* __restrict__ arp,
                                                     unsigned long long* cmax, double* clast, int64_t* citer,
                                                     double* work, int k) {
  if (st->done) return;
  __shared__ int64_t sh64[32];
  __shared__ int64_t s_keep, s_chunks;
  __shared__ double shd[4 * 32];
  const int32_t nl = (int32_t)hdr1[0];
  const int64_t it = st->iter + 1;
  const double eps = st->eps;
  if (threadIdx.x == 0) {
    s_keep = 0;
    s_chunks = 0;
  }
  unsigned long long mxb = 0ull;
  int64_t rows_old = 0, ent_old = 0, rows_new = 0, ent_new = 0;
  __syncthreads();
  for (int32_t base = 0; base < nl; base += CTL_NT) {
    const int32_t t = base + (int32_t)threadIdx.x;
    int32_t c = -1;
    int64_t keep = 0, nchk = 0;
    if (t < nl) {
      c = id[t];
      const unsigned long long b = cmax[c];
      cmax[c] = 0ull;
      mxb = b > mxb ? b : mxb;
      const double dl = __longlong_as_double((long long)(b > 0x7ff0000000000000ull ? 0x7ff0000000000000ull : b));
      clast[c] = dl;
      const int64_t r = coff[c + 1] - coff[c];
      const int64_t e = arp[coff[c + 1]] - arp[coff[c]];
      rows_old += r;
      ent_old += e;
      if (dl < eps) {
        citer[c] = it;
      } else {
        keep = 1;
        nchk = (r + BCH - 1) / BCH;
        rows_new += r;
        ent_new += e;
      }
    }
    int64_t tk, tc;
    const int64_t pk = block_excl_scan<int64_t>(keep, &tk, sh64);
    const int64_t pc = block_excl_scan<int64_t>(nchk, &tc, sh64);
    // every read of this tile happened before the scans' barriers; writes land at or
    // below the reader's own position, never in a later tile
    if (keep) {
      id[s_keep + pk] = c;
      pre[s_keep + pk] = s_chunks + pc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      s_keep += tk;
      s_chunks += tc;
    }
    __syncthreads();
  }
  double red[4] = {(double)rows_old, (double)ent_old, (double)rows_new, (double)ent_new};
  block_reduce<4, false>(red, shd);
  __shared__ unsigned long long s_mx;
  if (threadIdx.x == 0) s_mx = 0ull;
  __syncthreads();
  if (mxb) atomicMax(&s_mx, mxb);
  __syncthreads();
  if (threadIdx.x == 0) {
    pre[s_keep] = s_chunks;
    hdr1[0] = s_keep;
    hdr1[1] = s_chunks;
    const unsigned long long b = s_mx;
    st->last = __longlong_as_double((long long)(b > 0x7ff0000000000000ull ? 0x7ff0000000000000ull : b));
    st->refinements += 1;
    st->iter += 1;
    work[0] += red[0];
    work[1] += red[1];
    if (s_keep == 0) {
      st->done = 1;
      st->status = REACH_OK;
    } else if (st->iter + (k - 1) > st->max_iter) {
      st->done = 1;
      st->status = REACH_ENOTCONV;
    } else {
      st->iter += k - 1;
      work[2] += red[2] * (double)(k - 1);
      work[3] += red[3] * (double)(k - 1);
    }
  }
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

static ChainList chain_list(const reach_batch* b, int l) {
  return ChainList{b->lhdr + 2 * l, b->lid[l], b->lpre[l], b->coff};
}

// Grid of the chain-list kernels: one warp per chunk of list 0 at most.
static int chunk_grid(reach_batch* b, const void* kernel) {
  return grid_for(b->base, kernel, BT, b->chunks_all * 32);
}

static void l_bresid(reach_batch* b, bool report, cudaStream_t s) {
  reach_ctx* c = b->base;
  if (report) {
    k_bresid<true><<<chunk_grid(b, (const void*)k_bresid<true>), BT, 0, s>>>(
        chain_list(b, 0), c->a_rowptr, c->a_col, c->a_jv, c->d, b->sq, b->X, b->R, b->D[1], c->st, 63, b->cmax);
  } else {
    k_bresid<false><<<chunk_grid(b, (const void*)k_bresid<false>), BT, 0, s>>>(
        chain_list(b, 1), c->a_rowptr, c->a_col, c->a_jv, c->d, b->sq, b->X, b->R, b->D[1], c->st, 0, b->cmax);
  }
}

template <bool HINT, bool PIPE>
static void l_bsweep_q(reach_batch* b, const float* din, float* dout, cudaStream_t s) {
  reach_ctx* c = b->base;
  const void* fn = (const void*)k_bsweep_q<HINT, PIPE>;
  k_bsweep_q<HINT, PIPE><<<chunk_grid(b, fn), BT, 0, s>>>(chain_list(b, 1), c->a_rowptr, c->a_col, c->a_hi, b->sq,
                                                          b->R, din, dout, c->st);
}

// The FP32 sweep in the batch's variant (BSW_*): eight lanes per row, or two lanes per row
// with or without the evict-last gathers and the pipelined trips.
static void l_bsweep(reach_batch* b, const float* din, float* dout, cudaStream_t s) {
  reach_ctx* c = b->base;
  switch (b->sweep_variant) {
    case BSW_LANES8:
      k_bsweep<<<chunk_grid(b, (const void*)k_bsweep), BT, 0, s>>>(chain_list(b, 1), c->a_rowptr, c->a_col,
                                                                   c->a_hi, b->sq, b->R, din, dout, c->st);
      break;
    case BSW_Q_HINT: l_bsweep_q<true, false>(b, din, dout, s); break;
    case BSW_Q_PIPE: l_bsweep_q<false, true>(b, din, dout, s); break;
    case BSW_Q_HINT_PIPE: l_bsweep_q<true, true>(b, din, dout, s); break;
    default: l_bsweep_q<false, false>(b, din, dout, s); break;
  }
}

// Chain membership check: every positive entry of row s stays inside the chain of s.
// bad[0] = 1 and bad[1] = the smallest offending row on failure.
__global__ void k_chain_check(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                              const double* __restrict__ val, const int64_t* __restrict__ coff, int32_t nc,
                              unsigned long long* bad) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    int32_t lo = 0, hi = nc;  // coff[lo] <= s < coff[hi]
    while (hi - lo > 1) {
      const int32_t mid = (lo + hi) >> 1;
      if (coff[mid] <= s) lo = mid;
      else hi = mid;
    }
    const int64_t a = coff[lo], e = coff[lo + 1];
    for (int64_t k = rp[s]; k < rp[s + 1]; ++k) {
      const int64_t j = col[k];
      if (val[k] > 0.0 && (j < a || j >= e)) {
        bad[0] = 1ull;
        atomicMin(&bad[1], (unsigned long long)s);
        break;
      }
    }
  }
}

static void free_chains(reach_batch* b) {
  for (int l = 0; l < 2; ++l) {
    if (b->lid[l]) cudaFree(b->lid[l]);
    if (b->lpre[l]) cudaFree(b->lpre[l]);
    b->lid[l] = nullptr;
    b->lpre[l] = nullptr;
  }
  void* ps[] = {b->coff, b->lhdr, b->cmax, b->clast, b->citer, b->work};
  for (void* p : ps)
    if (p) cudaFree(p);
  b->coff = nullptr;
  b->lhdr = nullptr;
  b->cmax = nullptr;
  b->clast = nullptr;
  b->citer = nullptr;
  b->work = nullptr;
  b->n_chains = 0;
  b->chunks_all = 0;
}

// Installs chains with offsets h_off[0 .. nc] (host, already checked): device copies of
// the offsets, list 0 (every chain) and the per-chain state.  A captured solve graph
// holds the old pointers, so it is dropped.
static cudaError_t install_chains(reach_batch* b, int32_t nc, const int64_t* h_off) {
  cudaStream_t s = b->base->stream;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  if (b->g_exec[2]) cudaGraphExecDestroy(b->g_exec[2]);
  b->g_exec[2] = nullptr;
  b->g_key[2] = -1;
  free_chains(b);
  const size_t n1 = (size_t)nc + 1;
  if ((e = cudaMalloc((void**)&b->coff, n1 * 8)) != cudaSuccess || (e = cudaMalloc((void**)&b->lid[0], n1 * 4)) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->lid[1], n1 * 4)) != cudaSuccess || (e = cudaMalloc((void**)&b->lpre[0], n1 * 8)) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->lpre[1], n1 * 8)) != cudaSuccess || (e = cudaMalloc((void**)&b->lhdr, 4 * 8)) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->cmax, n1 * 8)) != cudaSuccess || (e = cudaMalloc((void**)&b->clast, n1 * 8)) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->citer, n1 * 8)) != cudaSuccess || (e = cudaMalloc((void**)&b->work, 4 * 8)) != cudaSuccess) {
    free_chains(b);
    return e;
  }
  std::vector<int32_t> id(nc);
  std::vector<int64_t> pre(n1), hdr(4);
  int64_t chunks = 0;
  for (int32_t c = 0; c < nc; ++c) {
    id[c] = c;
    pre[c] = chunks;
    chunks += (h_off[c + 1] - h_off[c] + BCH - 1) / BCH;
  }
  pre[nc] = chunks;
  hdr[0] = nc;
  hdr[1] = chunks;
  hdr[2] = nc;
  hdr[3] = chunks;
  e = cudaMemcpyAsync(b->coff, h_off, n1 * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->lid[0], id.data(), (size_t)nc * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->lpre[0], pre.data(), n1 * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->lhdr, hdr.data(), 4 * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->cmax, 0, n1 * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->clast, 0, n1 * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->citer, 0xff, n1 * 8, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    free_chains(b);
    return e;
  }
  b->n_chains = nc;
  b->chunks_all = chunks;
  return cudaSuccess;
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
  free_chains(b);
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
  // REACH_BSWEEP_LANES=8 selects the sweep with one lane per right-hand side;
  // REACH_BSWEEP_VARIANT=0..4 any variant (BSW_*)
  if (const char* v = std::getenv("REACH_BSWEEP_LANES")) b->sweep_variant = v[0] == '8' ? BSW_LANES8 : BSW_Q;
  if (const char* v = std::getenv("REACH_BSWEEP_VARIANT")) {
    const int x = std::atoi(v);
    if (x >= 0 && x < BSW_COUNT) b->sweep_variant = x;
  }
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
  if (e == cudaSuccess) {  // one chain until the caller names them
    const int64_t one[2] = {0, n};
    e = install_chains(b, 1, one);
  }
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

reach_status reach_batch_set_chains(reach_batch* b, int32_t n_chains, const int64_t* offsets) {
  if (!b) return bfail(nullptr, REACH_EINVAL, "reach_batch_set_chains: NULL batch");
  if (n_chains < 1 || !offsets) return bfail(b, REACH_EINVAL, "reach_batch_set_chains: need n_chains >= 1 and offsets");
  reach_ctx* c = b->base;
  const int64_t n = c->n;
  if (offsets[0] != 0 || offsets[n_chains] != n)
    return bfail(b, REACH_EINVAL, "reach_batch_set_chains: offsets must start at 0 and end at n");
  for (int32_t i = 0; i < n_chains; ++i)
    if (offsets[i + 1] < offsets[i]) return bfail(b, REACH_EINVAL, "reach_batch_set_chains: offsets must not decrease");
  cudaStream_t s = c->stream;
  int64_t* doff = nullptr;
  unsigned long long* bad = nullptr;
  unsigned long long hbad[2] = {0ull, ~0ull};
  cudaError_t e = balloc(&doff, (int64_t)n_chains + 1);
  if (e == cudaSuccess) e = balloc(&bad, 2);
  if (e == cudaSuccess) e = cudaMemcpyAsync(doff, offsets, sizeof(int64_t) * ((size_t)n_chains + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bad, hbad, sizeof(hbad), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    k_chain_check<<<grid_for(c, (const void*)k_chain_check, BT, n), BT, 0, s>>>(n, c->rowptr, c->col, c->val, doff,
                                                                              n_chains, bad);
    e = cudaMemcpyAsync(hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  bfree(doff);
  bfree(bad);
  if (e != cudaSuccess) return bcuda(b, e, "reach_batch_set_chains");
  if (hbad[0])
    return bfail(b, REACH_EINVAL, "reach_batch_set_chains: row " + std::to_string(hbad[1]) +
                                      " has an entry outside its chain");
  e = install_chains(b, n_chains, offsets);
  if (e != cudaSuccess) {
    // the batch keeps working as one chain
    const int64_t one[2] = {0, n};
    reach_status r = bcuda(b, e, "reach_batch_set_chains");
    install_chains(b, 1, one);
    return r;
  }
  return REACH_OK;
}

reach_status reach_batch_chain_info(reach_batch* b, int64_t* iters, double* last) {
  if (!b) return bfail(nullptr, REACH_EINVAL, "reach_batch_chain_info: NULL batch");
  cudaStream_t s = b->base->stream;
  cudaError_t e = cudaSuccess;
  if (iters) e = cudaMemcpyAsync(iters, b->citer, sizeof(int64_t) * (size_t)b->n_chains, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && last)
    e = cudaMemcpyAsync(last, b->clast, sizeof(double) * (size_t)b->n_chains, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? REACH_OK : bcuda(b, e, "reach_batch_chain_info");
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

reach_status reach_batch_autotune(reach_batch* b, int32_t* variant, double* sweep_ms, int32_t* refine_k) {
  if (!b) return bfail(nullptr, REACH_EINVAL, "reach_batch_autotune: NULL batch");
  if (!b->have_classes) return bfail(b, REACH_ESTATE, "reach_batch_autotune: call reach_batch_precompute first");
  if (b->n_chains < 1 || !b->lid[0]) return bfail(b, REACH_ESTATE, "reach_batch_autotune: no chain lists");
  reach_ctx* c = b->base;
  cudaStream_t s = c->stream;
  const int64_t n = c->n;
  const int32_t nc = b->n_chains;
  // a fresh state: every chain active, nothing done, finite vectors
  cudaError_t e = cudaMemsetAsync(c->st, 0, sizeof(SolveState), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->lid[1], b->lid[0], (size_t)nc * 4, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->lpre[1], b->lpre[0], (size_t)(nc + 1) * 8, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->lhdr + 2, b->lhdr, 2 * 8, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->R, 0, sizeof(float) * (size_t)n * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->D[0], 0, sizeof(float) * (size_t)n * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->D[1], 0, sizeof(float) * (size_t)n * 8, s);
  if (e != cudaSuccess) return bcuda(b, e, "reach_batch_autotune");
  k_batch_init_x<<<grid_for(c, (const void*)k_batch_init_x, BT, n * 8), BT, 0, s>>>(n, b->one, b->X);
  auto time_it = [&](const std::function<void()>& launch, int reps, float* avg) -> cudaError_t {
    launch();  // warm-up
    cudaError_t te = cudaEventRecord(c->ev0, s);
    for (int r = 0; r < reps && te == cudaSuccess; ++r) launch();
    if (te == cudaSuccess) te = cudaEventRecord(c->ev1, s);
    if (te == cudaSuccess) te = cudaEventSynchronize(c->ev1);
    float ms = 0.f;
    if (te == cudaSuccess) te = cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    if (te == cudaSuccess) te = cudaGetLastError();
    *avg = ms / (float)reps;
    return te;
  };
  int best = BSW_Q;
  float best_ms = 0.f;
  for (int v = 0; v < BSW_COUNT && e == cudaSuccess; ++v) {
    b->sweep_variant = v;
    float ms = 0.f;
    e = time_it([&] { l_bsweep(b, b->D[0], b->D[1], s); }, 3, &ms);
    if (e == cudaSuccess && (v == 0 || ms < best_ms)) {
      best = v;
      best_ms = ms;
    }
  }
  b->sweep_variant = best;
  // the FP64 residual step, for the refinement period
  float resid_ms = 0.f;
  if (e == cudaSuccess) e = time_it([&] { l_bresid(b, false, s); }, 2, &resid_ms);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->cmax, 0, (size_t)nc * 8, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bcuda(b, e, "reach_batch_autotune");
  // N sweeps cost N t + (N / k) c for the residual steps plus about k / 2 sweeps that a
  // chain runs past its stopping point (it stops only at a check): k = sqrt(2 N c / t),
  // N = 500 (the sweep count of the batched chains here), even, in [8, 62]
  const double k_opt = std::sqrt(2.0 * 500.0 * (double)resid_ms / std::max((double)best_ms, 1e-6));
  int k = (int)std::lround(k_opt / 2.0) * 2;
  k = std::min(62, std::max(8, k));
  b->tuned_k = k;
  if (variant) *variant = best;
  if (sweep_ms) *sweep_ms = best_ms;
  if (refine_k) *refine_k = k;
  return REACH_OK;
}

reach_status reach_batch_solve(reach_batch* b, double eps, int64_t max_iter, int32_t refine_k,
                               double* x_out, int32_t flags, reach_info* info) {
  if (!b) return bfail(nullptr, REACH_EINVAL, "reach_batch_solve: NULL batch");
  if (!b->have_classes) return bfail(b, REACH_ESTATE, "reach_batch_solve: call reach_batch_precompute first");
  if (b->n_chains < 1 || !b->lid[0]) return bfail(b, REACH_ESTATE, "reach_batch_solve: no chain lists (a failed reach_batch_set_chains)");
  if (!(eps > 0.0) || max_iter < 1) return bfail(b, REACH_EINVAL, "reach_batch_solve: bad eps or max_iter");
  // default period 32: the FP64 residual costs about five FP32 sweeps here, and longer
  // periods barely change the sweep count
  if (refine_k == 0) refine_k = b->tuned_k > 0 ? b->tuned_k : 32;
  if (refine_k < 2 || refine_k > 62 || (refine_k & 1))
    return bfail(b, REACH_EINVAL, "reach_batch_solve: refine_k must be even in [2, 62]");
  if (b->tuned_k == 0 && std::getenv("REACH_AUTOTUNE") && std::getenv("REACH_AUTOTUNE")[0] == '1') {
    int32_t v = 0, kk = 0;
    double ms = 0.0;
    const reach_status ts = reach_batch_autotune(b, &v, &ms, &kk);
    if (ts != REACH_OK) return ts;
  }
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
  const int kref = refine_k;
  const int32_t nc = b->n_chains;
  k_batch_init_x<<<grid_for(c, (const void*)k_batch_init_x, BT, n * 8), BT, 0, s>>>(n, b->one, b->X);
  // list 1 starts as every chain; per-chain state cleared
  e = cudaMemcpyAsync(b->lid[1], b->lid[0], (size_t)nc * 4, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->lpre[1], b->lpre[0], (size_t)(nc + 1) * 8, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->lhdr + 2, b->lhdr, 2 * 8, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->cmax, 0, (size_t)nc * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->clast, 0, (size_t)nc * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->citer, 0xff, (size_t)nc * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->work, 0, 4 * 8, s);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev0, s);
  if (e == cudaSuccess) {
    // the graph holds the chain-list pointers: set_chains drops it when they change
    const int64_t key = (((n * 1000003LL + c->m_q) * 64 + kref) * 1000003LL + b->chunks_all * 31 + nc) * 8 +
                        b->sweep_variant;
    e = run_loop(c, b->g_exec[2], b->g_key[2], key, [&](cudaStream_t cs, cudaGraphConditionalHandle, int) {
      l_bresid(b, false, cs);
      k_bchain_ctl<<<1, CTL_NT, 0, cs>>>(c->st, b->lhdr + 2, b->lid[1], b->lpre[1], b->coff, c->a_rowptr, b->cmax,
                                         b->clast, b->citer, b->work, kref);
      // kref - 1 FP32 sweeps: D[1] -> D[0] -> ...; kref even, so the last lands in D[0]
      for (int j = 1; j < kref; ++j) {
        const float* din = (j & 1) ? b->D[1] : b->D[0];
        float* dout = (j & 1) ? b->D[0] : b->D[1];
        l_bsweep(b, din, dout, cs);
      }
      k_bapply<<<chunk_grid(b, (const void*)k_bapply), BT, 0, cs>>>(chain_list(b, 1), b->X, b->D[0], c->st);
    });
  }
  if (e == cudaSuccess) {
    l_bresid(b, true, s);
    launch_finalize_resid(s, c->st);
    k_bout<<<grid_for(c, (const void*)k_bout, BT, n * b->k), BT, 0, s>>>(n, b->k, b->X, xdev);
    e = cudaEventRecord(c->ev1, s);
  }
  double work[4] = {0.0, 0.0, 0.0, 0.0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, c->st, sizeof(hs), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(work, b->work, sizeof(work), cudaMemcpyDeviceToHost, s);
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
    // over the rows each step actually visited (converged chains drop out):
    // residual steps: 8 B value + 4 B index per entry; per row 8 B rowptr, 64 B X read,
    // 2 x 32 B R and D written, 1 B mask.  Sweeps: 4 + 4 B per entry; per row 8 B rowptr,
    // 32 B R read, 32 B D written, 1 B mask.  X += D once per period: 160 B per row.
    // Gathers of X and D are not counted.
    info->bytes_moved = work[1] * 12.0 + work[0] * 137.0 + work[3] * 8.0 + work[2] * 73.0 +
                        work[2] / (double)(kref - 1) * 160.0;
    info->status = hs.status;
    info->refinements = hs.refinements;
    info->err_bound = INFINITY;   // no norm bound per goal set is computed for batches
  }
  if (hs.status != REACH_OK) bfail(b, REACH_ENOTCONV, "reach_batch_solve: max_iter reached before the stopping rule held");
  return (reach_status)hs.status;
}

}  // extern "C"
