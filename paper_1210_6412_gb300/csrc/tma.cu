// FP32 correction sweep of the mixed method with the row data staged through shared
// memory by the Tensor Memory Accelerator: d' = r + Aj_hi d (Jacobi form, as k_sweep32).
//
// A warp owns a row (rows from a device counter).  Its lane 0 issues 1-D bulk copies
// (cp.async.bulk, completion counted on an mbarrier) of the row's values and column
// indices, in segments of TMA_SEG entries, into a private ring of TMA_ST stages; the lanes
// consume a segment from shared memory (gathering d from L1 / L2) while the next ones are
// in flight.  Per SM this keeps far more bytes in flight than register-staged loads, which
// is what a streaming sweep needs to approach HBM bandwidth.  Segments start and end on
// 8-entry boundaries (bulk copies need 16-byte aligned addresses and sizes); entries of the
// neighbouring rows that this pulls in are masked.  Every wait is bounded: a wait that runs
// out marks the solve failed, drains the copies still in flight (again bounded) and leaves.
#include <cstdint>

#include "common.cuh"
#include "internal.h"

namespace reach {

constexpr int TMA_SEG = 512;   // entries per stage
constexpr int TMA_ST = 4;      // stages per warp
constexpr int TMA_WARPS = 8;   // warps per CTA
constexpr unsigned TMA_SPIN = 1u << 22;

RDEV uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

RDEV void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}

RDEV void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

RDEV void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

RDEV void mbar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

RDEV void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

RDEV bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase `parity` of bar to complete.
RDEV bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (unsigned spin = 0; spin < TMA_SPIN; ++spin) {
    if (mbar_test(bar, parity)) return true;
    if (spin > 64) __nanosleep(32);
  }
  return false;
}

template <typename IT>
__global__ void __launch_bounds__(TMA_WARPS * 32, 2) k_sweep32_tma(int64_t nq, const int64_t* __restrict__ rp,
                                                               const IT* __restrict__ ci,
                                                               const float* __restrict__ ah,
                                                               const float* __restrict__ r32,
                                                               const float* __restrict__ din,
                                                               float* __restrict__ dout, SolveState* st,
                                                               unsigned* ctr) {
  if (st->done) return;
  constexpr int HI_B = TMA_SEG * 4, CI_B = TMA_SEG * (int)sizeof(IT), STAGE_B = HI_B + CI_B;
  extern __shared__ __align__(128) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* ring = smem + warp * (TMA_ST * STAGE_B);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + TMA_WARPS * TMA_ST * STAGE_B) + warp * TMA_ST;
  if (lane == 0) {
    for (int s = 0; s < TMA_ST; ++s) mbar_init(&bars[s]);
    mbar_init_fence();
  }
  __syncwarp();
  uint32_t parity = 0;    // bit s: parity of the next completion of stage s
  uint32_t pending = 0;   // bit s: a copy into stage s is in flight
  bool failed = false;
  // lane 0: copy segment `seg` of [a0, a1) into stage s
  auto issue = [&](int s, int64_t a0, int64_t a1, int seg) {
    const int64_t k0 = a0 + (int64_t)seg * TMA_SEG;
    const uint32_t cnt = (uint32_t)min((int64_t)TMA_SEG, a1 - k0);
    proxy_fence();
    mbar_expect(&bars[s], cnt * (4u + (uint32_t)sizeof(IT)));
    bulk_load(ring + s * STAGE_B, ah + k0, cnt * 4u, &bars[s]);
    bulk_load(ring + s * STAGE_B + HI_B, ci + k0, cnt * (uint32_t)sizeof(IT), &bars[s]);
  };
  for (int64_t i = warp_fetch_row(ctr); i < nq && !failed; i = warp_fetch_row(ctr)) {
    const int64_t lo = rp[i], hi = rp[i + 1];
    const int64_t a0 = lo & ~int64_t(7), a1 = (hi + 7) & ~int64_t(7);
    const int nseg = (int)((a1 - a0 + TMA_SEG - 1) / TMA_SEG);
    if (lane == 0)
      for (int g = 0; g < nseg && g < TMA_ST; ++g) issue(g, a0, a1, g);
    pending = 0;
    for (int g = 0; g < nseg && g < TMA_ST; ++g) pending |= 1u << g;
    float acc = 0.0f;
    for (int g = 0; g < nseg; ++g) {
      const int s = g % TMA_ST;
      // every lane waits (each needs the completed phase before reading the stage), and
      // the outcome is made warp-uniform: a lane that gave up takes the whole warp out,
      // so no lane reaches the warp-wide shuffles below without the others
      if (!__all_sync(0xffffffffu, mbar_wait(&bars[s], (parity >> s) & 1u))) {
        failed = true;
        break;
      }
      parity ^= 1u << s;
      pending &= ~(1u << s);
      const int64_t k0 = a0 + (int64_t)g * TMA_SEG;
      const int cnt = (int)min((int64_t)TMA_SEG, a1 - k0);
      const float* sh = reinterpret_cast<const float*>(ring + s * STAGE_B);
      const IT* sc = reinterpret_cast<const IT*>(ring + s * STAGE_B + HI_B);
      // every lane owns slots lane, lane + 32, ... of the segment: all 16 gathers of d are
      // independent and in flight together (the row's own entries only)
      float part[TMA_SEG / 32];
#pragma unroll
      for (int u = 0; u < TMA_SEG / 32; ++u) {
        const int j = lane + 32 * u;
        const int64_t k = k0 + j;
        part[u] = (j < cnt && k >= lo && k < hi) ? sh[j] * __ldg(din + (int)sc[j]) : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < TMA_SEG / 32; ++u) acc += part[u];
      __syncwarp();
      if (g + TMA_ST < nseg) {
        if (lane == 0) issue(s, a0, a1, g + TMA_ST);
        pending |= 1u << s;
      }
    }
    if (failed) break;
    acc = warp_sum(acc);
    if (lane == 0) dout[i] = r32[i] + acc;
  }
  if (failed) {
    // let the copies still in flight land before the shared memory goes away
    for (int s = 0; s < TMA_ST; ++s)
      if ((pending >> s) & 1u) mbar_wait(&bars[s], (parity >> s) & 1u);
    if (lane == 0) {
      st->status = REACH_ETIMEOUT;
      st->done = 1;
    }
  }
}

template <typename IT>
static size_t tma_smem() {
  return (size_t)TMA_WARPS * TMA_ST * (TMA_SEG * (4 + sizeof(IT))) + TMA_WARPS * TMA_ST * sizeof(uint64_t);
}

template <typename IT>
static cudaError_t launch_tma(reach_ctx* c, const IT* ci, const float* din, float* dout, cudaStream_t s,
                              unsigned* ctr) {
  const void* fn = (const void*)k_sweep32_tma<IT>;
  const size_t sm = tma_smem<IT>();
  // the attribute belongs to the function on the current device: set it on every launch
  // (cheap) rather than once per process
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, TMA_WARPS * 32, sm);
  if (e != cudaSuccess) return e;
  const int64_t warps_needed = c->n_q;
  int grid = c->sm_count * (per_sm > 0 ? per_sm : 1);
  if ((int64_t)grid * TMA_WARPS > warps_needed) grid = (int)((warps_needed + TMA_WARPS - 1) / TMA_WARPS);
  if (grid < 1) grid = 1;
  k_sweep32_tma<IT><<<grid, TMA_WARPS * 32, sm, s>>>(c->n_q, c->a_rowptr, ci, c->a_hi, c->r32, din, dout, c->st, ctr);
  return cudaGetLastError();
}

cudaError_t sweep32_tma(reach_ctx* c, const float* din, float* dout, cudaStream_t s, unsigned* ctr) {
  if (c->a_col16) return launch_tma<uint16_t>(c, c->a_col16, din, dout, s, ctr);
  return launch_tma<int32_t>(c, c->a_col, din, dout, s, ctr);
}

}  // namespace reach
