// Strongly connected components of the digraph of A over S?, their levels in the
// condensation, and the Jacobi iteration run one level at a time (§8: the paper
// proposes taking the SCCs of the chain in reverse topological order, since the
// matrices of single components differ in size and density from the whole).
//
// Decomposition (device only, one conditional-while graph per stage):
//   1. trimming: a row without predecessors or without successors among the rows not
//      yet removed is a component of its own; removal lowers its neighbours' counts,
//      a queue carries the rows whose count reaches zero.  This peels every acyclic
//      part of the digraph in O(edges).
//   2. colouring on the cyclic core that is left: every row takes the largest row
//      index that reaches it (max-label propagation to a fixed point); a row that keeps
//      its own index is a root, and the rows of the root's colour that reach it (a
//      backward search inside the colour) are its component.  Repeated on what is left.
//      Each component is labelled by its largest row index.
//   3. levels: Kahn's peeling of the condensation from its sinks; a component's level
//      is one above the highest component it has an edge to.
// Rows are then ordered by level (components contiguous inside a level).
//
// Solve: level 0 first.  A level made of single-row components is exact after one
// sweep, written in place (its rows read only lower, finished levels).  Any other
// level runs the double-buffered Jacobi sweep of §3.1 on its own rows until
// max|x' - x| < eps over them.
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>

#include <cooperative_groups.h>

#include <vector>

#include "common.cuh"
#include "internal.h"

namespace reach {

constexpr int SCC_NT = 256;
constexpr int SCC_CHUNK = 256;          // members of a component handed out per work item

enum : int32_t {
  PH_TRIM_INIT = 0, PH_TRIM, PH_COLOR_INIT, PH_PROP, PH_ROOTS, PH_BWD, PH_MERGE,
  PH_LV_INIT, PH_LV_ROUND, PH_DONE
};

struct SccState {
  int32_t phase;
  int32_t cur;            // frontier ping-pong index
  uint32_t count[2];      // frontier sizes
  int32_t changed;        // a colour grew in this propagation pass
  int32_t round;          // colouring rounds finished
  int32_t max_rounds;
  int32_t exact;          // 0 once the round cap merged the cyclic core into one block
  int32_t core_max;       // largest row index of the cyclic core
  int32_t level;          // Kahn level being expanded
  int32_t n_levels;
  int32_t pad;
  int64_t remaining;      // rows without a component
  int64_t n_scc, largest, n_trivial;
  // block solve
  int32_t blk_level;      // level being solved
  int32_t pad2;
  int64_t blk_sweeps;     // sweeps of the current level
  double bytes;           // algorithmic bytes of the sweeps run
  int64_t passes;         // passes of the decomposition (its sequential depth)
};

struct SccPlan {
  int32_t* lab = nullptr;      // component label per row (largest row index in it)
  int32_t* color = nullptr;
  uint32_t* indeg = nullptr;   // trimming counts; later: unresolved out-edges per label
  uint32_t* outdeg = nullptr;  // trimming counts; later: member fill per label
  uint32_t* msize = nullptr;   // rows per label
  int64_t* mstart = nullptr;   // first member position per label
  int64_t* mnnz = nullptr;     // stored entries of the label's rows
  int32_t* mem = nullptr;      // rows grouped by label
  int32_t* lvl = nullptr;      // level per label
  uint32_t* lrows = nullptr;   // rows per level
  int64_t* lrow = nullptr;     // first position per level (n_levels + 1 used)
  int64_t* lnnz = nullptr;     // stored entries per level
  uint32_t* lfill = nullptr;
  int64_t* lbase = nullptr;    // offset of the label inside its level
  uint8_t* lkind = nullptr;    // 1: the level holds a component of more than one row
  int32_t* perm = nullptr;     // position -> row, ordered by level
  int32_t* rlev = nullptr;     // level of every row
  double* part = nullptr;      // max|x' - x| slots of the persistent solve (three, as integer bits)
  unsigned* bar = nullptr;     // grid barrier: arrival count, generation, error flag
  unsigned* pc = nullptr;      // counters of the persistent decomposition (frontiers, flags)
  SccState* ss = nullptr;
  bool ready = false;
  reach_scc_info info{};
  std::vector<int64_t> h_lrow, h_lnnz;   // level table on the host (plans the launches of a solve)
};

// ---------------------------------------------------------------- decomposition

// Grid-wide barrier of a cooperative launch (all CTAs resident).  Bounded: a CTA that
// waits past the limit raises the error word, and every CTA leaves at its next barrier.
struct GridBar {
  unsigned* count;
  unsigned* gen;
  unsigned* err;
};

RDEV bool grid_barrier(const GridBar& gb) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = gb.gen;
    const unsigned g = *vgen;
    __threadfence();
    if (atomicAdd(gb.count, 1u) == gridDim.x - 1) {
      atomicExch(gb.count, 0u);
      __threadfence();
      atomicAdd(gb.gen, 1u);
    } else {
      unsigned spins = 0;
      while (*vgen == g) {
        if (++spins > (1u << 24)) {   // about a second
          atomicExch(gb.err, 1u);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile unsigned*)gb.err == 0u;
}


RDEV uint32_t push_slot(uint32_t* count) { return atomicAdd(count, 1u); }

// One pass of the decomposition phase stored in ss->phase; the last CTA to finish
// moves the state machine on and sets st->done when the components are final.
template <int G>
__global__ void __launch_bounds__(SCC_NT) k_scc_step(int64_t nq, const int64_t* __restrict__ arp,
                                                     const int32_t* __restrict__ acol,
                                                     const int64_t* __restrict__ trp,
                                                     const int32_t* __restrict__ tcol, int32_t* lab,
                                                     int32_t* color, uint32_t* indeg, uint32_t* outdeg,
                                                     int32_t* q0, int32_t* q1, SccState* ss,
                                                     SolveState* st, unsigned* ticket) {
  const int ph = ss->phase;
  if (ph >= PH_LV_INIT) return;
  const int cur = ss->cur;
  const int32_t* qc = cur ? q1 : q0;
  int32_t* qn = cur ? q0 : q1;
  uint32_t* cnext = &ss->count[cur ^ 1];
  const uint32_t ncur = ss->count[cur];
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  RowGroups rg = RowGroups::make<G>();
  __shared__ int any_change;
  if (threadIdx.x == 0) any_change = 0;
  __syncthreads();

  switch (ph) {
    case PH_TRIM_INIT:
      for (int64_t v = tid; v < nq; v += nth) {
        const uint32_t od = (uint32_t)(arp[v + 1] - arp[v]);
        const uint32_t id = (uint32_t)(trp[v + 1] - trp[v]);
        outdeg[v] = od;
        indeg[v] = id;
        color[v] = -1;
        if (od == 0 || id == 0) {
          lab[v] = (int32_t)v;
          qn[push_slot(cnext)] = (int32_t)v;
        } else {
          lab[v] = -1;
        }
      }
      break;
    case PH_TRIM:
      for (int64_t i = rg.first; i < (int64_t)ncur; i += rg.stride) {
        const int32_t v = qc[i];
        for (int64_t k = arp[v] + rg.lane; k < arp[v + 1]; k += G) {
          const int32_t u = acol[k];
          if (__ldcg(lab + u) != -1) continue;
          if (atomicSub(indeg + u, 1u) == 1u && atomicCAS(lab + u, -1, u) == -1) qn[push_slot(cnext)] = u;
        }
        for (int64_t k = trp[v] + rg.lane; k < trp[v + 1]; k += G) {
          const int32_t u = tcol[k];
          if (__ldcg(lab + u) != -1) continue;
          if (atomicSub(outdeg + u, 1u) == 1u && atomicCAS(lab + u, -1, u) == -1) qn[push_slot(cnext)] = u;
        }
      }
      break;
    case PH_COLOR_INIT:
      for (int64_t v = tid; v < nq; v += nth) {
        if (lab[v] != -1) continue;
        color[v] = (int32_t)v;
        if (ss->round == 0) atomicMax(&ss->core_max, (int32_t)v);
      }
      break;
    case PH_PROP:
      for (int64_t v = rg.first; v < nq; v += rg.stride) {
        if (__ldcg(lab + v) != -1) continue;
        const int32_t c = __ldcg(color + v);
        for (int64_t k = arp[v] + rg.lane; k < arp[v + 1]; k += G) {
          const int32_t u = acol[k];
          if (__ldcg(lab + u) != -1) continue;
          if (__ldcg(color + u) < c) {
            atomicMax(color + u, c);
            any_change = 1;
          }
        }
      }
      break;
    case PH_ROOTS:
      for (int64_t v = tid; v < nq; v += nth) {
        if (lab[v] == -1 && color[v] == (int32_t)v) {
          lab[v] = (int32_t)v;
          qn[push_slot(cnext)] = (int32_t)v;
        }
      }
      break;
    case PH_BWD:
      for (int64_t i = rg.first; i < (int64_t)ncur; i += rg.stride) {
        const int32_t v = qc[i];
        const int32_t cv = color[v];
        for (int64_t k = trp[v] + rg.lane; k < trp[v + 1]; k += G) {
          const int32_t u = tcol[k];
          if (__ldcg(lab + u) != -1 || __ldcg(color + u) != cv) continue;
          if (atomicCAS(lab + u, -1, cv) == -1) qn[push_slot(cnext)] = u;
        }
      }
      break;
    case PH_MERGE:
      for (int64_t v = tid; v < nq; v += nth)
        if (color[v] >= 0) lab[v] = ss->core_max;
      break;
    default:
      break;
  }

  __syncthreads();
  if (threadIdx.x == 0 && any_change) ss->changed = 1;
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!(last && threadIdx.x == 0)) return;
  __threadfence();
  *ticket = 0u;
  const uint32_t pushed = atomicAdd(cnext, 0u);
  auto flip = [&]() {
    ss->count[cur] = 0u;
    ss->cur = cur ^ 1;
  };
  auto finish = [&]() {
    ss->phase = PH_LV_INIT;
    st->done = 1;
    st->status = REACH_OK;
  };
  switch (ph) {
    case PH_TRIM_INIT:
      ss->remaining = nq - (int64_t)pushed;
      flip();
      ss->phase = PH_TRIM;
      break;
    case PH_TRIM:
      ss->remaining -= pushed;
      flip();
      if (pushed == 0) {
        if (ss->remaining == 0) finish();
        else ss->phase = PH_COLOR_INIT;
      }
      break;
    case PH_COLOR_INIT:
      ss->changed = 0;
      ss->phase = PH_PROP;
      break;
    case PH_PROP:
      if (ss->changed) ss->changed = 0;
      else ss->phase = PH_ROOTS;
      break;
    case PH_ROOTS:
      ss->remaining -= pushed;
      flip();
      ss->phase = PH_BWD;
      break;
    case PH_BWD:
      ss->remaining -= pushed;
      flip();
      if (pushed == 0) {
        ss->round += 1;
        if (ss->remaining == 0) finish();
        else if (ss->round >= ss->max_rounds) ss->phase = PH_MERGE;
        else ss->phase = PH_COLOR_INIT;
      }
      break;
    case PH_MERGE:
      ss->exact = 0;
      ss->remaining = 0;
      finish();
      break;
    default:
      break;
  }
}

// Queue every member chunk of label L (the chunk is its first position in mem).
RDEV void push_chunks(int32_t L, const uint32_t* msize, const int64_t* mstart, int32_t* qn, uint32_t* cnext) {
  const uint32_t nch = (msize[L] + SCC_CHUNK - 1) / SCC_CHUNK;
  const uint32_t base = atomicAdd(cnext, nch);
  for (uint32_t j = 0; j < nch; ++j) qn[base + j] = (int32_t)(mstart[L] + (int64_t)j * SCC_CHUNK);
}

// One Kahn pass: a group of g lanes per queued chunk, the lanes taking the chunk's members
// in turn.  g is the largest power of two up to 32 that still gives every chunk its own
// group in one trip, so a pass of many one-row components (an acyclic chain) runs in one
// trip while a few big chunks get a warp each.  Every member releases its edges from other
// components; a component whose count of unreleased outgoing edges reaches 0 gets level
// h + 1 and queues its chunks.
RDEV void release_chunks(uint32_t size, const int32_t* __restrict__ qc, const int32_t* __restrict__ lab,
                         const uint32_t* __restrict__ msize, const int64_t* __restrict__ mstart,
                         const int32_t* __restrict__ mem, const int64_t* __restrict__ trp,
                         const int32_t* __restrict__ tcol, uint32_t* out_edges, int32_t* lvl, int32_t h,
                         int32_t* qn, uint32_t* cn, int64_t tid, int64_t nth) {
  int g = 32;
  while (g > 1 && (int64_t)size * g > nth) g >>= 1;
  const int lane = (int)(tid & (g - 1));
  for (int64_t w = tid / g; w < (int64_t)size; w += nth / g) {
    const int64_t p0 = qc[w];
    const int32_t L = lab[mem[p0]];
    const int64_t p1 = std::min<int64_t>(p0 + SCC_CHUNK, mstart[L] + msize[L]);
    for (int64_t p = p0 + lane; p < p1; p += g) {
      const int32_t v = mem[p];
      for (int64_t k = trp[v]; k < trp[v + 1]; ++k) {
        const int32_t Lu = lab[tcol[k]];
        if (Lu == L) continue;
        if (atomicSub(out_edges + Lu, 1u) == 1u) {
          lvl[Lu] = h + 1;
          push_chunks(Lu, msize, mstart, qn, cn);
        }
      }
    }
  }
}

// ---- the same decomposition in cooperative launches (grid barriers between passes)
//
// Frontier bookkeeping shared by every queue-driven pass: step f reads the frontier
// q[f & 1] of size pc[f % 3], pushes into q[(f + 1) & 1] / pc[(f + 1) % 3], and clears
// pc[(f + 2) % 3] for the step after (that count was last read two barriers earlier).
// Every CTA reads the same sizes after a barrier, so all of them take the same branches.
enum : int { PC_CHG = 3, PC_CORE = 6, PC_FAIL = 7, PC_ALLSINK = 8 };

RDEV unsigned ld_vol(const unsigned* p) { return *(const volatile unsigned*)p; }

template <int G>
__global__ void __launch_bounds__(SCC_NT, 2) k_scc_persist(int64_t nq, const int64_t* __restrict__ arp,
                                                          const int32_t* __restrict__ acol,
                                                          const int64_t* __restrict__ trp,
                                                          const int32_t* __restrict__ tcol, int32_t* lab,
                                                          int32_t* color, uint32_t* indeg, uint32_t* outdeg,
                                                          int32_t* lvl, int32_t* q0, int32_t* q1, unsigned* pc,
                                                          int32_t max_rounds, int64_t budget, SccState* ss,
                                                          GridBar gb) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  RowGroups rg = RowGroups::make<G>();
  int64_t f = 0, seen = 0, passes = 0;
  // Phase 1, trimming from the sinks (Kahn's order): a row whose successors are all gone
  // is a component of its own, and the pass that frees it is its level.  Removing such
  // rows never changes an in-degree that matters (their successors left before them),
  // so the in-degrees stay exact for phase 2.  On an acyclic system this alone yields
  // every component and level.
  for (int64_t v = tid; v < nq; v += nth) {
    const uint32_t od = (uint32_t)(arp[v + 1] - arp[v]);
    outdeg[v] = od;
    indeg[v] = (uint32_t)(trp[v + 1] - trp[v]);
    color[v] = -1;
    if (od == 0) {
      lab[v] = (int32_t)v;
      lvl[v] = 0;
      q1[atomicAdd(pc + 1, 1u)] = (int32_t)v;
    } else {
      lab[v] = -1;
    }
  }
  if (lead) pc[2] = 0u;
  if (!grid_barrier(gb)) return;
  f = 1;
  for (;;) {
    const unsigned size = ld_vol(pc + f % 3);
    seen += size;
    if (size == 0 || ++passes > budget) break;
    const int32_t* qc = (f & 1) ? q1 : q0;
    int32_t* qn = (f & 1) ? q0 : q1;
    unsigned* cn = pc + (f + 1) % 3;
    if (lead) pc[(f + 2) % 3] = 0u;
    for (int64_t i = rg.first; i < (int64_t)size; i += rg.stride) {
      const int32_t v = qc[i];
      for (int64_t k = trp[v] + rg.lane; k < trp[v + 1]; k += G) {
        const int32_t u = tcol[k];
        if (__ldcg(lab + u) != -1) continue;
        if (atomicSub(outdeg + u, 1u) == 1u && atomicCAS(lab + u, -1, u) == -1) {
          lvl[u] = (int32_t)f;
          qn[atomicAdd(cn, 1u)] = u;
        }
      }
    }
    if (!grid_barrier(gb)) return;
    ++f;
  }
  if (seen >= nq) {   // acyclic: every component is one row, and its level is known
    if (lead) {
      pc[PC_ALLSINK] = 1u;
      ss->n_levels = (int32_t)(f - 1);
      ss->n_scc = nq;
      ss->n_trivial = nq;
      ss->largest = nq > 0 ? 1 : 0;
      ss->round = 0;
      ss->exact = 1;
      ss->passes = passes;
      if (passes > budget) pc[PC_FAIL] = 1u;
    }
    return;
  }
  // Phase 2, trimming from both ends on what is left: seeds are the rows without
  // predecessors (rows without successors are gone already)
  {
    int32_t* qn = (f & 1) ? q0 : q1;
    unsigned* cn = pc + (f + 1) % 3;
    if (lead) pc[(f + 2) % 3] = 0u;
    for (int64_t v = tid; v < nq; v += nth) {
      if (lab[v] == -1 && indeg[v] == 0u) {
        lab[v] = (int32_t)v;
        qn[atomicAdd(cn, 1u)] = (int32_t)v;
      }
    }
    if (!grid_barrier(gb)) return;
    ++f;
  }
  for (;;) {
    const unsigned size = ld_vol(pc + f % 3);
    seen += size;
    if (size == 0 || ++passes > budget) break;
    const int32_t* qc = (f & 1) ? q1 : q0;
    int32_t* qn = (f & 1) ? q0 : q1;
    unsigned* cn = pc + (f + 1) % 3;
    if (lead) pc[(f + 2) % 3] = 0u;
    for (int64_t i = rg.first; i < (int64_t)size; i += rg.stride) {
      const int32_t v = qc[i];
      for (int64_t k = arp[v] + rg.lane; k < arp[v + 1]; k += G) {
        const int32_t u = acol[k];
        if (__ldcg(lab + u) != -1) continue;
        if (atomicSub(indeg + u, 1u) == 1u && atomicCAS(lab + u, -1, u) == -1) qn[atomicAdd(cn, 1u)] = u;
      }
      for (int64_t k = trp[v] + rg.lane; k < trp[v + 1]; k += G) {
        const int32_t u = tcol[k];
        if (__ldcg(lab + u) != -1) continue;
        if (atomicSub(outdeg + u, 1u) == 1u && atomicCAS(lab + u, -1, u) == -1) qn[atomicAdd(cn, 1u)] = u;
      }
    }
    if (!grid_barrier(gb)) return;
    ++f;
  }
  // colouring rounds on the cyclic core
  int32_t round = 0;
  bool exact = true;
  while (seen < nq && passes <= budget) {
    if (round >= max_rounds) {       // keep the whole core as one block
      const int32_t core = (int32_t)ld_vol(pc + PC_CORE);
      for (int64_t v = tid; v < nq; v += nth)
        if (color[v] >= 0) lab[v] = core;
      exact = false;
      if (!grid_barrier(gb)) return;
      break;
    }
    // every row left starts with its own index as colour and seeds the first
    // propagation frontier (step f); outdeg, no longer needed, stamps queued rows
    uint32_t* stamp = outdeg;
    {
      int32_t* qn = (f & 1) ? q0 : q1;
      unsigned* cn = pc + (f + 1) % 3;
      if (lead) pc[(f + 2) % 3] = 0u;
      for (int64_t v = tid; v < nq; v += nth) {
        if (lab[v] != -1) continue;
        color[v] = (int32_t)v;
        stamp[v] = 0xffffffffu;
        qn[atomicAdd(cn, 1u)] = (int32_t)v;
        if (round == 0) atomicMax(reinterpret_cast<int*>(pc + PC_CORE), (int)v);
      }
      if (!grid_barrier(gb)) return;
      ++f;
    }
    // max-label propagation over the frontier of rows whose colour rose in the last
    // pass; a row is queued once per pass (its stamp), and reads its latest colour
    for (;;) {
      const unsigned size = ld_vol(pc + f % 3);
      if (size == 0 || ++passes > budget) break;
      const int32_t* qc = (f & 1) ? q1 : q0;
      int32_t* qn = (f & 1) ? q0 : q1;
      unsigned* cn = pc + (f + 1) % 3;
      if (lead) pc[(f + 2) % 3] = 0u;
      for (int64_t i = rg.first; i < (int64_t)size; i += rg.stride) {
        const int32_t v = qc[i];
        const int32_t cv = __ldcg(color + v);
        for (int64_t k = arp[v] + rg.lane; k < arp[v + 1]; k += G) {
          const int32_t u = acol[k];
          if (__ldcg(lab + u) != -1 || __ldcg(color + u) >= cv) continue;
          if (atomicMax(color + u, cv) < cv && atomicExch(stamp + u, (uint32_t)f) != (uint32_t)f)
            qn[atomicAdd(cn, 1u)] = u;
        }
      }
      if (!grid_barrier(gb)) return;
      ++f;
    }
    // roots seed a frontier (step f); the backward search inside each colour follows
    {
      int32_t* qn = (f & 1) ? q0 : q1;
      unsigned* cn = pc + (f + 1) % 3;
      if (lead) pc[(f + 2) % 3] = 0u;
      for (int64_t v = tid; v < nq; v += nth) {
        if (lab[v] == -1 && color[v] == (int32_t)v) {
          lab[v] = (int32_t)v;
          qn[atomicAdd(cn, 1u)] = (int32_t)v;
        }
      }
      if (!grid_barrier(gb)) return;
      ++f;
    }
    for (;;) {
      const unsigned size = ld_vol(pc + f % 3);
      seen += size;
      if (size == 0 || ++passes > budget) break;
      const int32_t* qc = (f & 1) ? q1 : q0;
      int32_t* qn = (f & 1) ? q0 : q1;
      unsigned* cn = pc + (f + 1) % 3;
      if (lead) pc[(f + 2) % 3] = 0u;
      for (int64_t i = rg.first; i < (int64_t)size; i += rg.stride) {
        const int32_t v = qc[i];
        const int32_t cv = color[v];
        for (int64_t k = trp[v] + rg.lane; k < trp[v + 1]; k += G) {
          const int32_t u = tcol[k];
          if (__ldcg(lab + u) != -1 || __ldcg(color + u) != cv) continue;
          if (atomicCAS(lab + u, -1, cv) == -1) qn[atomicAdd(cn, 1u)] = u;
        }
      }
      if (!grid_barrier(gb)) return;
      ++f;
    }
    ++round;
  }
  if (lead) {
    ss->round = round;
    ss->exact = exact ? 1 : 0;
    ss->core_max = (int32_t)ld_vol(pc + PC_CORE);
    ss->passes = passes;
    if (passes > budget) pc[PC_FAIL] = 1u;
  }
}

template <int G>
__global__ void __launch_bounds__(SCC_NT, 2) k_lvl_persist(int64_t nq, const int64_t* __restrict__ trp,
                                                          const int32_t* __restrict__ tcol,
                                                          const int32_t* __restrict__ lab,
                                                          const uint32_t* __restrict__ msize,
                                                          const int64_t* __restrict__ mstart,
                                                          const int32_t* __restrict__ mem, uint32_t* out_edges,
                                                          int32_t* lvl, int32_t* q0, int32_t* q1, unsigned* pc,
                                                          SccState* ss, GridBar gb) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  // step 0: components without edges to others are level 0
  for (int64_t L = tid; L < nq; L += nth) {
    if (lab[L] != (int32_t)L) continue;
    const uint32_t sz = msize[L];
    atomicAdd(reinterpret_cast<unsigned long long*>(&ss->n_scc), 1ull);
    if (sz == 1) atomicAdd(reinterpret_cast<unsigned long long*>(&ss->n_trivial), 1ull);
    atomicMax(reinterpret_cast<unsigned long long*>(&ss->largest), (unsigned long long)sz);
    if (out_edges[L] == 0) {
      lvl[L] = 0;
      push_chunks((int32_t)L, msize, mstart, q1, pc + 1);
    }
  }
  if (lead) pc[2] = 0u;
  if (!grid_barrier(gb)) return;
  RowGroups rg = RowGroups::make<G>();
  int64_t f = 1;
  for (;; ++f) {
    const unsigned size = ld_vol(pc + f % 3);
    if (size == 0) break;
    const int32_t h = (int32_t)(f - 1);
    const int32_t* qc = (f & 1) ? q1 : q0;
    int32_t* qn = (f & 1) ? q0 : q1;
    unsigned* cn = pc + (f + 1) % 3;
    if (lead) pc[(f + 2) % 3] = 0u;
    release_chunks(size, qc, lab, msize, mstart, mem, trp, tcol, out_edges, lvl, h, qn, cn, tid, nth);
    if (!grid_barrier(gb)) return;
  }
  if (lead) {
    ss->n_levels = (int32_t)(f - 1);
    ss->passes += f;
  }
}

// Rows per label, stored entries per label, and edges leaving each label.
template <int G>
__global__ void __launch_bounds__(SCC_NT) k_lab_stats(int64_t nq, const int64_t* __restrict__ arp,
                                                      const int32_t* __restrict__ acol,
                                                      const int32_t* __restrict__ lab, uint32_t* msize,
                                                      int64_t* mnnz, uint32_t* out_edges) {
  RowGroups rg = RowGroups::make<G>();
  for (int64_t v = rg.first; warp_has_row<G>(v, nq); v += rg.stride) {
    uint32_t cross = 0;
    int32_t L = -1;
    if (v < nq) {
      L = lab[v];
      for (int64_t k = arp[v] + rg.lane; k < arp[v + 1]; k += G) cross += lab[acol[k]] != L;
    }
    cross = group_sum<G>(cross);
    if (v < nq && rg.lane == 0) {
      atomicAdd(msize + L, 1u);
      atomicAdd(reinterpret_cast<unsigned long long*>(mnnz + L), (unsigned long long)(arp[v + 1] - arp[v]));
      if (cross) atomicAdd(out_edges + L, cross);
    }
  }
}

__global__ void k_members(int64_t nq, const int32_t* __restrict__ lab, const int64_t* __restrict__ mstart,
                          uint32_t* fill, int32_t* mem) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nq;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t L = lab[v];
    mem[mstart[L] + atomicAdd(fill + L, 1u)] = (int32_t)v;
  }
}

// Kahn's peeling of the condensation, one level per pass.
template <int G>
__global__ void __launch_bounds__(SCC_NT) k_lvl_step(int64_t nq, const int64_t* __restrict__ trp,
                                                     const int32_t* __restrict__ tcol,
                                                     const int32_t* __restrict__ lab,
                                                     const uint32_t* __restrict__ msize,
                                                     const int64_t* __restrict__ mstart,
                                                     const int32_t* __restrict__ mem, uint32_t* out_edges,
                                                     int32_t* lvl, int32_t* q0, int32_t* q1, SccState* ss,
                                                     SolveState* st, unsigned* ticket) {
  const int ph = ss->phase;
  const int cur = ss->cur;
  const int32_t* qc = cur ? q1 : q0;
  int32_t* qn = cur ? q0 : q1;
  uint32_t* cnext = &ss->count[cur ^ 1];
  const uint32_t ncur = ss->count[cur];
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  if (ph == PH_LV_INIT) {
    for (int64_t L = tid; L < nq; L += nth) {
      if (lab[L] != (int32_t)L) continue;                 // not a label
      const uint32_t sz = msize[L];
      atomicAdd(reinterpret_cast<unsigned long long*>(&ss->n_scc), 1ull);
      if (sz == 1) atomicAdd(reinterpret_cast<unsigned long long*>(&ss->n_trivial), 1ull);
      atomicMax(reinterpret_cast<unsigned long long*>(&ss->largest), (unsigned long long)sz);
      if (out_edges[L] == 0) {
        lvl[L] = 0;
        push_chunks((int32_t)L, msize, mstart, qn, cnext);
      }
    }
  } else if (ph == PH_LV_ROUND) {
    const int32_t h = ss->level;
    RowGroups rg = RowGroups::make<G>();
    release_chunks(ncur, qc, lab, msize, mstart, mem, trp, tcol, out_edges, lvl, h, qn, cnext, tid, nth);
  } else {
    return;
  }
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!(last && threadIdx.x == 0)) return;
  __threadfence();
  *ticket = 0u;
  const uint32_t pushed = atomicAdd(cnext, 0u);
  ss->count[cur] = 0u;
  ss->cur = cur ^ 1;
  if (ph == PH_LV_INIT) {
    ss->level = 0;
    ss->phase = PH_LV_ROUND;
    ss->n_levels = pushed ? 1 : 0;
    if (!pushed) {
      ss->phase = PH_DONE;
      st->done = 1;
      st->status = REACH_OK;
    }
  } else if (pushed) {
    ss->level += 1;
    ss->n_levels = ss->level + 1;
  } else {
    ss->phase = PH_DONE;
    st->done = 1;
    st->status = REACH_OK;
  }
}

// Rows and stored entries per level; a level with a component of more than one row
// needs the iterated sweep.
__global__ void k_level_sizes(int64_t nq, const int32_t* __restrict__ lab, const uint32_t* __restrict__ msize,
                              const int64_t* __restrict__ mnnz, const int32_t* __restrict__ lvl,
                              uint32_t* lrows, int64_t* lnnz, uint32_t* lfill, int64_t* lbase, uint8_t* lkind) {
  for (int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; L < nq;
       L += (int64_t)gridDim.x * blockDim.x) {
    if (lab[L] != (int32_t)L) continue;
    const int32_t h = lvl[L];
    atomicAdd(lrows + h, msize[L]);
    atomicAdd(reinterpret_cast<unsigned long long*>(lnnz + h), (unsigned long long)mnnz[L]);
    lbase[L] = atomicAdd(lfill + h, msize[L]);
    if (msize[L] > 1) lkind[h] = 1;
  }
}

__global__ void k_perm(int64_t nq, const int32_t* __restrict__ mem, const int32_t* __restrict__ lab,
                       const int64_t* __restrict__ mstart, const int32_t* __restrict__ lvl,
                       const int64_t* __restrict__ lrow, const int64_t* __restrict__ lbase, int32_t* perm) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nq;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = mem[p];
    const int32_t L = lab[v];
    perm[lrow[lvl[L]] + lbase[L] + (p - mstart[L])] = v;
  }
}

__global__ void k_level_of_row(int64_t nq, const int32_t* __restrict__ lab, const int32_t* __restrict__ lvl,
                               int32_t* out) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nq;
       v += (int64_t)gridDim.x * blockDim.x)
    out[v] = lvl[lab[v]];
}

// ---------------------------------------------------------------- block solve

// Sweep over the rows of the current level.  Single-row components: exact value in
// place.  Otherwise x' into xn and max|x' - x| into the slot.
template <int G>
__global__ void __launch_bounds__(SCC_NT) k_blk_sweep(const int64_t* __restrict__ arp,
                                                      const int32_t* __restrict__ acol,
                                                      const double* __restrict__ aval,
                                                      const double* __restrict__ bj, double* x, double* xn,
                                                      const int32_t* __restrict__ perm,
                                                      const int64_t* __restrict__ lrow,
                                                      const uint8_t* __restrict__ lkind, const SccState* ss,
                                                      const SolveState* st, unsigned long long* slot) {
  if (st->done) return;
  const int32_t h = ss->blk_level;
  const int64_t r0 = lrow[h], nr = lrow[h + 1] - r0;
  const bool cyc = lkind[h] != 0;
  RowGroups rg = RowGroups::make<G>();
  double mx = 0.0;
  for (int64_t i = rg.first; warp_has_row<G>(i, nr); i += rg.stride) {
    double s0 = 0.0, s1 = 0.0;
    int32_t v = 0;
    if (i < nr) {
      v = perm[r0 + i];
      const int64_t hi = arp[v + 1];
      int64_t k = arp[v] + rg.lane;
      for (; k + G < hi; k += 2 * G) {
        s0 = fma(aval[k], x[acol[k]], s0);
        s1 = fma(aval[k + G], x[acol[k + G]], s1);
      }
      if (k < hi) s0 = fma(aval[k], x[acol[k]], s0);
    }
    const double s = group_sum<G>(s0 + s1);
    if (i < nr && rg.lane == 0) {
      const double xv = bj[v] + s;          // Jacobi form: aval = A_ij / d_i, bj = b_i / d_i
      if (cyc) {
        const double dv = fabs(xv - x[v]);
        mx = fmax(mx, dv != dv ? __longlong_as_double(0x7ff0000000000000LL) : dv);
        xn[v] = xv;
      } else {
        x[v] = xv;
      }
    }
  }
  if (!cyc) return;
  __shared__ double sh[32];
  double a[1] = {mx};
  block_reduce<1, true>(a, sh);
  if (threadIdx.x == 0) atomic_max_nonneg(slot, a[0]);
}

// Copies x' of an iterated level into x; the last CTA applies the stopping rule of the
// level and moves to the next level (or ends the solve).
__global__ void __launch_bounds__(SCC_NT) k_blk_apply(double* x, const double* __restrict__ xn,
                                                      const int32_t* __restrict__ perm,
                                                      const int64_t* __restrict__ lrow,
                                                      const int64_t* __restrict__ lnnz,
                                                      const uint8_t* __restrict__ lkind, SccState* ss,
                                                      SolveState* st, unsigned long long* slot, unsigned* ticket) {
  if (st->done) return;
  const int32_t h = ss->blk_level;
  const int64_t r0 = lrow[h], r1 = lrow[h + 1];
  const bool cyc = lkind[h] != 0;
  if (cyc) {
    for (int64_t p = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < r1;
         p += (int64_t)gridDim.x * blockDim.x) {
      const int32_t v = perm[p];
      x[v] = xn[v];
    }
  }
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!(last && threadIdx.x == 0)) return;
  __threadfence();
  *ticket = 0u;
  const double dl = cyc ? slot_value(slot) : 0.0;
  *slot = 0ull;
  st->iter += 1;
  ss->blk_sweeps += 1;
  // entries: index + value; rows: perm, rowptr, b, d, x (+ x' out, and the copy back)
  ss->bytes += (double)lnnz[h] * 12.0 + (double)(r1 - r0) * (cyc ? 64.0 : 36.0);
  st->last = dl;
  if (!cyc || dl < st->eps) {
    ss->blk_level = h + 1;
    ss->blk_sweeps = 0;
    if (h + 1 >= ss->n_levels) {
      st->done = 1;
      st->status = REACH_OK;
    }
  }
  if (!st->done && st->iter >= st->max_iter) {
    st->done = 1;
    st->status = REACH_ENOTCONV;
  }
}

// ---------------------------------------------------------------- block solve, persistent launches

constexpr int CL_SIZE = 16;       // CTAs of the cluster that runs small levels (non-portable size)
constexpr int CL_NT = 512;

// Barrier of the launch: the whole grid (cooperative launch), or one thread-block
// cluster (hardware barrier with release / acquire semantics at cluster scope).
template <bool CLUSTER>
RDEV bool sync_all(const GridBar& gb) {
  if constexpr (CLUSTER) {
    cooperative_groups::this_cluster().sync();
    return true;
  } else {
    return grid_barrier(gb);
  }
}

// Levels [h0, h1) of the level-by-level Jacobi in one launch: the CTAs walk the levels
// in order, with a barrier after every sweep instead of a kernel boundary.  Big levels
// run on the whole GPU (a cooperative grid with grid barriers); runs of small levels, the
// components §8 expects to differ most from the whole matrix, run on one cluster of 16
// CTAs, whose hardware barrier costs far less than a grid-wide one.  A level of
// single-row components is swept once, in place, into both buffers.  A cyclic level
// ping-pongs between the buffers until max|x' - x| < eps over its rows; its final
// values are then copied into the other buffer, so lower levels always read the same in
// both.  On the grid, a level with at least a quarter of all rows is swept in natural
// row order (rows of other levels skipped), so its loads stay coalesced; other levels go
// through perm.  Sweeps, bytes and the status accumulate in the solve state across
// launches; a launch whose predecessor stopped returns at once.
template <int G, bool CLUSTER>
__global__ void __launch_bounds__(CLUSTER ? CL_NT : SCC_NT, CLUSTER ? 1 : 4) k_blk_persist(int64_t nq, const int64_t* __restrict__ arp,
                                                        const int32_t* __restrict__ acol,
                                                        const double* __restrict__ aj,
                                                        const double* __restrict__ bj, double* xa, double* xb,
                                                        const int32_t* __restrict__ perm,
                                                        const int32_t* __restrict__ rlev,
                                                        const int64_t* __restrict__ lrow,
                                                        const int64_t* __restrict__ lnnz,
                                                        const uint8_t* __restrict__ lkind, int32_t h0, int32_t h1,
                                                        SccState* ss, SolveState* st,
                                                        unsigned long long* dslot, GridBar gb) {
  __shared__ double sh[32];
  if (st->status != REACH_OK) return;
  const double eps = st->eps;
  const int64_t max_iter = st->max_iter;
  int64_t iters = st->iter;
  double bytes = ss->bytes, last = st->last;
  int32_t status = REACH_OK;
  int64_t tc = 0;    // cyclic sweeps so far: max|x' - x| of sweep tc goes to dslot[tc % 3]
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  RowGroups rg = RowGroups::make<G>();
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gth = (int64_t)gridDim.x * blockDim.x;
  for (int32_t h = h0; h < h1 && status == REACH_OK; ++h) {
    const int64_t r0 = lrow[h], nr = lrow[h + 1] - r0;
    const bool cyc = lkind[h] != 0;
    const bool natural = !CLUSTER && nr * 4 >= nq;
    const int64_t span = natural ? nq : nr;
    const double lbytes = (double)lnnz[h] * 12.0 + (double)nr * (cyc ? 48.0 : 44.0) + (natural ? 4.0 * nq : 4.0 * nr);
    int t = 0;
    for (;;) {
      const double* xi = (t & 1) ? xb : xa;
      double* xo = (t & 1) ? xa : xb;
      unsigned long long mx = 0ull;
      for (int64_t i = rg.first; warp_has_row<G>(i, span); i += rg.stride) {
        int32_t v = 0;
        bool on = false;
        if (i < span) {
          v = natural ? (int32_t)i : perm[r0 + i];
          on = !natural || rlev[v] == h;
        }
        double s0 = 0.0, s1 = 0.0;
        if (on) {
          const int64_t hi = arp[v + 1];
          int64_t k = arp[v] + rg.lane;
          for (; k + G < hi; k += 2 * G) {
            s0 = fma(aj[k], xi[acol[k]], s0);
            s1 = fma(aj[k + G], xi[acol[k + G]], s1);
          }
          if (k < hi) s0 = fma(aj[k], xi[acol[k]], s0);
        }
        const double sum = group_sum<G>(s0 + s1);
        if (on && rg.lane == 0) {
          const double xv = bj[v] + sum;
          if (cyc) {
            const double dv = fabs(xv - xi[v]);
            const unsigned long long bits =
                dv != dv ? 0x7ff0000000000000ull : (unsigned long long)__double_as_longlong(dv);
            mx = mx > bits ? mx : bits;
            xo[v] = xv;
          } else {
            xa[v] = xv;          // exact: every column is in a lower, finished level
            xb[v] = xv;
          }
        }
      }
      ++iters;
      bytes += lbytes;
      if (!cyc) {
        if (!sync_all<CLUSTER>(gb)) return;
        break;
      }
      // the grid maximum: one integer atomicMax per CTA on the bits of a non-negative
      // double; the slot two sweeps ahead is cleared (everyone read it a barrier ago)
      double a[1] = {__longlong_as_double((long long)mx)};
      block_reduce<1, true>(a, sh);
      if (threadIdx.x == 0) atomicMax(dslot + tc % 3, (unsigned long long)__double_as_longlong(a[0]));
      if (lead) dslot[(tc + 1) % 3] = 0ull;
      if (!sync_all<CLUSTER>(gb)) return;
      last = __longlong_as_double((long long)*(volatile unsigned long long*)(dslot + tc % 3));
      ++tc;
      ++t;
      if (last < eps) break;
      if (iters >= max_iter) {
        status = REACH_ENOTCONV;
        break;
      }
    }
    if (cyc) {
      // the last sweep wrote buffer (t & 1) ? xb : xa; make the other one agree on this level
      const double* src = (t & 1) ? xb : xa;
      double* dst = (t & 1) ? xa : xb;
      for (int64_t i = gtid; i < nr; i += gth) {
        const int32_t v = perm[r0 + i];
        dst[v] = src[v];
      }
      bytes += (double)nr * 20.0;
      if (!sync_all<CLUSTER>(gb)) return;
    }
  }
  if (lead) {
    st->iter = iters;
    st->last = last;
    st->status = status;
    ss->bytes = bytes;
  }
}

// ---------------------------------------------------------------- host side

template <typename T>
static cudaError_t zalloc(T** p, int64_t n, cudaStream_t s) {
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (size_t)(n > 0 ? n : 1));
  if (e == cudaSuccess) e = cudaMemsetAsync(*p, 0, sizeof(T) * (size_t)(n > 0 ? n : 1), s);
  return e;
}

void scc_free(reach_ctx* c) {
  SccPlan* sp = static_cast<SccPlan*>(c->scc);
  if (!sp) return;
  void* bufs[] = {sp->lab, sp->color, sp->indeg, sp->outdeg, sp->msize, sp->mstart, sp->mnnz, sp->mem,
                  sp->lvl, sp->lrows, sp->lrow, sp->lnnz, sp->lfill, sp->lbase, sp->lkind, sp->perm, sp->ss,
                  sp->rlev, sp->part, sp->bar, sp->pc};
  for (void* p : bufs)
    if (p) cudaFree(p);
  delete sp;
  c->scc = nullptr;
}

static int scc_group(reach_ctx* c) {
  const int g = pick_group(c->n_q, c->m_q);
  return g >= 16 ? 32 : g;
}

#define SCC_G_DISPATCH(g, CALL) \
  switch (g) {                  \
    case 2: CALL(2); break;     \
    case 4: CALL(4); break;     \
    case 8: CALL(8); break;     \
    default: CALL(32); break;   \
  }

static cudaError_t reset_state(reach_ctx* c, int64_t max_bodies) {
  SolveState hs;
  std::memset(&hs, 0, sizeof(hs));
  hs.eps = 0.0;
  hs.max_iter = 1;
  hs.status = REACH_ETIMEOUT;
  hs.max_bodies = max_bodies;
  cudaError_t e = cudaMemcpyAsync(c->st, &hs, sizeof(hs), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e;
}

// Adds the loop bodies the last graph-driven stage ran to the pass count.
static cudaError_t add_bodies(reach_ctx* c, SccPlan* sp) {
  int64_t bodies = 0, prev = 0;
  cudaError_t e = cudaMemcpy(&bodies, &c->st->bodies, sizeof(int64_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&prev, &sp->ss->passes, sizeof(int64_t), cudaMemcpyDeviceToHost);
  prev += bodies;
  if (e == cudaSuccess) e = cudaMemcpy(&sp->ss->passes, &prev, sizeof(int64_t), cudaMemcpyHostToDevice);
  return e;
}

static cudaError_t loop_status(reach_ctx* c, int32_t* status) {
  cudaError_t e = cudaMemcpyAsync(status, &c->st->status, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e;
}

// Cooperative launches (one resident grid, grid barriers) unless REACH_SCC_GRAPH=1 or the
// device cannot run them; then the conditional-while graphs.
static bool use_persistent(reach_ctx* c) {
  const char* gv = std::getenv("REACH_SCC_GRAPH");
  if (gv && gv[0] == '1') return false;
  int coop = 0;
  return cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device) == cudaSuccess && coop;
}

template <typename... A>
static cudaError_t coop_launch(reach_ctx* c, const void* fn, A... a) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, SCC_NT, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  const int grid = c->sm_count * std::min(per_sm, 2);
  void* args[] = {(void*)&a...};
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(SCC_NT), args, 0, c->stream);
}

// REACH_OK, or REACH_ETIMEOUT when a grid barrier gave up or the pass budget ran out.
static cudaError_t coop_status(reach_ctx* c, SccPlan* sp, int32_t* status) {
  unsigned w[2] = {0u, 0u};
  cudaError_t e = cudaMemcpyAsync(&w[0], sp->bar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&w[1], sp->pc + PC_FAIL, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  *status = (w[0] || w[1]) ? REACH_ETIMEOUT : REACH_OK;
  return e;
}

cudaError_t scc_decompose(reach_ctx* c, int32_t max_rounds, bool* loop_ok) {
  *loop_ok = true;
  SccPlan* sp = static_cast<SccPlan*>(c->scc);
  if (sp && sp->ready) return cudaSuccess;
  cudaStream_t s = c->stream;
  const int64_t nq = c->n_q;
  cudaError_t e = build_transposed_system(c);
  if (e != cudaSuccess) return e;
  if (!sp) {
    sp = new SccPlan();
    c->scc = sp;
    if ((e = zalloc(&sp->lab, nq, s)) != cudaSuccess) return e;
    if ((e = zalloc(&sp->color, nq, s)) != cudaSuccess) return e;
    if ((e = zalloc(&sp->indeg, nq, s)) != cudaSuccess) return e;
    if ((e = zalloc(&sp->outdeg, nq, s)) != cudaSuccess) return e;
    if ((e = zalloc(&sp->msize, nq, s)) != cudaSuccess) return e;
    if ((e = zalloc(&sp->mstart, nq + 1, s)) != cudaSuccess) return e;
    if ((e = zalloc(&sp->mnnz, nq, s)) != cudaSuccess) return e;
    if ((e = zalloc(&sp->mem, nq, s)) != cudaSuccess) return e;
    if ((e = zalloc(&sp->lvl, nq, s)) != cudaSuccess) return e;
    if ((e = zalloc(&sp->lrows, nq + 1, s)) != cudaSuccess) return e;
    if ((e = zalloc(&sp->lrow, nq + 2, s)) != cudaSuccess) return e;
    if ((e = zalloc(&sp->lnnz, nq + 1, s)) != cudaSuccess) return e;
    if ((e = zalloc(&sp->lfill, nq + 1, s)) != cudaSuccess) return e;
    if ((e = zalloc(&sp->lbase, nq, s)) != cudaSuccess) return e;
    if ((e = zalloc(&sp->lkind, nq + 1, s)) != cudaSuccess) return e;
    if ((e = zalloc(&sp->perm, nq, s)) != cudaSuccess) return e;
    if ((e = zalloc(&sp->rlev, nq, s)) != cudaSuccess) return e;
    if ((e = zalloc(&sp->part, 2 * 64 * (int64_t)c->sm_count, s)) != cudaSuccess) return e;
    if ((e = zalloc(&sp->bar, 4, s)) != cudaSuccess) return e;
    if ((e = zalloc(&sp->pc, 16, s)) != cudaSuccess) return e;
    if ((e = zalloc(&sp->ss, 1, s)) != cudaSuccess) return e;
  }
  if ((e = cudaEventRecord(c->ev0, s)) != cudaSuccess) return e;
  // accumulators of this run (a run cut short by the loop bound may have left counts)
  {
    const size_t n4 = sizeof(uint32_t) * (size_t)std::max<int64_t>(nq, 1);
    const size_t l4 = sizeof(uint32_t) * (size_t)(nq + 1), l8 = sizeof(int64_t) * (size_t)(nq + 1);
    cudaMemsetAsync(sp->msize, 0, n4, s);
    cudaMemsetAsync(sp->mnnz, 0, sizeof(int64_t) * (size_t)std::max<int64_t>(nq, 1), s);
    cudaMemsetAsync(sp->lrows, 0, l4, s);
    cudaMemsetAsync(sp->lfill, 0, l4, s);
    cudaMemsetAsync(sp->lnnz, 0, l8, s);
    cudaMemsetAsync(sp->lkind, 0, (size_t)(nq + 1), s);
  }
  SccState hs;
  std::memset(&hs, 0, sizeof(hs));
  hs.phase = PH_TRIM_INIT;
  hs.max_rounds = max_rounds;
  hs.exact = 1;
  hs.core_max = -1;
  if ((e = cudaMemcpyAsync(sp->ss, &hs, sizeof(hs), cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(c->ticket, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
  // every pass of the loop makes progress: trimming and searching passes remove rows,
  // and a propagation pass raises a colour; the bound only guards against faults
  const int64_t bound = 8 * nq + 64 * (int64_t)max_rounds + 64;
  if ((e = reset_state(c, bound)) != cudaSuccess) return e;
  const int g = scc_group(c);
  const int grid = c->sm_count * 8;
  int32_t* q0 = c->queue;
  int32_t* q1 = c->queue + c->n;
  const int64_t key_base = nq * 7919 + c->m_q;
  const bool persistent = use_persistent(c);
  bool acyclic = false;   // the sink-side trimming found every component and level
  int32_t status = 0;
  if (persistent) {
    cudaMemsetAsync(sp->pc, 0, 16 * sizeof(unsigned), s);
    cudaMemsetAsync(sp->bar, 0, 4 * sizeof(unsigned), s);
#define SCC_P(G) e = coop_launch(c, (const void*)k_scc_persist<G>, nq, c->a_rowptr, c->a_col, c->at_rowptr,    \
                                 c->at_col, sp->lab, sp->color, sp->indeg, sp->outdeg, sp->lvl, q0, q1,        \
                                 sp->pc, max_rounds, bound, sp->ss, GridBar{sp->bar, sp->bar + 1, sp->bar + 2})
    SCC_G_DISPATCH(g, SCC_P)
#undef SCC_P
    if (e != cudaSuccess) return e;
    if ((e = coop_status(c, sp, &status)) != cudaSuccess) return e;
    unsigned allsink = 0;
    if ((e = cudaMemcpy(&allsink, sp->pc + PC_ALLSINK, sizeof(unsigned), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return e;
    acyclic = allsink != 0;
  } else {
#define SCC_STEP(G)                                                                                      \
  k_scc_step<G><<<grid, SCC_NT, 0, cs>>>(nq, c->a_rowptr, c->a_col, c->at_rowptr, c->at_col, sp->lab,   \
                                        sp->color, sp->indeg, sp->outdeg, q0, q1, sp->ss, c->st, c->ticket)
    e = run_loop(c, c->g_exec[5], c->g_key[5], key_base, [&](cudaStream_t cs, cudaGraphConditionalHandle, int) {
      SCC_G_DISPATCH(g, SCC_STEP)
    });
#undef SCC_STEP
    if (e != cudaSuccess) return e;
    if ((e = loop_status(c, &status)) != cudaSuccess) return e;
    if ((e = add_bodies(c, sp)) != cudaSuccess) return e;
  }
  if (status != REACH_OK) {
    *loop_ok = false;
    return cudaSuccess;
  }
  // labels -> sizes, member lists
  uint32_t* out_edges = sp->indeg;
  uint32_t* fill = sp->outdeg;
  cudaMemsetAsync(out_edges, 0, sizeof(uint32_t) * (size_t)std::max<int64_t>(nq, 1), s);
  cudaMemsetAsync(fill, 0, sizeof(uint32_t) * (size_t)std::max<int64_t>(nq, 1), s);
#define LAB_STATS(G)                                                                                          \
  k_lab_stats<G><<<grid_for(c, (const void*)k_lab_stats<G>, SCC_NT, nq * G), SCC_NT, 0, s>>>(              \
      nq, c->a_rowptr, c->a_col, sp->lab, sp->msize, sp->mnnz, out_edges)
  SCC_G_DISPATCH(g, LAB_STATS)
#undef LAB_STATS
  if ((e = exclusive_scan_u32(c, sp->msize, sp->mstart, nq)) != cudaSuccess) return e;
  k_members<<<grid_for(c, (const void*)k_members, SCC_NT, nq), SCC_NT, 0, s>>>(nq, sp->lab, sp->mstart, fill,
                                                                                sp->mem);
  // levels
  if (persistent && !acyclic) {
    cudaMemsetAsync(sp->pc, 0, 16 * sizeof(unsigned), s);
    cudaMemsetAsync(sp->bar, 0, 4 * sizeof(unsigned), s);
#define LVL_P(G) e = coop_launch(c, (const void*)k_lvl_persist<G>, nq, c->at_rowptr, c->at_col, sp->lab,     \
                                 sp->msize, sp->mstart, sp->mem, out_edges, sp->lvl, q0, q1, sp->pc, sp->ss,  \
                                 GridBar{sp->bar, sp->bar + 1, sp->bar + 2})
    SCC_G_DISPATCH(g, LVL_P)
#undef LVL_P
    if (e != cudaSuccess) return e;
    if ((e = coop_status(c, sp, &status)) != cudaSuccess) return e;
    if (status != REACH_OK) {
      *loop_ok = false;
      return cudaSuccess;
    }
  }
  if (!persistent) {
    if ((e = reset_state(c, 2 * nq + 8)) != cudaSuccess) return e;
    // the colouring left ss->phase at PH_LV_INIT with empty frontiers
    int32_t ph = PH_LV_INIT;
    cudaMemcpyAsync(&sp->ss->phase, &ph, sizeof(ph), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(sp->ss->count, 0, sizeof(hs.count), s);
    cudaMemsetAsync(&sp->ss->cur, 0, sizeof(int32_t), s);
#define LVL_STEP(G)                                                                                       \
  k_lvl_step<G><<<grid, SCC_NT, 0, cs>>>(nq, c->at_rowptr, c->at_col, sp->lab, sp->msize, sp->mstart,    \
                                        sp->mem, out_edges, sp->lvl, q0, q1, sp->ss, c->st, c->ticket)
    e = run_loop(c, c->g_exec[6], c->g_key[6], key_base + 1, [&](cudaStream_t cs, cudaGraphConditionalHandle, int) {
      SCC_G_DISPATCH(g, LVL_STEP)
    });
#undef LVL_STEP
    if (e != cudaSuccess) return e;
    if ((e = loop_status(c, &status)) != cudaSuccess) return e;
    if ((e = add_bodies(c, sp)) != cudaSuccess) return e;
    if (status != REACH_OK) {
      *loop_ok = false;
      return cudaSuccess;
    }
  }
  // order rows by level
  k_level_sizes<<<grid_for(c, (const void*)k_level_sizes, SCC_NT, nq), SCC_NT, 0, s>>>(
      nq, sp->lab, sp->msize, sp->mnnz, sp->lvl, sp->lrows, sp->lnnz, sp->lfill, sp->lbase, sp->lkind);
  if ((e = exclusive_scan_u32(c, sp->lrows, sp->lrow, nq + 1)) != cudaSuccess) return e;
  k_perm<<<grid_for(c, (const void*)k_perm, SCC_NT, nq), SCC_NT, 0, s>>>(nq, sp->mem, sp->lab, sp->mstart,
                                                                          sp->lvl, sp->lrow, sp->lbase, sp->perm);
  k_level_of_row<<<grid_for(c, (const void*)k_level_of_row, SCC_NT, nq), SCC_NT, 0, s>>>(nq, sp->lab, sp->lvl,
                                                                                        sp->rlev);
  if ((e = cudaEventRecord(c->ev1, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(&hs, sp->ss, sizeof(hs), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  sp->h_lrow.assign((size_t)hs.n_levels + 1, 0);
  sp->h_lnnz.assign((size_t)hs.n_levels + 1, 0);
  if (hs.n_levels > 0) {
    e = cudaMemcpy(sp->h_lrow.data(), sp->lrow, sizeof(int64_t) * (size_t)(hs.n_levels + 1), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaMemcpy(sp->h_lnnz.data(), sp->lnnz, sizeof(int64_t) * (size_t)hs.n_levels, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
  }
  sp->info.n_q = nq;
  sp->info.n_scc = hs.n_scc;
  sp->info.n_levels = hs.n_levels;
  sp->info.n_trivial = hs.n_trivial;
  sp->info.largest = hs.largest;
  sp->info.exact = hs.exact;
  sp->info.rounds = hs.round;
  sp->info.passes = hs.passes;
  sp->info.ms = ms;
  sp->ready = true;
  return cudaGetLastError();
}

cudaError_t scc_outputs(reach_ctx* c, int32_t* label, int32_t* level, cudaMemcpyKind kind, reach_scc_info* info) {
  SccPlan* sp = static_cast<SccPlan*>(c->scc);
  cudaStream_t s = c->stream;
  const int64_t nq = c->n_q;
  cudaError_t e = cudaSuccess;
  if (info) *info = sp->info;
  if (label && nq > 0) e = cudaMemcpyAsync(label, sp->lab, sizeof(int32_t) * (size_t)nq, kind, s);
  if (e == cudaSuccess && level && nq > 0)
    e = cudaMemcpyAsync(level, sp->rlev, sizeof(int32_t) * (size_t)nq, kind, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

template <int G>
static cudaError_t launch_grid_run(reach_ctx* c, SccPlan* sp, int32_t h0, int32_t h1) {
  const void* fn = (const void*)k_blk_persist<G, false>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, SCC_NT, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  const int grid = c->sm_count * std::min(per_sm, 4);
  int64_t nq = c->n_q;
  GridBar gb{sp->bar, sp->bar + 1, sp->bar + 2};
  unsigned long long* dslot = reinterpret_cast<unsigned long long*>(sp->part);
  void* args[] = {&nq, &c->a_rowptr, &c->a_col, &c->a_jv, &c->bj, &c->x, &c->x2, &sp->perm, &sp->rlev,
                  &sp->lrow, &sp->lnnz, &sp->lkind, &h0, &h1, &sp->ss, &c->st, &dslot, &gb};
  cudaMemsetAsync(sp->part, 0, 3 * sizeof(unsigned long long), c->stream);
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(SCC_NT), args, 0, c->stream);
}

// Cluster size the device can host for the small-level kernel (16, else 8, else 0).
template <int G>
static int cluster_size(reach_ctx* c) {
  const void* fn = (const void*)k_blk_persist<G, true>;
  for (int cs : {CL_SIZE, 8}) {
    if (cs > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(CL_NT);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) == cudaSuccess && n > 0) return cs;
    cudaGetLastError();
  }
  return 0;
}

template <int G>
static cudaError_t launch_cluster_run(reach_ctx* c, SccPlan* sp, int cs, int32_t h0, int32_t h1) {
  const void* fn = (const void*)k_blk_persist<G, true>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(CL_NT);
  cfg.stream = c->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int64_t nq = c->n_q;
  GridBar gb{sp->bar, sp->bar + 1, sp->bar + 2};
  unsigned long long* dslot = reinterpret_cast<unsigned long long*>(sp->part);
  void* args[] = {&nq, &c->a_rowptr, &c->a_col, &c->a_jv, &c->bj, &c->x, &c->x2, &sp->perm, &sp->rlev,
                  &sp->lrow, &sp->lnnz, &sp->lkind, &h0, &h1, &sp->ss, &c->st, &dslot, &gb};
  cudaMemsetAsync(sp->part, 0, 3 * sizeof(unsigned long long), c->stream);
  return cudaLaunchKernelExC(&cfg, fn, args);
}

// Bytes one sweep of a level moves below which the level runs on a single cluster.
// Measured per sweep: a cluster of 16 CTAs costs about 1.3 us + rows / 1100 per us (its
// 16 SMs are latency-bound on the dependent loads of a row), the cooperative grid about
// 5 us + rows / 9000 per us (the grid barrier dominates); they cross near 4,600 rows,
// about 0.35 MB of a sparse level.
constexpr double SMALL_LEVEL_BYTES = 0.35e6;

// The level-by-level solve as a few persistent launches: maximal runs of small levels on
// one cluster, runs of big levels on the whole grid.  Returns ran = false (nothing
// launched) when the device cannot run cooperative launches.
static cudaError_t solve_scc_persistent(reach_ctx* c, SccPlan* sp, bool* ran) {
  *ran = false;
  int coop = 0;
  cudaError_t e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device);
  if (e != cudaSuccess || !coop) return e;
  cudaStream_t s = c->stream;
  const int64_t nq = c->n_q;
  const int g = scc_group(c);
  int cs = 0;
#define CSIZE(G) cs = cluster_size<G>(c)
  SCC_G_DISPATCH(g, CSIZE)
#undef CSIZE
  const char* cv = std::getenv("REACH_SCC_CLUSTER");
  if (cv && cv[0] == '0') cs = 0;
  // x2 starts as a copy of x: a level's first sweep may read lower rows from either
  cudaMemcpyAsync(c->x2, c->x, sizeof(double) * nq, cudaMemcpyDeviceToDevice, s);
  cudaMemsetAsync(sp->bar, 0, 4 * sizeof(unsigned), s);
  {
    int32_t ok = REACH_OK;
    double zero = 0.0;
    cudaMemcpyAsync(&c->st->status, &ok, sizeof(ok), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(&sp->ss->bytes, &zero, sizeof(zero), cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
  }
  const int32_t nl = (int32_t)sp->info.n_levels;
  auto small = [&](int32_t h) {
    const double b = (double)sp->h_lnnz[h] * 12.0 + (double)(sp->h_lrow[h + 1] - sp->h_lrow[h]) * 48.0;
    return cs > 0 && b <= SMALL_LEVEL_BYTES;
  };
  for (int32_t h0 = 0; h0 < nl && e == cudaSuccess;) {
    const bool sm = small(h0);
    int32_t h1 = h0 + 1;
    while (h1 < nl && small(h1) == sm) ++h1;
#define RUN_C(G) e = launch_cluster_run<G>(c, sp, cs, h0, h1)
#define RUN_G(G) e = launch_grid_run<G>(c, sp, h0, h1)
    if (sm) {
      SCC_G_DISPATCH(g, RUN_C)
    } else {
      SCC_G_DISPATCH(g, RUN_G)
    }
#undef RUN_C
#undef RUN_G
    h0 = h1;
  }
  if (e != cudaSuccess) return e;
  unsigned err = 0;
  e = cudaMemcpyAsync(&err, sp->bar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  SolveState hs;
  e = cudaMemcpy(&hs, c->st, sizeof(hs), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  if (err) hs.status = REACH_ETIMEOUT;   // a grid barrier gave up
  hs.done = 1;
  e = cudaMemcpy(c->st, &hs, sizeof(hs), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  *ran = true;
  return cudaSuccess;
}

cudaError_t solve_scc_jacobi(reach_ctx* c, const double* x0q, double* bytes_out) {
  cudaStream_t s = c->stream;
  const int64_t nq = c->n_q;
  SccPlan* sp = static_cast<SccPlan*>(c->scc);
  if (x0q) cudaMemcpyAsync(c->x, x0q, sizeof(double) * nq, cudaMemcpyDeviceToDevice, s);
  else cudaMemsetAsync(c->x, 0, sizeof(double) * nq, s);
  const char* gv = std::getenv("REACH_SCC_GRAPH");
  if (!(gv && gv[0] == '1')) {
    bool ran = false;
    cudaError_t pe = solve_scc_persistent(c, sp, &ran);
    if (pe != cudaSuccess) return pe;
    if (ran) {
      if (bytes_out) {
        pe = cudaMemcpyAsync(bytes_out, &sp->ss->bytes, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (pe == cudaSuccess) pe = cudaStreamSynchronize(s);
        if (pe != cudaSuccess) return pe;
      }
      return residual_report(c, c->x);
    }
  }
  {
    int32_t zero[2] = {0, 0};
    cudaMemcpyAsync(&sp->ss->blk_level, zero, sizeof(zero), cudaMemcpyHostToDevice, s);
    int64_t z64 = 0;
    cudaMemcpyAsync(&sp->ss->blk_sweeps, &z64, sizeof(z64), cudaMemcpyHostToDevice, s);
    double zd = 0.0;
    cudaMemcpyAsync(&sp->ss->bytes, &zd, sizeof(zd), cudaMemcpyHostToDevice, s);
  }
  cudaMemsetAsync(&c->st->slot[0], 0, sizeof(unsigned long long), s);
  cudaMemsetAsync(c->ticket, 0, sizeof(unsigned), s);
  const int g = scc_group(c);
  const int grid = c->sm_count * 8;
  const int64_t key = nq * 7919 + c->m_q + 2;
#define BLK(G)                                                                                              \
  k_blk_sweep<G><<<grid, SCC_NT, 0, cs>>>(c->a_rowptr, c->a_col, c->a_jv, c->bj, c->x, c->x2, sp->perm,        \
                                         sp->lrow, sp->lkind, sp->ss, c->st, &c->st->slot[0])
  cudaError_t e = run_loop(c, c->g_exec[7], c->g_key[7], key, [&](cudaStream_t cs, cudaGraphConditionalHandle, int) {
    SCC_G_DISPATCH(g, BLK)
    k_blk_apply<<<grid, SCC_NT, 0, cs>>>(c->x, c->x2, sp->perm, sp->lrow, sp->lnnz, sp->lkind, sp->ss, c->st,
                                         &c->st->slot[0], c->ticket);
  });
#undef BLK
  if (e != cudaSuccess) return e;
  if (bytes_out) {
    e = cudaMemcpyAsync(bytes_out, &sp->ss->bytes, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
  }
  return residual_report(c, c->x);
}

bool scc_ready(const reach_ctx* c) {
  const SccPlan* sp = static_cast<const SccPlan*>(c->scc);
  return sp && sp->ready;
}

int64_t scc_levels(const reach_ctx* c) {
  const SccPlan* sp = static_cast<const SccPlan*>(c->scc);
  return sp ? sp->info.n_levels : 0;
}

}  // namespace reach
