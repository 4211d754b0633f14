// Host-side declarations shared by the library's translation units: the
// context layout, the device-state blocks read by the solver graphs, and the
// kernel launchers.  Not part of the public ABI (include/reach.h is).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <functional>
#include <string>

#include "../../include/reach.h"

namespace reach {

enum : uint8_t { CLS_S0 = 0, CLS_S1 = 1, CLS_SQ = 2 };

// Validation error bits written by k_validate.
enum : unsigned { VERR_ROWPTR = 1u, VERR_COL = 2u, VERR_VAL = 4u, VERR_ROWSUM = 8u };

// Per-solve state in device memory.  Kernels of a captured solve graph read the
// stopping parameters from here and write the outcome, so one instantiated graph
// serves every later solve of the same shape.
struct SolveState {
  double eps;
  int64_t max_iter;
  int64_t iter;
  double last;          // stopping quantity of the last check
  double resid;         // FP64 max|b - (I - A) x| after the loop
  double resid_ub;      // certified upper bound of the exact max|b - (I - A) x| (rounding included)
  int32_t status;       // reach_status
  int32_t done;         // set once the stopping rule held or max_iter ran out
  int32_t refinements;
  int32_t pad;
  int64_t bodies;       // loop bodies run (hard stop at max_bodies)
  int64_t max_bodies;
  unsigned long long slot[64];  // per-sweep max|dx| bit patterns (non-negative doubles)
  unsigned rowctr[64];          // per-launch row counters of warp-per-row kernels (dynamic rows)
};

// BiCGStab scalars (§3.2 names: y = rho, a = alpha, w = omega) in device memory.
struct BiState {
  double y, yprev, a, w, beta, qv, ts, tt, snorm, rnorm, rr;
  int32_t s_done;       // max|s| < eps after the a-step: finish with x += a p
  int32_t restarted;    // a breakdown restart has happened (only one is allowed)
  int32_t restart;      // next p-update restarts: q = r, p = r, v = 0
  int32_t skip;         // rest of this iteration is skipped (breakdown at q.v)
};

// Level-synchronous backward search: level L reads the frontier of count[L % 3] entries,
// pushes into count[(L + 1) % 3] and may clear count[(L + 2) % 3] (the frontier of level
// L - 1, read by everyone before the barrier that ended level L - 1), so a level needs
// one barrier.
// Slot of reach_ctx::keys that the extraction reduces Varah's margin into.
constexpr int VARAH_KEY = 2;

struct BfsState {
  int32_t level;
  uint32_t count[3];
};

struct Tuning {
  int g = 0;            // lanes per row for CSR kernels (0 = pick from mean degree; 64 = warp + vector
                        // loads; 80 = FP32 sweep staged by bulk copies; 128 = entry-balanced tiles)
  int gm[3] = {0, 0, 0};  // autotuned lanes-per-row code per method (0 = none)
  int k = 16;           // sweeps between convergence checks / refinement period
  int k_auto = 0;       // autotuned sweeps between checks for FP64 Jacobi (0 = none)
  int sweep_u = 2;      // quads per lane per trip of the vector FP32 sweep (2, or 4 for layout code 66)
  int cta = 256;        // threads per CTA
};

struct DeviceBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace reach

struct reach_ctx {
  int device = 0;
  int sm_count = 0;
  cudaStream_t stream = nullptr;       // user stream (may be the legacy default)
  cudaStream_t cap = nullptr;          // private stream used for graph capture
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::string err;

  int64_t n = 0, m = 0;
  int64_t* rowptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
  uint8_t* goal = nullptr;

  // reversed underlying digraph (pattern of P^T, entries with P > 0)
  int64_t* t_rowptr = nullptr;
  int32_t* t_col = nullptr;

  // general system M x = b (no partition): A = -(off-diagonal of M), d = diag(M)
  bool general = false;

  // partition
  bool have_classes = false;
  int mode = 0;
  uint8_t* cls = nullptr;
  int64_t* qidx = nullptr;     // state -> S? row (valid on S?)
  int64_t* qstate = nullptr;   // S? row -> state
  uint32_t* vis = nullptr;     // BFS visited bitmask
  int32_t* queue = nullptr;    // two BFS queues of n entries
  reach::BfsState* bfs = nullptr;

  // system over S? (§2.3): A off-diagonal CSR, d = 1 - A_ii, b
  int64_t n_q = 0, m_q = 0;
  int64_t* a_rowptr = nullptr;
  int32_t* a_col = nullptr;
  double* a_val = nullptr;
  float* a_hi = nullptr;
  float* a_lo = nullptr;
  uint16_t* a_col16 = nullptr;  // a_col narrowed to 16 bits when n? <= 65536 (mixed sweeps)
  double* d = nullptr;
  double* b = nullptr;
  // the Jacobi form of the system: x' = bj + Aj x with Aj_ij = A_ij / d_i, bj_i = b_i / d_i
  // (one correctly rounded division per entry, once per system, instead of a division
  // per row in every sweep: FP64 division is a long sequence on the narrow FP64 pipe)
  double* a_jv = nullptr;
  double* bj = nullptr;

  // transposed system for the adjoint
  int64_t* at_rowptr = nullptr;
  int32_t* at_col = nullptr;
  double* at_val = nullptr;
  double* at_jv = nullptr;     // its Jacobi form: A_ij / d_j in row j of the transpose
  double* at_b = nullptr;      // right-hand side of an adjoint BiCGStab solve (e_init)

  // solve workspace (n_q each)
  double* x = nullptr;
  double* x2 = nullptr;
  double* vr = nullptr;     // BiCGStab r
  double* vq = nullptr;     // BiCGStab q
  double* vp = nullptr;     // BiCGStab p
  double* vv = nullptr;     // BiCGStab v
  double* vs = nullptr;     // BiCGStab s
  double* vt = nullptr;     // BiCGStab t
  float* r32 = nullptr;     // mixed: residual
  float* xf = nullptr;      // mixed: FP32 copy of x (lo-part products of the residual)
  float* dl[2] = {nullptr, nullptr};  // mixed: correction ping-pong
  double* xfull = nullptr;  // full-state x of the last successful solve
  bool have_x = false;

  reach::SolveState* st = nullptr;
  reach::BiState* bi = nullptr;
  double* part = nullptr;   // per-CTA partials (8 * max grid)
  unsigned* ticket = nullptr;
  unsigned* verr = nullptr;
  int64_t* vrow = nullptr;
  unsigned long long* maxrow = nullptr;  // longest row of P (device, written by validation)
  int64_t max_row = 0;                   // its host copy

  // norm bounds of (I - A)^-1 for the certified error bound of every solve: Varah's
  // (from the row-dominance margin, at precompute), the one from an approximate
  // tau = (I - A)^-1 1 (reach_norm_bound), and Varah's over the transpose (adjoint)
  double kinv_varah = INFINITY;
  double kinv_tau = INFINITY;
  double kinv_varah_t = -1.0;           // < 0: not computed yet
  unsigned long long* keys = nullptr;   // ordered-key reduction words (VARAH_KEY: the extraction's)
  bool varah_key = false;               // keys[VARAH_KEY] holds the margin of the current system
  double* tau_save = nullptr;           // b and bj while the tau system is solved (2 n?)

  reach::Tuning tune;
  bool device_loops = true;   // conditional-while graphs (false: host-driven loops)
  bool rev_ready = false;     // t_rowptr / t_col hold the reversed graph of the current P
  double ms_precompute = 0.0;

  // cached solve graphs, keyed by method and shape
  // 0-3 solvers, 4 entry-balanced Jacobi, 5-6 SCC decomposition, 7 level-by-level Jacobi
  cudaGraphExec_t g_exec[10] = {nullptr, nullptr, nullptr, nullptr, nullptr,
                                 nullptr, nullptr, nullptr, nullptr, nullptr};
  int64_t g_key[10] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1};

  // rows and entries of the fullest CTA when the system is split over 1, 2, 4, 8, 16 CTAs
  // (small.cu; -1 = not measured yet)
  int64_t small_ext[5][2] = {{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}};
  void* seg = nullptr;      // tile plan of the entry-balanced Jacobi sweep (segscan.cu)
  void* scc = nullptr;      // components, levels and row order (scc.cu)
};

namespace reach {

// ---- graph.cu
cudaError_t launch_validate(reach_ctx* c);
cudaError_t check_diagonal(reach_ctx* c);
cudaError_t build_reverse_pattern(reach_ctx* c);
cudaError_t bfs_backward(reach_ctx* c, int source_kind, bool avoid_goal);
cudaError_t classify_and_extract(reach_ctx* c, int mode);
cudaError_t extract_rows(reach_ctx* c);
cudaError_t extract_all_rows(reach_ctx* c);
cudaError_t split_hilo(reach_ctx* c);
cudaError_t build_jacobi_form(reach_ctx* c);
cudaError_t build_transposed_system(reach_ctx* c);

// ---- solve.cu
cudaError_t solve_jacobi64(reach_ctx* c, const double* x0q, bool transposed);
cudaError_t solve_mixed(reach_ctx* c, const double* x0q);
cudaError_t solve_bicgstab(reach_ctx* c, const double* x0q);
cudaError_t solve_bicgstab_transposed(reach_ctx* c);
cudaError_t residual_inf(reach_ctx* c, const double* xq, double* out_host);
cudaError_t scatter_full(reach_ctx* c, const double* xq, double* full);
cudaError_t gather_q(reach_ctx* c, const double* full, double* xq);
cudaError_t grad_entries(reach_ctx* c, const double* yq, double* grad);
// Runs body inside a cached conditional-while graph (or host loop) until SolveState::done.
cudaError_t run_loop(reach_ctx* c, cudaGraphExec_t& exec, int64_t& exec_key, int64_t key,
                     const std::function<void(cudaStream_t, cudaGraphConditionalHandle, int)>& body);
void launch_check_mixed(cudaStream_t s, SolveState* st, int slot, int k);
cudaError_t autotune(reach_ctx* c, int method, int* chosen, float* best_ms);
cudaError_t time_kernel(reach_ctx* c, int kernel, int launches, float* avg_ms);
void launch_finalize_resid(cudaStream_t s, SolveState* st);

// ---- small.cu
bool small_system(reach_ctx* c, int method);
cudaError_t solve_small(reach_ctx* c, int method, int k);
// ---- segscan.cu
cudaError_t solve_jacobi_seg(reach_ctx* c, const double* x0q);
cudaError_t seg_plan(reach_ctx* c);
void seg_sweep(reach_ctx* c, const double* x, double* xn, unsigned long long* slot, cudaStream_t s);
void seg_sweep32(reach_ctx* c, const float* din, float* dout, cudaStream_t s);
void seg_spmv64(reach_ctx* c, const double* u, double* y, cudaStream_t s);
void seg_resid_hilo(reach_ctx* c, unsigned long long* slot, cudaStream_t s);
void seg_free(reach_ctx* c);
// ---- tma.cu
cudaError_t sweep32_tma(reach_ctx* c, const float* din, float* dout, cudaStream_t s, unsigned* ctr);
// ---- scc.cu
cudaError_t scc_decompose(reach_ctx* c, int32_t max_rounds, bool* loop_ok);
cudaError_t scc_outputs(reach_ctx* c, int32_t* label, int32_t* level, cudaMemcpyKind kind, reach_scc_info* info);
cudaError_t solve_scc_jacobi(reach_ctx* c, const double* x0q, double* bytes_out);
bool scc_ready(const reach_ctx* c);
void scc_free(reach_ctx* c);
// ---- more of graph.cu / solve.cu used by segscan.cu and scc.cu
cudaError_t exclusive_scan_u8(reach_ctx* c, const uint8_t* in, int64_t* out, int64_t n, int64_t* total_dev);
cudaError_t exclusive_scan_u32(reach_ctx* c, const uint32_t* in, int64_t* out, int64_t n);
cudaError_t residual_report(reach_ctx* c, const double* xq);
cudaError_t varah_norm_bound(reach_ctx* c, bool transposed, double* kinv);
cudaError_t tau_rhs_begin(reach_ctx* c);
cudaError_t tau_rhs_end(reach_ctx* c);
cudaError_t tau_norm_bound(reach_ctx* c, const double* tau, double* kinv);

// ---- shared host helpers (api.cu)
int pick_group(int64_t rows, int64_t nnz);
int grid_for(reach_ctx* c, const void* kernel, int threads, int64_t work_items);
int grid_rows(reach_ctx* c, const void* kernel, int threads, int g, int64_t rows, bool dynamic = false);
bool set_err(reach_ctx* c, const std::string& msg);

}  // namespace reach
