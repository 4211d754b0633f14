// The C ABI of include/reach.h: context lifetime, argument checks, and the
// orchestration of the precompute (§2.2-§2.3) and the solvers (§3).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>

#include "internal.h"

namespace reach {

static thread_local std::string g_tls_err;

bool set_err(reach_ctx* c, const std::string& msg) {
  if (c) c->err = msg;
  else g_tls_err = msg;
  return false;
}

int pick_group(int64_t rows, int64_t nnz) {
  const double mean = rows > 0 ? (double)nnz / (double)rows : 0.0;
  if (mean <= 2.5) return 2;
  if (mean <= 5.0) return 4;
  if (mean <= 10.0) return 8;
  if (mean <= 20.0) return 16;
  return 32;
}

constexpr int MAX_GRID = 4096;

int grid_for(reach_ctx* c, const void* kernel, int threads, int64_t work) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> occ;
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = occ.find(kernel);
    if (it == occ.end()) {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess)
        per_sm = 1;
      occ[kernel] = per_sm;
    } else {
      per_sm = it->second;
    }
  }
  per_sm = std::max(per_sm, 1);
  int64_t full = (int64_t)c->sm_count * per_sm;
  int64_t need = std::max<int64_t>(1, (work + threads - 1) / threads);
  return (int)std::min<int64_t>(std::min<int64_t>(full, need), MAX_GRID);
}

// Grid for a kernel in which G lanes own one row and rows are dealt round-robin.
// With R resident row-groups at most, every group gets ceil(rows / R) rows; the grid is
// then shrunk so that all groups get that many (the last few one fewer), so a sweep
// over rows of similar length ends with every warp busy until the end.
int grid_rows(reach_ctx* c, const void* kernel, int threads, int g, int64_t rows, bool dynamic) {
  const int full = grid_for(c, kernel, threads, INT64_MAX / 2);
  // dynamic rows: every resident CTA, capped at one warp per row
  if (dynamic) return (int)std::max<int64_t>(1, std::min<int64_t>(full, (rows + threads / 32 - 1) / (threads / 32)));
  const int64_t groups_per_cta = threads / g;
  const int64_t max_groups = (int64_t)full * groups_per_cta;
  if (rows <= 0) return 1;
  const int64_t per = (rows + max_groups - 1) / max_groups;
  const int64_t groups = (rows + per - 1) / per;
  return (int)std::max<int64_t>(1, (groups + groups_per_cta - 1) / groups_per_cta);
}

}  // namespace reach

using namespace reach;

namespace {

const char* cuda_msg(cudaError_t e) { return cudaGetErrorString(e); }

reach_status fail(reach_ctx* c, reach_status s, const std::string& msg) {
  set_err(c, msg);
  return s;
}

reach_status cuda_fail(reach_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cuda_msg(e);
  set_err(c, m);
  return e == cudaErrorMemoryAllocation ? REACH_ENOMEM : REACH_ECUDA;
}

bool inject_enomem() {
  const char* v = std::getenv("REACH_FAULT_ENOMEM");
  return v && v[0] == '1';
}

template <typename T>
cudaError_t dalloc(T** p, int64_t count) {
  *p = nullptr;
  if (inject_enomem()) return cudaErrorMemoryAllocation;
  if (count <= 0) count = 1;
  return cudaMalloc((void**)p, sizeof(T) * (size_t)count);
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void free_system(reach_ctx* c) {
  dfree(c->a_rowptr); dfree(c->a_col); dfree(c->a_val); dfree(c->a_hi); dfree(c->a_lo); dfree(c->a_col16);
  dfree(c->d); dfree(c->b); dfree(c->a_jv); dfree(c->bj); dfree(c->qstate);
  dfree(c->at_rowptr); dfree(c->at_col); dfree(c->at_val); dfree(c->at_jv); dfree(c->at_b);
  dfree(c->x); dfree(c->x2); dfree(c->vr); dfree(c->vq); dfree(c->vp); dfree(c->vv);
  dfree(c->vs); dfree(c->vt); dfree(c->r32); dfree(c->xf); dfree(c->dl[0]); dfree(c->dl[1]);
  dfree(c->tau_save);
  for (auto& e : c->small_ext) e[0] = e[1] = -1;
  c->varah_key = false;
  c->kinv_varah = INFINITY;
  c->kinv_tau = INFINITY;
  c->kinv_varah_t = -1.0;
  seg_free(c);
  scc_free(c);
}

void drop_graphs(reach_ctx* c) {
  for (int i = 0; i < 10; ++i) {
    if (c->g_exec[i]) cudaGraphExecDestroy(c->g_exec[i]);
    c->g_exec[i] = nullptr;
    c->g_key[i] = -1;
  }
}

cudaMemcpyKind kind_to_dev(int32_t flags) {
  return flags == REACH_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
cudaMemcpyKind kind_from_dev(int32_t flags) {
  return flags == REACH_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

// Certified max-norm error: ||M^-1|| (kinv, an upper bound) times the upper bound of the
// exact residual norm, the product rounded up; 0 for an empty system, +inf without a bound.
double error_bound(int64_t n_q, double kinv, double resid_ub) {
  if (n_q == 0) return 0.0;
  if (!(kinv < INFINITY) || !(resid_ub < INFINITY)) return INFINITY;
  return std::nextafter(kinv * resid_ub, INFINITY);
}

}  // namespace

extern "C" {

const char* reach_version(void) { return "reach-gb300 0.1 (sm_103a)"; }

const char* reach_last_error(const reach_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_tls_err.c_str();
}

void reach_destroy(reach_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  drop_graphs(c);
  free_system(c);
  dfree(c->rowptr); dfree(c->col); dfree(c->val); dfree(c->goal);
  dfree(c->t_rowptr); dfree(c->t_col);
  dfree(c->cls); dfree(c->qidx); dfree(c->vis); dfree(c->queue); dfree(c->bfs);
  dfree(c->xfull); dfree(c->st); dfree(c->bi); dfree(c->part); dfree(c->ticket);
  dfree(c->verr); dfree(c->vrow); dfree(c->maxrow); dfree(c->keys);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->cap) cudaStreamDestroy(c->cap);
  delete c;
}

// Copies and validates P (a chain, or a general system when `general`).
static reach_status create_common(reach_ctx** out, int64_t n, int64_t m, const int64_t* rowptr,
                                  const int32_t* col, const double* val, const uint8_t* goal,
                                  int32_t flags, void* stream, bool general, const char* who) {
  const std::string w(who);
  if (!out) return fail(nullptr, REACH_EINVAL, w + ": out is NULL");
  if (n < 1 || n > INT32_MAX - 1) return fail(nullptr, REACH_EINVAL, w + ": n must be in [1, 2^31-2]");
  if (m < 0) return fail(nullptr, REACH_EINVAL, w + ": m < 0");
  if (!rowptr || (!general && !goal) || (m > 0 && (!col || !val)))
    return fail(nullptr, REACH_EINVAL, w + ": NULL input pointer");
  if (flags != REACH_HOST && flags != REACH_DEVICE)
    return fail(nullptr, REACH_EINVAL, w + ": flags must be REACH_HOST or REACH_DEVICE");

  reach_ctx* c = new reach_ctx();
  c->stream = (cudaStream_t)stream;
  c->n = n;
  c->m = m;
  c->general = general;
  const char* hl = std::getenv("REACH_HOST_LOOPS");
  c->device_loops = !(hl && hl[0] == '1');
  // REACH_LANES fixes the row mapping of every solver kernel that has none autotuned:
  // 1, 2, 4, 8, 16 or 32 lanes per row, 48 = half a warp with vector loads, 64 = a warp with
  // vector loads, 72 = the FP32 sweep with its vector in shared memory and 80 = the FP32 sweep
  // with rows staged by bulk copies (other kernels as 64), 128 = entry-balanced tiles
  if (const char* ln = std::getenv("REACH_LANES")) {
    const int v = std::atoi(ln);
    if (v == 1 || v == 2 || v == 4 || v == 8 || v == 16 || v == 32 || v == 48 || v == 64 || v == 72 || v == 80 ||
        v == 128)
      c->tune.g = v;
  }
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
  if (e != cudaSuccess) {
    reach_status s = cuda_fail(nullptr, e, (w + ": device setup").c_str());
    reach_destroy(c);
    return s;
  }
  const int64_t words = (n + 31) >> 5;
  const int64_t part_n = std::max<int64_t>(16 * 4096, n / 8192 + 64);
  if ((e = dalloc(&c->rowptr, n + 1)) != cudaSuccess || (e = dalloc(&c->col, m + 8)) != cudaSuccess ||
      (e = dalloc(&c->val, m + 8)) != cudaSuccess || (e = dalloc(&c->goal, n)) != cudaSuccess ||
      (e = dalloc(&c->t_rowptr, n + 1)) != cudaSuccess || (e = dalloc(&c->t_col, m + 8)) != cudaSuccess ||
      (e = dalloc(&c->cls, n)) != cudaSuccess || (e = dalloc(&c->qidx, n + 1)) != cudaSuccess ||
      (e = dalloc(&c->vis, 2 * words)) != cudaSuccess || (e = dalloc(&c->queue, 2 * n)) != cudaSuccess ||
      (e = dalloc(&c->bfs, 1)) != cudaSuccess || (e = dalloc(&c->xfull, n)) != cudaSuccess ||
      (e = dalloc(&c->st, 1)) != cudaSuccess || (e = dalloc(&c->bi, 1)) != cudaSuccess ||
      (e = dalloc(&c->part, part_n)) != cudaSuccess || (e = dalloc(&c->ticket, 1)) != cudaSuccess ||
      (e = dalloc(&c->verr, 1)) != cudaSuccess || (e = dalloc(&c->vrow, 1)) != cudaSuccess ||
      (e = dalloc(&c->maxrow, 1)) != cudaSuccess || (e = dalloc(&c->keys, 3)) != cudaSuccess) {
    reach_status s = cuda_fail(nullptr, e, (w + ": allocation").c_str());
    reach_destroy(c);
    return s;
  }
  cudaStream_t s = c->stream;
  e = cudaMemcpyAsync(c->rowptr, rowptr, sizeof(int64_t) * (n + 1), kind_to_dev(flags), s);
  if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(c->col, col, sizeof(int32_t) * m, kind_to_dev(flags), s);
  if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(c->val, val, sizeof(double) * m, kind_to_dev(flags), s);
  if (e == cudaSuccess) {
    if (goal) e = cudaMemcpyAsync(c->goal, goal, n, kind_to_dev(flags), s);
    else e = cudaMemsetAsync(c->goal, 0, n, s);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(c->col + m, 0, 8 * sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->val + m, 0, 8 * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->ticket, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->st, 0, sizeof(SolveState), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->bi, 0, sizeof(BiState), s);
  int64_t ends[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[0], c->rowptr, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[1], c->rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    reach_status st = cuda_fail(nullptr, e, (w + ": copying inputs").c_str());
    reach_destroy(c);
    return st;
  }
  if (ends[0] != 0 || ends[1] != m) {
    reach_destroy(c);
    return fail(nullptr, REACH_EINVAL, w + ": rowptr[0] must be 0 and rowptr[n] must equal m");
  }
  e = launch_validate(c);
  unsigned verr = 0;
  int64_t vrow = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&verr, c->verr, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&vrow, c->vrow, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    reach_status st = cuda_fail(nullptr, e, (w + ": validation").c_str());
    reach_destroy(c);
    return st;
  }
  if (verr) {
    std::string why = w + (general ? ": invalid system" : ": not a Markov chain") + " (first bad row " +
                      std::to_string(vrow) + ":";
    if (verr & VERR_ROWPTR) why += " rowptr not non-decreasing within [0, m];";
    if (verr & VERR_COL) why += " column outside [0, n);";
    if (verr & VERR_VAL) why += general ? " value not finite;" : " value not finite in [0, 1];";
    if (verr & VERR_ROWSUM) why += " row does not sum to 1 within 1e-9;";
    why += ")";
    reach_destroy(c);
    return fail(nullptr, REACH_EINVAL, why);
  }
  *out = c;
  return REACH_OK;
}

static cudaError_t alloc_workspace(reach_ctx* c) {
  const int64_t nq = c->n_q;
  cudaError_t e;
  if ((e = dalloc(&c->x, nq)) != cudaSuccess || (e = dalloc(&c->x2, nq)) != cudaSuccess ||
      (e = dalloc(&c->vr, nq)) != cudaSuccess || (e = dalloc(&c->vq, nq)) != cudaSuccess ||
      (e = dalloc(&c->vp, nq)) != cudaSuccess || (e = dalloc(&c->vv, nq)) != cudaSuccess ||
      (e = dalloc(&c->vs, nq)) != cudaSuccess || (e = dalloc(&c->vt, nq)) != cudaSuccess ||
      (e = dalloc(&c->r32, nq)) != cudaSuccess || (e = dalloc(&c->xf, nq)) != cudaSuccess ||
      (e = dalloc(&c->dl[0], nq)) != cudaSuccess ||
      (e = dalloc(&c->dl[1], nq)) != cudaSuccess)
    free_system(c);
  return e;
}

reach_status reach_create(reach_ctx** out, int64_t n, int64_t m, const int64_t* rowptr,
                          const int32_t* col, const double* val, const uint8_t* goal, int32_t flags,
                          void* stream) {
  return create_common(out, n, m, rowptr, col, val, goal, flags, stream, false, "reach_create");
}

reach_status reach_system_create(reach_ctx** out, int64_t n, int64_t m, const int64_t* rowptr,
                                 const int32_t* col, const double* val, const double* b, int32_t flags,
                                 void* stream) {
  if (!b) return fail(nullptr, REACH_EINVAL, "reach_system_create: b is NULL");
  reach_ctx* c = nullptr;
  reach_status st = create_common(&c, n, m, rowptr, col, val, nullptr, flags, stream, true,
                                  "reach_system_create");
  if (st != REACH_OK) return st;
  cudaStream_t s = c->stream;
  cudaError_t e = cudaEventRecord(c->ev0, s);
  if (e == cudaSuccess) e = extract_all_rows(c);       // d = diag(M), A = -(off-diagonal of M)
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->b, b, sizeof(double) * n, kind_to_dev(flags), s);
  if (e == cudaSuccess) e = check_diagonal(c);
  unsigned verr = 0;
  int64_t vrow = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&verr, c->verr, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&vrow, c->vrow, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && !verr) e = build_jacobi_form(c);
  if (e == cudaSuccess && !verr) e = alloc_workspace(c);
  if (e == cudaSuccess && !verr) e = varah_norm_bound(c, false, &c->kinv_varah);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(c->ev1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  if (e != cudaSuccess) {
    st = cuda_fail(nullptr, e, "reach_system_create");
    reach_destroy(c);
    return st;
  }
  if (verr) {
    reach_destroy(c);
    return fail(nullptr, REACH_EINVAL,
                "reach_system_create: zero diagonal entry in row " + std::to_string(vrow) + " (Jacobi divides by it)");
  }
  c->ms_precompute = ms;
  c->have_classes = true;
  *out = c;
  return REACH_OK;
}

reach_status reach_precompute(reach_ctx* c, int32_t mode) {
  if (!c) return fail(nullptr, REACH_EINVAL, "reach_precompute: NULL context");
  if (mode != REACH_PROB01 && mode != REACH_PROB0_ONLY)
    return fail(c, REACH_EINVAL, "reach_precompute: unknown mode");
  if (c->general) return fail(c, REACH_ESTATE, "reach_precompute: a general system has no partition");
  cudaStream_t s = c->stream;
  drop_graphs(c);
  free_system(c);
  c->have_classes = false;
  c->have_x = false;
  cudaError_t e = cudaEventRecord(c->ev0, s);
  c->rev_ready = false;   // the reversed graph of P is built when a search first needs it
  if (e == cudaSuccess) e = bfs_backward(c, 0, false);
  if (e == cudaSuccess && mode == REACH_PROB01) e = bfs_backward(c, 1, true);
  if (e == cudaSuccess) e = classify_and_extract(c, mode);
  if (e == cudaSuccess) e = build_jacobi_form(c);
  if (e != cudaSuccess) return cuda_fail(c, e, "reach_precompute");
  if ((e = alloc_workspace(c)) != cudaSuccess) return cuda_fail(c, e, "reach_precompute: workspace");
  // the norm bound behind every solve's certified error (Varah's, from the exit margins)
  e = varah_norm_bound(c, false, &c->kinv_varah);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(c->ev1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  if (e != cudaSuccess) return cuda_fail(c, e, "reach_precompute");
  c->ms_precompute = ms;
  c->mode = mode;
  c->have_classes = true;
  return REACH_OK;
}

reach_status reach_get_classes(reach_ctx* c, uint8_t* cls, int32_t flags) {
  if (!c) return fail(nullptr, REACH_EINVAL, "reach_get_classes: NULL context");
  if (!c->have_classes) return fail(c, REACH_ESTATE, "reach_get_classes: call reach_precompute first");
  if (!cls || (flags != REACH_HOST && flags != REACH_DEVICE))
    return fail(c, REACH_EINVAL, "reach_get_classes: bad output");
  cudaError_t e = cudaMemcpyAsync(cls, c->cls, c->n, kind_from_dev(flags), c->stream);
  if (e == cudaSuccess && flags == REACH_HOST) e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? REACH_OK : cuda_fail(c, e, "reach_get_classes");
}

static reach_status start_state(reach_ctx* c, double eps, int64_t max_iter, int64_t max_bodies) {
  SolveState hs;
  std::memset(&hs, 0, sizeof(hs));
  hs.eps = eps;
  hs.max_iter = max_iter;
  hs.status = REACH_ENOTCONV;
  hs.max_bodies = max_bodies;
  cudaError_t e = cudaMemcpyAsync(c->st, &hs, sizeof(hs), cudaMemcpyHostToDevice, c->stream);
  // hs lives on this stack frame: wait for the copy before returning
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? REACH_OK : cuda_fail(c, e, "solve state");
}

reach_status reach_solve(reach_ctx* c, int32_t method, double eps, int64_t max_iter, int32_t refine_k,
                         const double* x0, double* x_out, int32_t flags, reach_info* info) {
  if (!c) return fail(nullptr, REACH_EINVAL, "reach_solve: NULL context");
  if (!c->have_classes) return fail(c, REACH_ESTATE, "reach_solve: call reach_precompute first");
  if (method < REACH_JACOBI_FP64 || method > REACH_SCC_JACOBI)
    return fail(c, REACH_EINVAL, "reach_solve: unknown method");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(c, REACH_EINVAL, "reach_solve: eps must be > 0");
  if (max_iter < 1) return fail(c, REACH_EINVAL, "reach_solve: max_iter must be >= 1");
  const int32_t refine_k_given = refine_k;
  if (refine_k == 0) refine_k = 16;
  if (refine_k < 2 || refine_k > 62 || (refine_k & 1))
    return fail(c, REACH_EINVAL, "reach_solve: refine_k must be even in [2, 62]");
  if (!x_out || (flags != REACH_HOST && flags != REACH_DEVICE))
    return fail(c, REACH_EINVAL, "reach_solve: bad output");
  cudaStream_t s = c->stream;
  const char* at = std::getenv("REACH_AUTOTUNE");
  if (at && at[0] == '1' && c->n_q > 0 && method <= REACH_BICGSTAB_FP64 && c->tune.gm[method] == 0) {
    int chosen = 0;
    float ms = 0.f;
    cudaError_t te = autotune(c, method, &chosen, &ms);
    if (te != cudaSuccess) return cuda_fail(c, te, "reach_solve: autotune");
  }
  if (refine_k == 16 && refine_k_given == 0 && method == REACH_JACOBI_FP64 && c->tune.k_auto > 0)
    refine_k = c->tune.k_auto;
  c->tune.k = refine_k;
  // level-by-level Jacobi: the decomposition first (it resets the solve state)
  double ms_scc = 0.0;
  if (method == REACH_SCC_JACOBI && c->n_q > 0 && !scc_ready(c)) {
    bool ok = true;
    cudaError_t de = scc_decompose(c, 256, &ok);
    if (de != cudaSuccess) return cuda_fail(c, de, "reach_solve: SCC decomposition");
    if (!ok) return fail(c, REACH_ETIMEOUT, "reach_solve: SCC decomposition loop bound reached");
    reach_scc_info si;
    if ((de = scc_outputs(c, nullptr, nullptr, cudaMemcpyDeviceToHost, &si)) != cudaSuccess)
      return cuda_fail(c, de, "reach_solve: SCC decomposition");
    ms_scc = si.ms;
  }
  const int64_t max_bodies = method == REACH_BICGSTAB_FP64 || method == REACH_SCC_JACOBI
                                 ? max_iter + 4 : max_iter / refine_k + 4;
  reach_status rs = start_state(c, eps, max_iter, max_bodies);
  if (rs != REACH_OK) return rs;
  cudaError_t e = cudaSuccess;
  const double* x0q = nullptr;
  if (x0 && c->n_q > 0) {
    e = cudaMemcpyAsync(c->xfull, x0, sizeof(double) * c->n, kind_to_dev(flags), s);
    if (e == cudaSuccess) e = gather_q(c, c->xfull, c->vt);
    x0q = c->vt;
    if (e == cudaSuccess && method == REACH_BICGSTAB_FP64) {
      // the BiCGStab workspace reuses vt: move the start vector out of it first
      e = cudaMemcpyAsync(c->x2, c->vt, sizeof(double) * c->n_q, cudaMemcpyDeviceToDevice, s);
      x0q = c->x2;
    }
  }
  double scc_bytes = 0.0;
  if (e == cudaSuccess) e = cudaEventRecord(c->ev0, s);
  if (e == cudaSuccess && c->n_q > 0) {
    if (method == REACH_JACOBI_FP64) e = solve_jacobi64(c, x0q, false);
    else if (method == REACH_JACOBI_MIXED) e = solve_mixed(c, x0q);
    else if (method == REACH_JACOBI_SEG) e = solve_jacobi_seg(c, x0q);
    else if (method == REACH_SCC_JACOBI) e = solve_scc_jacobi(c, x0q, &scc_bytes);
    else e = solve_bicgstab(c, x0q);
  }
  if (e == cudaSuccess) e = scatter_full(c, c->x, c->xfull);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev1, s);
  SolveState hs;
  std::memset(&hs, 0, sizeof(hs));
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, c->st, sizeof(hs), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(x_out, c->xfull, sizeof(double) * c->n, kind_from_dev(flags), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  if (e != cudaSuccess) return cuda_fail(c, e, "reach_solve");
  if (c->n_q == 0) {
    hs.status = REACH_OK;
    hs.done = 1;
  }
  const double mq = (double)c->m_q, nq = (double)c->n_q;
  double bytes = 0.0;
  // per sweep, Jacobi form: entries (index + value), rows (rowptr, bj, x read, x' write)
  const double colb = c->n_q <= 65536 ? 2.0 : 4.0;   // the mixed sweeps use 16-bit indices when they fit
  if (method == REACH_JACOBI_FP64 || method == REACH_JACOBI_SEG) bytes = (double)hs.iter * (mq * 12.0 + nq * 32.0);
  else if (method == REACH_JACOBI_MIXED)   // FP64 residual (hi, lo; rowptr, bj, x, xf, r, d0) + FP32 sweeps
    bytes = (double)hs.refinements * (mq * (8.0 + colb) + nq * 36.0) +
            (double)(hs.iter - hs.refinements) * (mq * (4.0 + colb) + nq * 16.0);
  else if (method == REACH_SCC_JACOBI) bytes = scc_bytes;
  else bytes = (double)hs.iter * (2.0 * (mq * 12.0 + nq * 40.0) + nq * 8.0 * 10.0);
  if (info) {
    info->iters = hs.iter;
    info->n_q = c->n_q;
    info->m_q = c->m_q;
    info->last_delta = hs.last;
    info->resid_inf = hs.resid;
    info->ms_precompute = c->ms_precompute;
    info->ms_solve = ms + ms_scc;
    info->bytes_moved = bytes;
    info->status = hs.status;
    info->refinements = hs.refinements;
    info->err_bound = error_bound(c->n_q, std::min(c->kinv_varah, c->kinv_tau), hs.resid_ub);
  }
  c->have_x = hs.status == REACH_OK;
  if (hs.status != REACH_OK) {
    const char* why = hs.status == REACH_ENOTCONV ? "reach_solve: max_iter reached before the stopping rule held"
                      : hs.status == REACH_EBREAKDOWN ? "reach_solve: BiCGStab breakdown"
                      : hs.status == REACH_ETIMEOUT ? "reach_solve: loop bound reached"
                                                    : "reach_solve: failed";
    set_err(c, why);
  }
  return (reach_status)hs.status;
}

reach_status reach_get_system(reach_ctx* c, int64_t* n_q, int64_t* m_q, int64_t* rowptr, int32_t* col, double* val,
                              double* d, double* b, int64_t* state, int32_t flags) {
  if (!c) return fail(nullptr, REACH_EINVAL, "reach_get_system: NULL context");
  if (!c->have_classes) return fail(c, REACH_ESTATE, "reach_get_system: call reach_precompute first");
  if (flags != REACH_HOST && flags != REACH_DEVICE) return fail(c, REACH_EINVAL, "reach_get_system: bad flags");
  if (n_q) *n_q = c->n_q;
  if (m_q) *m_q = c->m_q;
  cudaStream_t s = c->stream;
  const cudaMemcpyKind k = kind_from_dev(flags);
  cudaError_t e = cudaSuccess;
  const int64_t nq = c->n_q, mq = c->m_q;
  if (rowptr) e = cudaMemcpyAsync(rowptr, c->a_rowptr, sizeof(int64_t) * (nq + 1), k, s);
  if (e == cudaSuccess && col && mq > 0) e = cudaMemcpyAsync(col, c->a_col, sizeof(int32_t) * mq, k, s);
  if (e == cudaSuccess && val && mq > 0) e = cudaMemcpyAsync(val, c->a_val, sizeof(double) * mq, k, s);
  if (e == cudaSuccess && d && nq > 0) e = cudaMemcpyAsync(d, c->d, sizeof(double) * nq, k, s);
  if (e == cudaSuccess && b && nq > 0) e = cudaMemcpyAsync(b, c->b, sizeof(double) * nq, k, s);
  if (e == cudaSuccess && state && nq > 0) e = cudaMemcpyAsync(state, c->qstate, sizeof(int64_t) * nq, k, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? REACH_OK : cuda_fail(c, e, "reach_get_system");
}

reach_status reach_norm_bound(reach_ctx* c, int32_t method, double eps, int64_t max_iter, double* kinv,
                              reach_info* info) {
  if (!c) return fail(nullptr, REACH_EINVAL, "reach_norm_bound: NULL context");
  if (!c->have_classes) return fail(c, REACH_ESTATE, "reach_norm_bound: call reach_precompute first");
  if (c->general)
    return fail(c, REACH_ESTATE, "reach_norm_bound: needs a chain (the bound uses (I - A)^-1 >= 0)");
  if (method != REACH_JACOBI_FP64 && method != REACH_JACOBI_MIXED && method != REACH_BICGSTAB_FP64)
    return fail(c, REACH_EINVAL, "reach_norm_bound: method must be JACOBI_FP64, JACOBI_MIXED or BICGSTAB_FP64");
  if (!(eps > 0.0) || !std::isfinite(eps) || max_iter < 1)
    return fail(c, REACH_EINVAL, "reach_norm_bound: need eps > 0 and max_iter >= 1");
  if (info) std::memset(info, 0, sizeof(*info));
  if (c->n_q == 0) {
    if (kinv) *kinv = 0.0;
    return REACH_OK;
  }
  cudaError_t e = cudaSuccess;
  if (!c->tau_save && (e = dalloc(&c->tau_save, 2 * c->n_q)) != cudaSuccess)
    return cuda_fail(c, e, "reach_norm_bound: allocation");
  c->tune.k = 16;
  const int64_t max_bodies = method == REACH_BICGSTAB_FP64 ? max_iter + 4 : max_iter / 16 + 4;
  reach_status rs = start_state(c, eps, max_iter, max_bodies);
  if (rs != REACH_OK) return rs;
  cudaStream_t s = c->stream;
  e = cudaEventRecord(c->ev0, s);
  if (e == cudaSuccess) e = tau_rhs_begin(c);
  if (e == cudaSuccess) {
    if (method == REACH_JACOBI_FP64) e = solve_jacobi64(c, nullptr, false);
    else if (method == REACH_JACOBI_MIXED) e = solve_mixed(c, nullptr);
    else e = solve_bicgstab(c, nullptr);
  }
  // the system's own right-hand side goes back whatever happened to the solve
  const cudaError_t e2 = tau_rhs_end(c);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaEventRecord(c->ev1, s);
  SolveState hs;
  std::memset(&hs, 0, sizeof(hs));
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, c->st, sizeof(hs), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  // tau' itself is in c->x whether or not the stopping rule held: any tau' certifies
  double kt = INFINITY;
  if (e == cudaSuccess) e = tau_norm_bound(c, c->x, &kt);
  if (e != cudaSuccess) return cuda_fail(c, e, "reach_norm_bound");
  if (kt < c->kinv_tau) c->kinv_tau = kt;
  if (kinv) *kinv = std::min(c->kinv_varah, c->kinv_tau);
  if (info) {
    info->iters = hs.iter;
    info->n_q = c->n_q;
    info->m_q = c->m_q;
    info->last_delta = hs.last;
    info->resid_inf = hs.resid;
    info->ms_precompute = c->ms_precompute;
    info->ms_solve = ms;
    info->status = hs.status;
    info->refinements = hs.refinements;
    info->err_bound = kt;
  }
  // a tau solve that stopped early still gives a valid (looser, possibly infinite) bound
  if (hs.status != REACH_OK && hs.status != REACH_ENOTCONV) {
    set_err(c, "reach_norm_bound: the solve for tau failed");
    return (reach_status)hs.status;
  }
  return REACH_OK;
}

reach_status reach_scc(reach_ctx* c, int32_t* label, int32_t* level, int32_t flags, int32_t max_rounds,
                       reach_scc_info* info) {
  if (!c) return fail(nullptr, REACH_EINVAL, "reach_scc: NULL context");
  if (!c->have_classes) return fail(c, REACH_ESTATE, "reach_scc: call reach_precompute first");
  if (flags != REACH_HOST && flags != REACH_DEVICE) return fail(c, REACH_EINVAL, "reach_scc: bad flags");
  if (max_rounds < 0) return fail(c, REACH_EINVAL, "reach_scc: max_rounds must be >= 0");
  if (max_rounds == 0) max_rounds = 256;
  if (c->n_q == 0) {
    if (info) std::memset(info, 0, sizeof(*info)), info->exact = 1;
    return REACH_OK;
  }
  bool ok = true;
  cudaError_t e = scc_decompose(c, max_rounds, &ok);
  if (e != cudaSuccess) return cuda_fail(c, e, "reach_scc");
  if (!ok) return fail(c, REACH_ETIMEOUT, "reach_scc: loop bound reached");
  e = scc_outputs(c, label, level, kind_from_dev(flags), info);
  return e == cudaSuccess ? REACH_OK : cuda_fail(c, e, "reach_scc");
}

reach_status reach_autotune(reach_ctx* c, int32_t method, int32_t* lanes, double* sweep_ms,
                            int32_t* check_every) {
  if (!c) return fail(nullptr, REACH_EINVAL, "reach_autotune: NULL context");
  if (!c->have_classes) return fail(c, REACH_ESTATE, "reach_autotune: call reach_precompute first");
  if (method < REACH_JACOBI_FP64 || method > REACH_BICGSTAB_FP64)
    return fail(c, REACH_EINVAL, "reach_autotune: unknown method");
  int chosen = 0;
  float ms = 0.f;
  cudaError_t e = autotune(c, method, &chosen, &ms);
  if (e != cudaSuccess) return cuda_fail(c, e, "reach_autotune");
  if (lanes) *lanes = chosen;
  if (sweep_ms) *sweep_ms = ms;
  if (check_every) *check_every = method == REACH_JACOBI_FP64 ? c->tune.k_auto : 16;
  return REACH_OK;
}

reach_status reach_time_kernel(reach_ctx* c, int32_t kernel, int32_t launches, double* avg_ms) {
  if (!c) return fail(nullptr, REACH_EINVAL, "reach_time_kernel: NULL context");
  if (!c->have_classes) return fail(c, REACH_ESTATE, "reach_time_kernel: call reach_precompute first");
  if (kernel < 0 || kernel > 3 || launches < 1 || launches > 1000 || !avg_ms)
    return fail(c, REACH_EINVAL, "reach_time_kernel: kernel in [0, 3], launches in [1, 1000]");
  float ms = 0.f;
  cudaError_t e = time_kernel(c, kernel, launches, &ms);
  if (e != cudaSuccess) return cuda_fail(c, e, "reach_time_kernel");
  *avg_ms = ms;
  c->have_x = false;   // the launches overwrote solve workspace
  return REACH_OK;
}

reach_status reach_grad(reach_ctx* c, int64_t init, double eps, int64_t max_iter, double* grad,
                        int32_t flags, reach_info* info) {
  return reach_grad_method(c, REACH_JACOBI_FP64, init, eps, max_iter, grad, flags, info);
}

reach_status reach_grad_method(reach_ctx* c, int32_t method, int64_t init, double eps, int64_t max_iter,
                               double* grad, int32_t flags, reach_info* info) {
  if (!c) return fail(nullptr, REACH_EINVAL, "reach_grad: NULL context");
  if (method != REACH_JACOBI_FP64 && method != REACH_BICGSTAB_FP64)
    return fail(c, REACH_EINVAL, "reach_grad: the adjoint method must be JACOBI_FP64 or BICGSTAB_FP64");
  if (c->general) return fail(c, REACH_ESTATE, "reach_grad: defined for chains only");
  if (!c->have_x) return fail(c, REACH_ESTATE, "reach_grad: needs a successful reach_solve first");
  if (init < 0 || init >= c->n) return fail(c, REACH_EINVAL, "reach_grad: init outside [0, n)");
  if (!(eps > 0.0) || max_iter < 1) return fail(c, REACH_EINVAL, "reach_grad: bad eps or max_iter");
  if (!grad || (flags != REACH_HOST && flags != REACH_DEVICE))
    return fail(c, REACH_EINVAL, "reach_grad: bad output");
  cudaStream_t s = c->stream;
  double* gdev = grad;
  cudaError_t e = cudaSuccess;
  if (flags == REACH_HOST) {
    if ((e = dalloc(&gdev, c->m + 1)) != cudaSuccess) return cuda_fail(c, e, "reach_grad: allocation");
  }
  uint8_t kind = 0;
  int64_t row = -1;
  e = cudaMemcpyAsync(&kind, c->cls + init, 1, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&row, c->qidx + init, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  reach_status status = REACH_OK;
  SolveState hs;
  std::memset(&hs, 0, sizeof(hs));
  float ms = 0.f;
  if (e == cudaSuccess && kind != CLS_SQ) {
    e = cudaMemsetAsync(gdev, 0, sizeof(double) * c->m, s);
    hs.status = REACH_OK;
  } else if (e == cudaSuccess) {
    e = build_transposed_system(c);
    if (e == cudaSuccess && c->kinv_varah_t < 0.0) e = varah_norm_bound(c, true, &c->kinv_varah_t);
    const int k = c->tune.k;
    const bool bi = method == REACH_BICGSTAB_FP64;
    if (e == cudaSuccess) {
      reach_status rs = start_state(c, eps, max_iter, bi ? max_iter + 4 : max_iter / k + 4);
      if (rs != REACH_OK) {
        if (flags == REACH_HOST) cudaFree(gdev);
        return rs;
      }
    }
    // right-hand side e_init: vp for the Jacobi sweeps, at_b for BiCGStab (whose p is vp)
    double* rhs = bi ? c->at_b : c->vp;
    const double one = 1.0;
    if (e == cudaSuccess) e = cudaMemsetAsync(rhs, 0, sizeof(double) * c->n_q, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rhs + row, &one, sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev0, s);
    if (e == cudaSuccess) e = bi ? solve_bicgstab_transposed(c) : solve_jacobi64(c, nullptr, true);
    if (e == cudaSuccess) e = grad_entries(c, bi ? c->x2 : c->vr, gdev);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev1, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, c->st, sizeof(hs), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  }
  if (e == cudaSuccess && flags == REACH_HOST)
    e = cudaMemcpyAsync(grad, gdev, sizeof(double) * c->m, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (flags == REACH_HOST) cudaFree(gdev);
  if (e != cudaSuccess) return cuda_fail(c, e, "reach_grad");
  status = (reach_status)hs.status;
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iters = hs.iter;
    info->n_q = c->n_q;
    info->m_q = c->m_q;
    info->last_delta = hs.last;
    info->resid_inf = hs.resid;
    info->ms_precompute = c->ms_precompute;
    info->ms_solve = ms;
    info->status = status;
    // the adjoint's own error: ||(I - A)^-T|| from Varah's margin over the columns of A
    info->err_bound = kind == CLS_SQ ? error_bound(c->n_q, c->kinv_varah_t, hs.resid_ub) : 0.0;
  }
  if (status != REACH_OK) set_err(c, "reach_grad: adjoint solve did not converge");
  return status;
}

}  // extern "C"
