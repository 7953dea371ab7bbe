// C-ABI entry points of the amgc library (declared in include/amgc.h).
#include "amgc_internal.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>

namespace amgc {

static thread_local std::string g_last_error;
std::atomic<long long> g_launches{0};

// ---- stream-ordered device memory
static thread_local cudaStream_t g_alloc_stream = nullptr;
StreamScope::StreamScope(cudaStream_t s) : prev(g_alloc_stream) { g_alloc_stream = s; }
StreamScope::~StreamScope() { g_alloc_stream = prev; }

constexpr int kMaxPoolDevices = 64;
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[kMaxPoolDevices] = {};

// The library's memory pool on the current device (created on first use, nothing released to
// the driver until amgc_trim_memory); nullptr with the error set if it cannot be had.
static cudaMemPool_t device_pool() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxPoolDevices) {
    set_error("memory pool: no usable current device");
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) {
      set_error(std::string("cudaMemPoolCreate: ") + cudaGetErrorString(e));
      return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[dev] = pool;
  }
  return g_pools[dev];
}

int pool_alloc(void** p, size_t bytes) {
  *p = nullptr;
  cudaMemPool_t pool = device_pool();
  if (!pool) return AMGC_ECUDA;
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, g_alloc_stream);
  if (e != cudaSuccess) {
    *p = nullptr;
    set_error(std::string("device allocation of ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
    return AMGC_ENOMEM;
  }
  return AMGC_OK;
}

void pool_free(void* p) { cudaFreeAsync(p, g_alloc_stream); }
bool allocations_ordered_on(cudaStream_t s) { return s == g_alloc_stream; }
void set_error(const std::string& msg) { g_last_error = msg; }

static thread_local std::string g_launch_site;
LaunchSite::~LaunchSite() {
  if (g_launch_site.empty() && cudaPeekAtLastError() != cudaSuccess) {
    const char* base = std::strrchr(file, '/');
    g_launch_site = std::string(" (launch at ") + (base ? base + 1 : file) + ":" + std::to_string(line) + ")";
  }
}
std::string take_launch_site() {
  std::string s;
  s.swap(g_launch_site);
  return s;
}

// Largest coarsest system solved with the dense explicit inverse.
constexpr int kMaxDenseRows = 16384;

// rows of the largest instance of a level (the whole level when not batched)
static int max_instance_rows(const amgc_hierarchy* h, const Level& L) {
  if (h->n_inst <= 1) return L.rows();
  int m = 0;
  for (int q = 0; q < h->n_inst; ++q)
    m = std::max(m, L.bu * (L.nptr[q + 1] - L.nptr[q]) + 3 * (L.lptr[q + 1] - L.lptr[q]));
  return m;
}

static int build(amgc_hierarchy* h, const amgc_bsr* K, const double* D_diag, const amgc_csr* M,
                 const int32_t* slave_node, const int32_t* master_node, const double* triad,
                 const uint8_t* active, const int32_t* body_id, const double* nullspace,
                 const std::vector<int>& h_nptr, const std::vector<int>& h_lptr) {
  const auto t0 = std::chrono::steady_clock::now();
  std::memset(&h->stats, 0, sizeof(h->stats));
  AMGC_TRY(h->status.alloc(1));
  AMGC_CUDA_TRY(cudaMemsetAsync(h->status.p, 0, sizeof(int), h->stream));
  AMGC_TRY(h->partial.alloc(4096));
  AMGC_CUDA_TRY(cudaMallocHost(&h->h_pinned, 64 * sizeof(double)));
  h->L.reserve(16);
  h->L.emplace_back();
  h->L[0].nptr = h_nptr;
  h->L[0].lptr = h_lptr;
  {
    PhaseTimer pt(h, 0);
    AMGC_TRY(build_fine_level(h, K, D_diag, M, slave_node, master_node, triad, active, body_id, nullspace));
  }
  {
    PhaseTimer pt(h, 9);
    AMGC_TRY(build_sell(h, 0));
  }
  const amgc_options& o = h->opts;
  while ((int)h->L.size() < std::min(o.levels_max, 16) && max_instance_rows(h, h->L.back()) >= o.coarse_max_rows) {
    const int l = (int)h->L.size() - 1;
    {
      PhaseTimer pt(h, 4);
      AMGC_TRY(smoother_setup(h, l));
    }
    AMGC_TRY(coarsen_level(h, l));
    if (h->L[l + 1].nn >= h->L[l].nn) {   // no reduction: keep the finer level as the coarsest
      h->L.pop_back();
      break;
    }
  }
  const int lc = (int)h->L.size() - 1;
  // the level smoother on the coarsest level needs no merged dense matrix
  const bool coarse_smooth = o.coarse_solver == 1 && lc > 0;
  if (!coarse_smooth && max_instance_rows(h, h->L[lc]) > kMaxDenseRows) {
    set_error("coarsest level has " + std::to_string(h->L[lc].rows()) +
              " rows; raise levels_max or lower coarse_max_rows (dense limit " + std::to_string(kMaxDenseRows) + ")");
    return AMGC_EINVAL;
  }
  {
    PhaseTimer pt(h, 8);
    if (coarse_smooth) {
      AMGC_TRY(smoother_setup(h, lc));
      AMGC_TRY(smoother_finish(h, lc));
    } else {
      AMGC_TRY(coarse_setup(h, lc));
    }
  }
  {
    PhaseTimer pt(h, 9);
    if (lc > 0) AMGC_TRY(build_sell(h, 0));
    AMGC_TRY(make_views(h));
    if (o.autotune && lc > 0) AMGC_TRY(autotune(h));
  }
  AMGC_CUDA_TRY(cudaStreamSynchronize(h->stream));
  // statistics
  amgc_stats_t& st = h->stats;
  st.n_levels = (int)h->L.size();
  double nnz0 = 0.0, nnz_all = 0.0;
  for (int l = 0; l < st.n_levels; ++l) {
    const Level& L = h->L[l];
    st.rows[l] = L.rows();
    st.disp_nodes[l] = L.nn;
    st.lm_nodes[l] = L.nl;
    st.dofs_per_node[l] = L.bu;
    st.nnz[l] = L.K.nnzb * L.bu * L.bu + L.B1.nnzb * L.bu * 3 + L.B2.nnzb * 3 * L.bu + (int64_t)L.nl * 9;
    st.lambda_max[l] = L.lam_max;
    if (l == 0) nnz0 = (double)st.nnz[l];
    nnz_all += (double)st.nnz[l];
  }
  st.operator_complexity = nnz0 > 0 ? nnz_all / nnz0 : 0.0;
  st.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return AMGC_OK;
}

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
PhaseTimer::PhaseTimer(amgc_hierarchy* hh, int ph) : h(hh), phase(ph) {
  cudaStreamSynchronize(h->stream);
  t0 = now_ms();
}
PhaseTimer::~PhaseTimer() {
  cudaStreamSynchronize(h->stream);
  h->stats.setup_phase_ms[phase] += now_ms() - t0;
}

constexpr int kProfPairs = 1024;

int prof_flush(amgc_hierarchy* h) {
  if (h->prof_pending == 0) return AMGC_OK;
  AMGC_CUDA_TRY(cudaEventSynchronize(h->prof_ev[2 * h->prof_pending - 1]));
  for (int i = 0; i < h->prof_pending; ++i) {
    float ms = 0.f;
    AMGC_CUDA_TRY(cudaEventElapsedTime(&ms, h->prof_ev[2 * i], h->prof_ev[2 * i + 1]));
    h->prof_ms += ms;
  }
  h->prof_pending = 0;
  return AMGC_OK;
}

int prof_begin(amgc_hierarchy* h, int kind) {
  if (!(h->prof & kind)) return AMGC_OK;
  if (h->prof_ev.empty()) {
    h->prof_ev.resize(2 * kProfPairs);
    for (auto& e : h->prof_ev) AMGC_CUDA_TRY(cudaEventCreate(&e));
  }
  if (h->prof_pending == kProfPairs) AMGC_TRY(prof_flush(h));
  AMGC_CUDA_TRY(cudaEventRecord(h->prof_ev[2 * h->prof_pending], h->stream));
  return AMGC_OK;
}

int prof_end(amgc_hierarchy* h, int kind, double bytes, double flops) {
  if (!(h->prof & kind)) return AMGC_OK;
  AMGC_CUDA_TRY(cudaEventRecord(h->prof_ev[2 * h->prof_pending + 1], h->stream));
  h->prof_pending++;
  h->prof_launches++;
  h->prof_bytes += bytes;
  h->prof_flops += flops;
  return AMGC_OK;
}

}  // namespace amgc

using namespace amgc;

extern "C" {

void amgc_default_options(amgc_options* o) {
  if (!o) return;
  o->levels_max = 10;
  o->coarse_max_rows = 5000;
  o->transfer = 1;
  o->smoother_sweeps = 1;
  o->jacobi_sweeps = 1;
  o->simplec = 0;
  o->precision = 64;
  o->fgmres_restart = 50;
  o->fgmres_maxit = 1000;
  o->seed = 0x5EED;
  o->sa_omega = 4.0 / 3.0;
  o->jacobi_omega = 0.0;
  o->simple_alpha = 0.8;
  o->tol = 1e-8;
  o->autotune = 0;
  o->schur_damping = 0;
  o->coarse_solver = 0;
}

int amgc_setup(const amgc_bsr* K, const double* D_diag, const amgc_csr* M, const int32_t* slave_node,
               const int32_t* master_node, const double* triad, const uint8_t* active, const int32_t* body_id,
               const double* nullspace, const amgc_options* opts, void* stream, struct amgc_hierarchy** out) {
  if (!out) {
    set_error("amgc_setup: out is NULL");
    return AMGC_EINVAL;
  }
  *out = nullptr;
  if (!K || !M || !opts || !K->rowptr || !K->col || !K->val || !body_id || !nullspace || !M->rowptr ||
      K->br != 3 || K->bc != 3 || K->n_brow != K->n_bcol || K->n_brow <= 0 || M->n_row < 1 || M->n_col < 0 ||
      (M->n_row > 0 && (!D_diag || !slave_node || !triad || !active)) || (M->n_col > 0 && !master_node) ||
      opts->levels_max < 1 || opts->smoother_sweeps < 0 || opts->jacobi_sweeps < 1 || opts->fgmres_restart < 1 ||
      opts->fgmres_restart > 256 || opts->fgmres_maxit < 1 || !(opts->tol > 0.0) || (opts->precision != 64 && opts->precision != 32) ||
      (opts->schur_damping != 0 && opts->schur_damping != 1) || (opts->coarse_solver != 0 && opts->coarse_solver != 1)) {
    set_error(M && M->n_row < 1 ? "amgc_setup: no slave interface nodes (the system has no multiplier block)"
                                : "amgc_setup: invalid argument");
    return AMGC_EINVAL;
  }
  amgc_hierarchy* h = new (std::nothrow) amgc_hierarchy();
  if (!h) return AMGC_ENOMEM;
  h->opts = *opts;
  h->stream = (cudaStream_t)stream;
  StreamScope scope_(h->stream);
  h->n_inst = 1;
  std::vector<int> np = {0, K->n_brow}, lp = {0, M->n_row};
  int st = build(h, K, D_diag, M, slave_node, master_node, triad, active, body_id, nullspace, np, lp);
  if (st == AMGC_OK && cudaStreamSynchronize(h->stream) != cudaSuccess) {
    set_error("setup: stream synchronisation failed");
    st = AMGC_ECUDA;
  }
  if (st != AMGC_OK) {
    cudaStreamSynchronize(h->stream);
    amgc_destroy(h);
    return st;
  }
  *out = h;
  return AMGC_OK;
}

int amgc_setup_batched(const amgc_bsr* K, const double* D_diag, const amgc_csr* M, const int32_t* slave_node,
                       const int32_t* master_node, const double* triad, const uint8_t* active, const int32_t* body_id,
                       const double* nullspace, int32_t n_inst, const int32_t* node_ptr, const int32_t* lm_ptr,
                       const amgc_options* opts, void* stream, struct amgc_hierarchy** out) {
  if (!out || n_inst < 1 || !node_ptr || !lm_ptr || !K || !M || !opts) {
    set_error("amgc_setup_batched: invalid argument");
    if (out) *out = nullptr;
    return AMGC_EINVAL;
  }
  *out = nullptr;
  std::vector<int> np(node_ptr, node_ptr + n_inst + 1), lp(lm_ptr, lm_ptr + n_inst + 1);
  bool ok = np[0] == 0 && lp[0] == 0 && np[n_inst] == K->n_brow && lp[n_inst] == M->n_row;
  for (int q = 0; q < n_inst && ok; ++q) ok = np[q + 1] > np[q] && lp[q + 1] > lp[q];
  if (!ok) {
    set_error("amgc_setup_batched: node_ptr / lm_ptr must be strictly ascending and cover K and M");
    return AMGC_EINVAL;
  }
  if (n_inst == 1)
    return amgc_setup(K, D_diag, M, slave_node, master_node, triad, active, body_id, nullspace, opts, stream, out);
  if (!K->rowptr || !K->col || !K->val || !body_id || !nullspace || !M->rowptr || K->br != 3 || K->bc != 3 ||
      K->n_brow != K->n_bcol || (M->n_row > 0 && (!D_diag || !slave_node || !triad || !active)) ||
      (M->n_col > 0 && !master_node) || opts->levels_max < 1 || opts->smoother_sweeps < 0 ||
      opts->jacobi_sweeps < 1 || opts->fgmres_restart < 1 || opts->fgmres_restart > 256 || opts->fgmres_maxit < 1 ||
      !(opts->tol > 0.0) || (opts->precision != 64 && opts->precision != 32) ||
      (opts->schur_damping != 0 && opts->schur_damping != 1) || opts->coarse_solver != 0) {
    set_error(opts->coarse_solver != 0 ? "amgc_setup_batched: coarse_solver 1 is for single hierarchies only"
                                       : "amgc_setup_batched: invalid argument");
    return AMGC_EINVAL;
  }
  amgc_hierarchy* h = new (std::nothrow) amgc_hierarchy();
  if (!h) return AMGC_ENOMEM;
  h->opts = *opts;
  h->stream = (cudaStream_t)stream;
  StreamScope scope_(h->stream);
  h->n_inst = n_inst;
  int st = build(h, K, D_diag, M, slave_node, master_node, triad, active, body_id, nullspace, np, lp);
  if (st == AMGC_OK && cudaStreamSynchronize(h->stream) != cudaSuccess) {
    set_error("setup: stream synchronisation failed");
    st = AMGC_ECUDA;
  }
  if (st != AMGC_OK) {
    cudaStreamSynchronize(h->stream);
    amgc_destroy(h);
    return st;
  }
  *out = h;
  return AMGC_OK;
}

int amgc_solve_batched(struct amgc_hierarchy* h, int32_t nrhs, const double* rhs, double* x, int32_t* iters,
                       double* relres, void* stream) {
  if (!h || nrhs < 1 || !rhs || !x || rhs == x) {
    set_error("amgc_solve_batched: invalid argument");
    return AMGC_EINVAL;
  }
  h->stream = (cudaStream_t)stream;
  StreamScope scope_(h->stream);
  return fgmres_batched(h, nrhs, rhs, x, iters, relres);
}

int amgc_vcycle(struct amgc_hierarchy* h, const double* r, double* z, void* stream) {
  if (!h || !r || !z || r == z) {
    set_error("amgc_vcycle: invalid argument");
    return AMGC_EINVAL;
  }
  h->stream = (cudaStream_t)stream;
  StreamScope scope_(h->stream);
  AMGC_TRY(precond_apply(h, r, z));
  // the staged FP32 apply's bounded waits report through the status word
  if (staged_apply_in_use(h)) return check_status(h, "amgc_vcycle (FP32 V-cycle)");
  return AMGC_OK;
}

int amgc_set_row_mapping(struct amgc_hierarchy* h, int32_t level, int32_t matrix, int32_t precision,
                         int32_t mapping) {
  if (!h) {
    set_error("amgc_set_row_mapping: invalid argument");
    return AMGC_EINVAL;
  }
  StreamScope scope_(h->stream);
  AMGC_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return set_row_mapping(h, level, matrix, precision, mapping);
}

int amgc_set_smoother(struct amgc_hierarchy* h, int32_t kind, double omega, int32_t sgs_sweeps, double sgs_omega,
                      void* stream) {
  if (!h || kind < 0 || kind > 3 ||
      (kind != 0 && (!(omega > 0.0) || !std::isfinite(omega) || sgs_sweeps < 1 || !(sgs_omega > 0.0) ||
                     !std::isfinite(sgs_omega)))) {
    set_error("amgc_set_smoother: invalid argument");
    return AMGC_EINVAL;
  }
  if (kind != 0 && (h->n_inst > 1 || h->opts.precision != 64)) {
    set_error("amgc_set_smoother: the block smoothers need a single FP64 hierarchy");
    return AMGC_EINVAL;
  }
  h->stream = (cudaStream_t)stream;
  StreamScope scope_(h->stream);
  const int prev = h->smoother_kind;
  h->smoother_kind = kind;
  h->block_omega = omega;
  h->sgs_sweeps = sgs_sweeps;
  h->sgs_omega = sgs_omega;
  if (kind != 0) {
    const int st = block_smoother_setup(h, false);
    if (st != AMGC_OK) {
      h->smoother_kind = prev;
      return st;
    }
  }
  drop_cycle_graphs(h);
  return AMGC_OK;
}

int amgc_set_preconditioner(struct amgc_hierarchy* h, int32_t kind, int32_t outer_sweeps, double omega, void* stream) {
  if (!h || (kind != 0 && kind != 1) || (kind == 1 && (outer_sweeps < 1 || !(omega > 0.0) || !std::isfinite(omega)))) {
    set_error("amgc_set_preconditioner: invalid argument");
    return AMGC_EINVAL;
  }
  if (kind == 1 && (h->n_inst > 1 || h->opts.precision != 64)) {
    set_error("amgc_set_preconditioner: nested multigrid needs a single FP64 hierarchy");
    return AMGC_EINVAL;
  }
  h->stream = (cudaStream_t)stream;
  StreamScope scope_(h->stream);
  if (kind == 1) {
    h->nest_sweeps = outer_sweeps;
    h->nest_omega = omega;
    if (h->nest.empty()) AMGC_TRY(nested_setup(h));
  }
  h->prec_kind = kind;
  return AMGC_OK;
}

int amgc_set_wait_limit(struct amgc_hierarchy* h, int64_t polls) {
  if (!h || polls > 0xffffffffLL) {
    set_error("amgc_set_wait_limit: invalid argument");
    return AMGC_EINVAL;
  }
  AMGC_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return set_wait_limit(h, polls);
}

int amgc_apply(struct amgc_hierarchy* h, const double* x, double* y, void* stream) {
  if (!h || !x || !y || x == y) {
    set_error("amgc_apply: invalid argument");
    return AMGC_EINVAL;
  }
  h->stream = (cudaStream_t)stream;
  StreamScope scope_(h->stream);
  return saddle_apply(h, 0, x, y);
}

int amgc_solve(struct amgc_hierarchy* h, const double* rhs, double* x, int32_t* iters, double* relres, void* stream) {
  if (!h || !rhs || !x || rhs == x) {
    set_error("amgc_solve: invalid argument");
    return AMGC_EINVAL;
  }
  h->stream = (cudaStream_t)stream;
  StreamScope scope_(h->stream);
  int it = 0;
  double rr = 0.0;
  int st = fgmres(h, rhs, x, 0.0, &it, &rr);
  if (iters) *iters = it;
  if (relres) *relres = rr;
  return st;
}

int amgc_solve_split(struct amgc_hierarchy* h, const double* rhs, double* u, double* lam, int32_t* iters,
                     double* relres, void* stream) {
  if (!h || !rhs || !u || (!lam && h->L[0].nl > 0) || u == rhs || lam == rhs) {
    set_error("amgc_solve_split: invalid argument");
    return AMGC_EINVAL;
  }
  h->stream = (cudaStream_t)stream;
  StreamScope scope_(h->stream);
  const size_t n = (size_t)h->L[0].rows();
  const size_t nu = (size_t)h->L[0].nu();
  DBuf<double> x;
  AMGC_TRY(x.alloc(n));
  int it = 0;
  double rr = 0.0;
  const int st = fgmres(h, rhs, x.p, 0.0, &it, &rr);
  if (iters) *iters = it;
  if (relres) *relres = rr;
  if (st == AMGC_OK || st == AMGC_NOT_CONVERGED) {
    AMGC_CUDA_TRY(cudaMemcpyAsync(u, x.p, nu * sizeof(double), cudaMemcpyDefault, h->stream));
    if (n > nu) AMGC_CUDA_TRY(cudaMemcpyAsync(lam, x.p + nu, (n - nu) * sizeof(double), cudaMemcpyDefault, h->stream));
  }
  AMGC_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return st;
}

int amgc_solve_host(struct amgc_hierarchy* h, const double* rhs_host, double* x_host, int32_t* iters, double* relres,
                    void* stream) {
  if (!h || !rhs_host || !x_host) {
    set_error("amgc_solve_host: invalid argument");
    return AMGC_EINVAL;
  }
  h->stream = (cudaStream_t)stream;
  StreamScope scope_(h->stream);
  const size_t n = (size_t)h->L[0].rows();
  DBuf<double> b, x;
  AMGC_TRY(b.alloc(n));
  AMGC_TRY(x.alloc(n));
  AMGC_CUDA_TRY(cudaMemcpyAsync(b.p, rhs_host, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  int it = 0;
  double rr = 0.0;
  int st = fgmres(h, b.p, x.p, 0.0, &it, &rr);
  if (st == AMGC_OK || st == AMGC_NOT_CONVERGED)
    AMGC_CUDA_TRY(cudaMemcpyAsync(x_host, x.p, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  AMGC_CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (iters) *iters = it;
  if (relres) *relres = rr;
  return st;
}

static int enter_transposed(amgc_hierarchy* h, void* stream, const char* where) {
  if (!h) {
    set_error(std::string(where) + ": invalid argument");
    return AMGC_EINVAL;
  }
  if (h->n_inst > 1) {
    set_error(std::string(where) + ": not available for batched hierarchies");
    return AMGC_EINVAL;
  }
  if (h->opts.coarse_solver != 0) {
    set_error(std::string(where) + ": the transposed cycle needs coarse_solver 0 (the coarsest inverse)");
    return AMGC_EINVAL;
  }
  if (h->prec_kind != 0 || h->smoother_kind != 0) {
    set_error(std::string(where) + ": the transposed cycle is that of the coupled V-cycle with CheapSIMPLE smoothing");
    return AMGC_EINVAL;
  }
  h->stream = (cudaStream_t)stream;
  StreamScope scope_(h->stream);
  if (!h->L[0].has_transposed) AMGC_TRY(transposed_setup(h));
  h->transposed = true;
  return AMGC_OK;
}

int amgc_apply_transposed(struct amgc_hierarchy* h, const double* x, double* y, void* stream) {
  if (!x || !y || x == y) {
    set_error("amgc_apply_transposed: invalid argument");
    return AMGC_EINVAL;
  }
  AMGC_TRY(enter_transposed(h, stream, "amgc_apply_transposed"));
  int st = saddle_apply(h, 0, x, y);
  h->transposed = false;
  return st;
}

int amgc_vcycle_transposed(struct amgc_hierarchy* h, const double* r, double* z, void* stream) {
  if (!r || !z || r == z) {
    set_error("amgc_vcycle_transposed: invalid argument");
    return AMGC_EINVAL;
  }
  AMGC_TRY(enter_transposed(h, stream, "amgc_vcycle_transposed"));
  int st = precond_apply(h, r, z);
  h->transposed = false;
  return st;
}

int amgc_solve_transposed(struct amgc_hierarchy* h, const double* rhs, double* x, double tol, int32_t* iters,
                          double* relres, void* stream) {
  if (!rhs || !x || rhs == x) {
    set_error("amgc_solve_transposed: invalid argument");
    return AMGC_EINVAL;
  }
  AMGC_TRY(enter_transposed(h, stream, "amgc_solve_transposed"));
  int it = 0;
  double rr = 0.0;
  int st = fgmres(h, rhs, x, tol, &it, &rr);
  h->transposed = false;
  if (iters) *iters = it;
  if (relres) *relres = rr;
  return st;
}

int amgc_grad_scatter(struct amgc_hierarchy* h, const double* adj, const double* x, double* gK, double* gB1,
                      double* gB2, void* stream) {
  if (!h || !adj || !x || !gK) {
    set_error("amgc_grad_scatter: invalid argument");
    return AMGC_EINVAL;
  }
  h->stream = (cudaStream_t)stream;
  StreamScope scope_(h->stream);
  return grad_scatter(h, adj, x, gK, gB1, gB2);
}

int amgc_grad_elements(int32_t ne, const int32_t* conn, const int32_t* shape, const double* Khat,
                       const int32_t* node_free, const double* adj, const double* x, const double* uD,
                       const uint8_t* lift_mask, const double* E, double* gE, double* gt, void* stream) {
  if (ne < 0 || (ne > 0 && (!conn || !shape || !Khat || !node_free || !adj || !x || !uD || !gE)) ||
      (gt && (!lift_mask || !E))) {
    set_error("amgc_grad_elements: invalid argument");
    return AMGC_EINVAL;
  }
  StreamScope scope_((cudaStream_t)stream);
  return grad_elements(ne, conn, shape, Khat, node_free, adj, x, uD, lift_mask, E, gE, gt, (cudaStream_t)stream);
}

int amgc_stats(const struct amgc_hierarchy* h, amgc_stats_t* out) {
  if (!h || !out) {
    set_error("amgc_stats: invalid argument");
    return AMGC_EINVAL;
  }
  *out = h->stats;
  return AMGC_OK;
}

int64_t amgc_export(const struct amgc_hierarchy* h, int32_t level, int32_t what, void* dst, int64_t bytes) {
  if (!h || level < 0 || level >= (int)h->L.size()) {
    set_error("amgc_export: invalid level");
    return AMGC_EINVAL;
  }
  const Level& L = h->L[level];
  const void* src = nullptr;
  int64_t nb = 0;
  double scal[2] = {L.lam_max, L.omega_j};
  switch (what) {
    case AMGC_EXPORT_AGG: src = L.agg.p; nb = L.agg.p ? (int64_t)L.nn * 4 : 0; break;
    case AMGC_EXPORT_LAGG: src = L.lagg.p; nb = L.lagg.p ? (int64_t)L.nl * 4 : 0; break;
    case AMGC_EXPORT_P_ROWPTR: src = L.P.rowptr.p; nb = L.P.rowptr.p ? (int64_t)(L.P.nbr + 1) * 4 : 0; break;
    case AMGC_EXPORT_P_COL: src = L.P.col.p; nb = L.P.nnzb * 4; break;
    case AMGC_EXPORT_P_VAL: src = L.P.val.p; nb = L.P.nnzb * L.P.br * L.P.bc * 8; break;
    case AMGC_EXPORT_K_ROWPTR: src = L.K.rowptr.p; nb = (int64_t)(L.K.nbr + 1) * 4; break;
    case AMGC_EXPORT_K_COL: src = L.K.col.p; nb = L.K.nnzb * 4; break;
    case AMGC_EXPORT_K_VAL: src = L.K.val.p; nb = L.K.nnzb * L.K.br * L.K.bc * 8; break;
    case AMGC_EXPORT_B1_ROWPTR: src = L.B1.rowptr.p; nb = (int64_t)(L.B1.nbr + 1) * 4; break;
    case AMGC_EXPORT_B1_COL: src = L.B1.col.p; nb = L.B1.nnzb * 4; break;
    case AMGC_EXPORT_B1_VAL: src = L.B1.val.p; nb = L.B1.nnzb * L.B1.br * L.B1.bc * 8; break;
    case AMGC_EXPORT_B2_ROWPTR: src = L.B2.rowptr.p; nb = (int64_t)(L.B2.nbr + 1) * 4; break;
    case AMGC_EXPORT_B2_COL: src = L.B2.col.p; nb = L.B2.nnzb * 4; break;
    case AMGC_EXPORT_B2_VAL: src = L.B2.val.p; nb = L.B2.nnzb * L.B2.br * L.B2.bc * 8; break;
    case AMGC_EXPORT_Z: src = L.Z.p; nb = (int64_t)L.nl * 9 * 8; break;
    case AMGC_EXPORT_SINV: src = L.Sinv.p; nb = L.Sinv.p ? (int64_t)L.nl * 9 * 8 : 0; break;
    case AMGC_EXPORT_NULLSPACE: src = L.B.p; nb = (int64_t)L.nu() * 6 * 8; break;
    case AMGC_EXPORT_PL_W: src = L.pl_w.p; nb = L.pl_w.p ? (int64_t)L.nl * 8 : 0; break;
    case AMGC_EXPORT_ATINV: src = L.atinv.p; nb = L.atinv.p ? (int64_t)L.nu() * 8 : 0; break;
    case AMGC_EXPORT_OMEGA: src = scal; nb = 16; break;
    case AMGC_EXPORT_COARSE_INV: src = L.Ainv.p; nb = L.Ainv.p ? (int64_t)L.Ainv.n * 8 : 0; break;
    case AMGC_EXPORT_SCHUR_RHO: src = L.schur_rho.data(); nb = (int64_t)L.schur_rho.size() * 8; break;
    case AMGC_EXPORT_COLOR: src = L.color.p; nb = L.color.p ? (int64_t)L.nn * 4 : 0; break;
    default: set_error("amgc_export: unknown array"); return AMGC_EINVAL;
  }
  if (!dst || nb == 0) return nb;
  if (bytes < nb) {
    set_error("amgc_export: destination too small");
    return AMGC_EINVAL;
  }
  AMGC_CUDA_TRY(cudaStreamSynchronize(h->stream));
  AMGC_CUDA_TRY(cudaMemcpy(dst, src, nb, cudaMemcpyDefault));
  return nb;
}

int amgc_profile(struct amgc_hierarchy* h, int32_t enable) {
  if (!h) {
    set_error("amgc_profile: invalid argument");
    return AMGC_EINVAL;
  }
  AMGC_TRY(prof_flush(h));
  h->prof = enable & 3;
  h->prof_ms = 0.0;
  h->prof_bytes = 0.0;
  h->prof_flops = 0.0;
  h->prof_launches = 0;
  return AMGC_OK;
}

int amgc_profile_read(struct amgc_hierarchy* h, double* total_ms, int64_t* launches, double* bytes,
                      double* flops) {
  if (!h) {
    set_error("amgc_profile_read: invalid argument");
    return AMGC_EINVAL;
  }
  AMGC_TRY(prof_flush(h));
  if (total_ms) *total_ms = h->prof_ms;
  if (launches) *launches = h->prof_launches;
  if (bytes) *bytes = h->prof_bytes;
  if (flops) *flops = h->prof_flops;
  return AMGC_OK;
}

void amgc_destroy(struct amgc_hierarchy* h) {
  if (!h) return;
  StreamScope scope_(h->stream);
  cudaStreamSynchronize(h->stream);
  if (h->aux_stream) {
    cudaStreamSynchronize(h->aux_stream);
    cudaStreamDestroy(h->aux_stream);
  }
  for (auto& L : h->L)
    if (L.lmx_done) cudaEventDestroy(L.lmx_done);
  for (auto& e : h->prof_ev) cudaEventDestroy(e);
  for (auto& g : h->cycle_graph)
    if (g) cudaGraphExecDestroy(g);
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  if (h->side_stream) {
    cudaStreamSynchronize(h->side_stream);
    cudaStreamDestroy(h->side_stream);
  }
  if (h->fork_ev) cudaEventDestroy(h->fork_ev);
  if (h->join_ev) cudaEventDestroy(h->join_ev);
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  mc_state_free(h->mc);
  delete h;
}

const char* amgc_strerror(int code) {
  switch (code) {
    case AMGC_OK: return "ok";
    case AMGC_EINVAL: return "invalid argument or input structure";
    case AMGC_ESINGULAR: return "singular block, rank-deficient aggregate or coarse pivot";
    case AMGC_NOT_CONVERGED: return "FGMRES did not converge";
    case AMGC_BREAKDOWN: return "non-finite value or Krylov breakdown";
    case AMGC_TIMEOUT: return "bounded device wait expired";
    case AMGC_ECUDA: return "CUDA runtime error";
    case AMGC_ENOMEM: return "device allocation failed";
    default: return "unknown error";
  }
}

const char* amgc_last_error(void) { return g_last_error.c_str(); }

int64_t amgc_launch_count(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

int amgc_f64_to_f32(int64_t n, const double* x, float* y, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y))) {
    set_error("amgc_f64_to_f32: invalid argument");
    return AMGC_EINVAL;
  }
  return convert_f64_f32(n, x, y, (cudaStream_t)stream);
}

int amgc_trim_memory(void) {
  cudaMemPool_t pool = device_pool();
  if (!pool) return AMGC_ECUDA;
  AMGC_CUDA_TRY(cudaDeviceSynchronize());
  AMGC_CUDA_TRY(cudaMemPoolTrimTo(pool, 0));
  return AMGC_OK;
}

}  // extern "C"
