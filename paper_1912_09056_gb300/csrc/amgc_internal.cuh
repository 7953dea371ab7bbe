// Internal data structures and device helpers of the amgc library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/amgc.h"

namespace amgc {

struct McState;                 // work buffers of the multi-column cycle (batch_cycle.cu)
constexpr int kMcCols = 4;      // right-hand sides per multi-column cycle

// ------------------------------------------------------------------ error handling
void set_error(const std::string& msg);
// Source location of the first launch in this thread that left a launch error, if any since the
// last report (appended to the message of the CUDA error that reports it; then cleared).
std::string take_launch_site();

#define AMGC_CUDA_TRY(expr)                                                                          \
  do {                                                                                               \
    cudaError_t e_ = (expr);                                                                         \
    if (e_ != cudaSuccess) {                                                                         \
      ::amgc::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_) + ::amgc::take_launch_site()); \
      return e_ == cudaErrorMemoryAllocation ? AMGC_ENOMEM : AMGC_ECUDA;                             \
    }                                                                                                \
  } while (0)

#define AMGC_TRY(expr)            \
  do {                            \
    int s_ = (expr);              \
    if (s_ != AMGC_OK) return s_; \
  } while (0)

// Every kernel launch of the library goes through AMGC_LAUNCH, which counts it.  A LaunchSite
// temporary lives to the end of the launch expression; its destructor notes the source line of
// the first launch that leaves a launch error (an invalid configuration), so that the error, when
// a later check reports it, names the launch.
extern std::atomic<long long> g_launches;
struct LaunchSite {
  const char* file;
  int line;
  LaunchSite(const char* f, int l) : file(f), line(l) {}
  ~LaunchSite();
};
#define AMGC_LAUNCH(...) \
  (::amgc::LaunchSite(__FILE__, __LINE__), ::amgc::g_launches.fetch_add(1, std::memory_order_relaxed), __VA_ARGS__)

// Device status bits written by kernels that detect bad input or a singular block.
enum : int {
  ST_BAD_INDEX = 1,
  ST_NO_DIAG = 2,
  ST_SINGULAR = 4,
  ST_RANK = 8,
  ST_ROW_TOO_DENSE = 16,
  ST_NONFINITE = 32,
  ST_TIMEOUT = 64,           // a bounded wait on an asynchronous copy gave up
};

// ------------------------------------------------------------------ device memory
// Device buffers come from a stream-ordered memory pool of the current device (created on first
// use; freed memory stays in the pool for reuse until amgc_trim_memory).  Allocations and frees
// are ordered on the stream of the entry point in progress (StreamScope), so releasing a
// temporary never synchronises the device.
struct StreamScope {
  cudaStream_t prev;
  explicit StreamScope(cudaStream_t s);
  ~StreamScope();
};
int pool_alloc(void** p, size_t bytes);
void pool_free(void* p);
// true when buffers freed now are ordered on stream s (s is the stream of the entry point in progress)
bool allocations_ordered_on(cudaStream_t s);

// Owning device buffer; the hierarchy keeps these alive.
template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  void release() {
    if (p) pool_free(p);
    p = nullptr;
    n = 0;
  }
  int alloc(size_t count) {
    release();
    n = count;
    if (count == 0) return AMGC_OK;
    void* q = nullptr;
    const int st = pool_alloc(&q, count * sizeof(T));
    if (st != AMGC_OK) {
      n = 0;
      return st;
    }
    p = static_cast<T*>(q);
    return AMGC_OK;
  }
  size_t bytes() const { return n * sizeof(T); }
};

// Block-sparse row matrix on the device (row-major br x bc blocks).
struct DBsr {
  int nbr = 0, nbc = 0, br = 0, bc = 0;
  int64_t nnzb = 0;
  DBuf<int> rowptr, col;
  DBuf<double> val;
};

// SELL-32 copy of a BSR matrix for the thread-per-row apply: rows in slices of 32, each slice
// padded to its longest row; slot t of slice s holds the t-th block of its 32 rows, the block
// column at (off[s] + t) * 32 + lane and value k of the br x bc block at
// ((off[s] + t) * br * bc + k) * 32 + lane.  Padding blocks point at column 0 with zero values.
struct Sell {
  int br = 0, bc = 0;
  int nslice = 0;
  int64_t slots = 0;
  DBuf<int> off, len, col;
  DBuf<double> val;
  DBuf<int> perm;   // SELL position -> block row (rows sorted by length within windows); empty: identity
};

// FP32 mirrors of the cycle data of one level (values only; index arrays are shared).
struct LevelF32 {
  DBuf<float> K, B1, B2, P, R, Z, Ks, Ps, Rs, jdinv, atinv, pl_w;
  DBuf<float> x, b, r, t, dlam, ir_u;
};

// Non-owning views of one level's cycle data in storage type T.
template <class T>
struct BsrV {
  int nbr = 0, nbc = 0, br = 0, bc = 0;
  int64_t nnzb = 0;
  const int* rp = nullptr;
  const int* col = nullptr;
  const T* val = nullptr;
};
template <class T>
struct SellV {
  int br = 0, bc = 0, nslice = 0;
  const int* off = nullptr;
  const int* len = nullptr;
  const int* col = nullptr;
  const T* val = nullptr;
  const int* perm = nullptr;  // SELL position -> block row, null for the identity
  unsigned* ctr = nullptr;   // slice counter of the staged FP32 kernel (fine level), else null
  int* st = nullptr;         // status word for its bounded waits
  long long polls = -1;      // poll limit of those waits (< 0: the kernel's default)
};
template <class T>
struct LevelV {
  int nn = 0, bu = 3, nl = 0;
  int nu() const { return nn * bu; }
  int rows() const { return nn * bu + 3 * nl; }
  double omega_j = 0.0;
  BsrV<T> K, B1, B2, P, R;
  SellV<T> Ks, Ps, Rs;
  int kmap = -1, pmap = -1, rmap = -1;   // row mappings (see Level)
  int fuse = 0;                          // smoother form, resolved: 0, 1 or 2 (see Level)
  const int* ir_rows = nullptr;          // interface rows and B2's columns among them (see Level)
  const int* ir_b2c = nullptr;
  int n_ir = 0;
  T* ir_u = nullptr;
  const T* Z = nullptr;
  const double* Sinv = nullptr;    // FP64 in both precisions
  const T* dinv = nullptr;
  const T* atinv = nullptr;
  const T* pl_w = nullptr;
  const int* lagg = nullptr;
  const int* rl_ptr = nullptr;
  const int* rl_idx = nullptr;
  const int* b1_rows = nullptr;
  int n_b1_rows = 0;
  const double* Ainv = nullptr;    // coarsest level, FP64 in both precisions
  // batched coarsest level (null when not batched)
  const int* c_inst = nullptr;
  const int* c_loc = nullptr;
  const int* c_glob = nullptr;
  const int* c_goff = nullptr;
  const int64_t* c_doff = nullptr;
  // transposed cycle (FP64 only)
  BsrV<T> B1T, B2T;
  const T* ZT = nullptr;
  const double* SinvT = nullptr;
  const double* AinvT = nullptr;
  const int* b2t_rows = nullptr;
  int n_b2t_rows = 0;
  T* x = nullptr;
  T* b = nullptr;
  T* r = nullptr;
  T* t = nullptr;
  T* dlam = nullptr;
  T* tsw = nullptr;     // transposed sweep with several Jacobi steps: two work vectors of nu
};

// One level of the hierarchy.
struct Level {
  int nn = 0;     // displacement (super)nodes
  int bu = 3;     // DOFs per displacement node
  int nl = 0;     // multiplier nodes (3 DOFs each)
  int nu() const { return nn * bu; }
  int rows() const { return nn * bu + 3 * nl; }

  DBsr K, B1, B2;          // saddle blocks
  Sell Ks, Ps, Rs;         // SELL-32 copies of K, P, R (finest level; others when autotuned)
  // row mapping of the K, P, R applies per precision (0: FP64, 1: FP32):
  // 0 = warp per row, 1 = SELL one thread per row, 2 = SELL two threads per row, -1 = default
  int kmap[2] = {-1, -1}, pmap[2] = {-1, -1}, rmap[2] = {-1, -1};
  // smoother form per precision: 0 = the sweep's corrector and B1 update as two launches after the
  // Jacobi step, 1 = both in one single-CTA launch, 2 = split (the interface rows' Jacobi step,
  // the corrector and the B1 update beside the Jacobi step of the other rows), -1 = default (0);
  // the autotuner's choice where it ran
  int fuse[2] = {-1, -1};
  // interface rows: the displacement nodes with B1 entries or B2 columns, ascending; B2's block
  // columns as positions in that list; the split sweep's interface iterate (FP64 cycle)
  DBuf<int> ir_rows, ir_b2c;
  int n_ir = 0;
  DBuf<double> ir_u;
  DBuf<double> Z;          // nl*9
  DBuf<int> body;          // nn
  DBuf<double> B;          // nullspace nu*6
  DBuf<double> Bl;         // multiplier nullspace per node (nl)
  DBuf<int> lm_dnode;      // nl: displacement node coupled through D

  // transfer to the next level
  DBuf<int> agg;           // nn
  int n_agg = 0;
  DBuf<int> lagg;          // nl
  int n_lagg = 0;
  DBsr P, R;               // u prolongator (bu x 6) and restriction (6 x bu)
  DBuf<double> pl_w;       // nl weights of P-hat^lambda
  DBuf<int> rl_ptr, rl_idx;  // coarse multiplier node -> sorted member list

  // CheapSIMPLE data
  double lam_max = 0.0, omega_j = 0.0;
  // lambda_max power iteration running on the auxiliary stream (single-instance levels): its
  // buffers, and the event that marks its end; joined before the smoothed prolongator
  DBuf<double> lmx_x, lmx_y, lmx_sc, lmx_part;
  cudaEvent_t lmx_done = nullptr;
  bool smoother_pending = false;
  DBuf<double> kdiag, dinv, atinv;  // nu: pointwise diagonal of K, its inverse, A~^-1
  DBuf<double> jdinv;               // nu: omega_J D^-1 (omega_J per instance when batched)
  std::vector<double> inst_lam_max; // per instance (batched hierarchies)
  std::vector<double> schur_rho;    // per instance: rho(S_bd^-1 S_hat) when schur_damping = 1
  DBuf<int> key_base;               // batched: first node of the node's instance (MIS-2 keys)
  DBuf<double> Sinv;         // nl*9
  DBuf<int> b1_rows;         // displacement nodes with B1 entries
  int n_b1_rows = 0;

  // coarsest level
  DBuf<double> Ainv;         // rows*rows (row-major); batched: one dense block per instance

  // instances of a batched hierarchy: displacement nodes [nptr[i], nptr[i+1]) and multiplier
  // nodes [lptr[i], lptr[i+1]) of every level belong to instance i
  std::vector<int> nptr, lptr;
  // batched coarsest level: row -> instance and local index, per-instance global row lists
  // (u rows then multiplier rows), dense block offsets
  DBuf<int> c_inst, c_loc, c_glob, c_goff;
  DBuf<int64_t> c_doff;

  // transposed-cycle data (adjoint solves): B1^T, B2^T, blockwise transposed Z and S^-1,
  // the transposed coarsest inverse, and the rows of B2^T with entries
  DBsr B1T, B2T;
  DBuf<double> ZT, SinvT, AinvT;
  DBuf<int> b2t_rows;
  int n_b2t_rows = 0;
  DBuf<double> tsw;          // 2 nu: work vectors of the transposed multi-step Jacobi predictor
  bool has_transposed = false;

  // interface data of the finest level, kept for active-set updates: D, M (CSR over slave rows),
  // slave and master node ids, triads
  DBuf<double> if_D, if_Mv, if_T;
  DBuf<int> if_Mrp, if_Mcol, if_Sl, if_Ms;
  DBuf<uint8_t> if_act;    // the current active set (one byte per slave node)
  // block smoothers other than CheapSIMPLE (Uzawa, Braess-Sarazin, SIMPLE with SGS):
  // Jones-Plassmann colouring of K's node graph, inverted nodal diagonal blocks of K, and the
  // assembled Schur approximation factored in place by block ILU(0) with its level schedules
  int ncolor = 0;
  DBuf<int> color, col_ptr, col_nodes;
  std::vector<int> h_col_ptr;       // host copy of col_ptr (launch sizes)
  DBuf<double> kdblk_inv;           // nn x bu x bu
  DBsr S;                           // Schur approximation -> ILU(0) factors (L unit-lower, U)
  DBuf<int> s_diag;                 // position of each row's diagonal block in S
  DBuf<double> s_uinv;              // inverted diagonal blocks of U
  int s_nlev_l = 0, s_nlev_u = 0;
  DBuf<int> s_lptr, s_lrows, s_uptr, s_urows;   // rows of S by forward / backward level
  DBuf<double> bs_w, bs_d;          // work vectors (nu) of the block smoothers
  DBuf<double> bs_l, bs_m;          // work vectors (3 nl)
  // tentative multiplier transfer to the next level and its transpose (BSR, 3x3 diagonal blocks),
  // kept for the coarse constraint blocks of an active-set update
  DBsr Pl, Rl;

  // work vectors [u; lambda]
  DBuf<double> x, b, r, t;
  DBuf<double> dlam;         // nl*3

  LevelF32 f;                // FP32 cycle data (precision 32)
};

}  // namespace amgc

struct amgc_hierarchy {
  std::vector<amgc::Level> L;
  amgc_options opts{};
  amgc_stats_t stats{};
  cudaStream_t stream = nullptr;
  amgc::DBuf<int> status;          // device status word
  amgc::DBuf<double> scratch;      // reductions
  // FGMRES workspace
  int m_alloc = 0;
  amgc::DBuf<double> V, Zs, H, givens, gvec, y, wk, xk, rk;
  amgc::DBuf<float> Vf;             // FP32 copy of the Arnoldi basis (first projection pass)
  amgc::DBuf<unsigned> tma_ctr;    // slice counter of the staged FP32 fine-level apply
  long long wait_polls = -1;       // poll limit of the bounded device waits (< 0: kernel default)
  amgc::DBuf<double> partial;      // per-block partial dot products
  std::vector<amgc::LevelV<double>> v64;   // cycle views, FP64
  std::vector<amgc::LevelV<float>> v32;    // cycle views, FP32 (precision 32)
  bool transposed = false;                 // FGMRES/cycle act on A^T (adjoint solve)
  int n_inst = 1;                          // instances of a batched hierarchy
  // CUDA graphs of the forward V-cycle core (index 0: FP64, 1: FP32), captured on first use
  cudaGraphExec_t cycle_graph[2] = {nullptr, nullptr};
  long long cycle_graph_kernels[2] = {0, 0};
  cudaStream_t capture_stream = nullptr;
  cudaStream_t aux_stream = nullptr;    // setup work overlapped with the main stream
  cudaStream_t side_stream = nullptr;   // short multiplier-row kernels beside the long ones
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  amgc::DBuf<double> cyc_in, cyc_out;      // fixed FP64 input/output of the captured FP64 cycle
  // batched FGMRES workspace
  amgc::McState* mc = nullptr;     // multi-column cycle buffers (created on first use)
  amgc::DBuf<int> b_chunk_row0, b_chunk_row1, b_chunk_ptr, b_chunk_inst, b_row_inst;
  int b_nchunk = 0;
  double* h_pinned = nullptr;      // pinned host scalars
  // level smoother: 0 CheapSIMPLE, 1 Uzawa, 2 Braess-Sarazin, 3 SIMPLE with an SGS predictor
  int smoother_kind = 0;
  double block_omega = 0.7;        // the block smoother's damping omega
  int sgs_sweeps = 1;
  double sgs_omega = 0.7;
  // preconditioner of amgc_vcycle / amgc_solve: 0 the fully coupled V-cycle, 1 nested multigrid
  // (outer SIMPLE sweeps with a single-field AMG V-cycle on K and the exact Schur complement)
  int prec_kind = 0;
  int nest_sweeps = 1;
  double nest_omega = 0.8;
  amgc::DBuf<double> nest_Kinv;     // dense inverse of the coarsest level's K
  amgc::DBuf<double> nest_Sinv;     // dense inverse of S_hat = Z + B2 A~^-1 B1 (finest level)
  struct NestBufs {
    amgc::DBuf<double> x, b, r, t;
  };
  std::vector<NestBufs> nest;        // per-level work vectors of the K V-cycle
  // event timing of the fine-level K applies (amgc_profile)
  int prof = 0;                    // mask: 1 FP64 applies, 2 FP32 applies
  std::vector<cudaEvent_t> prof_ev;
  int prof_pending = 0;
  double prof_ms = 0.0, prof_bytes = 0.0, prof_flops = 0.0;
  int64_t prof_launches = 0;
};

namespace amgc {

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// FP64 -> FP32, rounded to nearest even, on the integer pipe for results in FP32's normal range
// (GB300 issues the FP64 -> FP32 conversion instruction at a small fraction of its integer
// rate).  The sign is kept, the exponent rebiased (1023 -> 127), the 52-bit fraction cut to 23
// bits and rounded on the 29 dropped bits, a carry running into the exponent (to infinity above
// FP32's largest value, as the conversion does).  Inputs whose FP32 result is zero, subnormal,
// infinite or NaN outside that path take the conversion instruction.
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned int hi = static_cast<unsigned int>(b >> 32);
  const int e = static_cast<int>((hi >> 20) & 0x7ffu);   // biased FP64 exponent
  if (e < 897 || e > 1150) {                              // outside FP32's normal exponents
    if ((b << 1) == 0ULL) return __uint_as_float(hi & 0x80000000u);   // signed zero
    return static_cast<float>(x);
  }
  const unsigned int keep = static_cast<unsigned int>((b >> 29) & 0x7fffffu);
  const unsigned int rest = static_cast<unsigned int>(b & 0x1fffffffu);
  unsigned int f = (static_cast<unsigned int>(e - 896) << 23) | keep;
  if (rest > 0x10000000u || (rest == 0x10000000u && (keep & 1u))) f += 1u;
  return __uint_as_float((hi & 0x80000000u) | f);
}

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// MurmurHash3's 32-bit finaliser (A. Appleby): the hash of the node priorities
// fmix32(i ^ seed) * 2^32 + i of the MIS-2 aggregation and of the Jones-Plassmann colouring.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

// ------------------------------------------------------------------ host-side kernel drivers
// scan.cu
int exclusive_scan(const int* in, int* out, int n, cudaStream_t s, int* total_host);
// assembly / setup (setup.cu)
int build_fine_level(amgc_hierarchy* h, const amgc_bsr* K, const double* D, const amgc_csr* M,
                     const int* slave_node, const int* master_node, const double* triad,
                     const uint8_t* active, const int* body_id, const double* nullspace);
int coarsen_level(amgc_hierarchy* h, int l);
int smoother_setup(amgc_hierarchy* h, int l);
int build_sell(amgc_hierarchy* h, int l);
int build_sell_of(amgc_hierarchy* h, const DBsr& A, Sell& S);
int autotune(amgc_hierarchy* h);
int coarse_setup(amgc_hierarchy* h, int l);
// block SpGEMM C = A B (BSR, sorted block columns; sym: C symmetric, formed on and above the diagonal)
int spgemm(amgc_hierarchy* h, const DBsr& A, const DBsr& B, DBsr& C, bool sym = false);
// ptr / idx: the indices i < n grouped by bucket[i] (in [0, nb); < 0 skipped), ascending in each
int bucket_lists(int n, const int* bucket, int nb, DBuf<int>& ptr, DBuf<int>& idx, cudaStream_t s);
int check_status(amgc_hierarchy* h, const char* where);
int transposed_setup(amgc_hierarchy* h);
// new active set of the slave nodes (device or host bytes, n_s of them): rebuilds the constraint
// blocks B2 and Z on every level, the Schur-block inverses (and their damping), the coarsest
// inverse and the views; keeps aggregates, transfers, lambda_max, coarse K and B1
int update_active_set(amgc_hierarchy* h, const uint8_t* active);
// setup phase timer: synchronises the stream and adds the elapsed wall time to a phase
struct PhaseTimer {
  amgc_hierarchy* h;
  int phase;
  double t0;
  PhaseTimer(amgc_hierarchy* hh, int ph);
  ~PhaseTimer();
};
double now_ms();

// kernel timing (api.cu)
int prof_begin(amgc_hierarchy* h, int kind);
int prof_end(amgc_hierarchy* h, int kind, double bytes, double flops);
int prof_flush(amgc_hierarchy* h);
// sparse kernels (cycle.cu)
int bsr_spmv(const DBsr& A, const double* x, double* y, double alpha, double beta, cudaStream_t s);
int lambda_max_estimate(amgc_hierarchy* h, Level& L, double* out);
int convert_f64_f32(int64_t n, const double* x, float* y, cudaStream_t s);
int lambda_max_start(amgc_hierarchy* h, Level& L);
int lambda_max_finish(amgc_hierarchy* h, Level& L, double* out);
int smoother_finish(amgc_hierarchy* h, int l);
int lambda_max_instances(amgc_hierarchy* h, Level& L, std::vector<double>& lam);
int schur_damping_setup(amgc_hierarchy* h, Level& L);
int dot(amgc_hierarchy* h, int64_t n, const double* a, const double* b, const double* wgt, double* out_dev);
// V-cycle (cycle.cu)
int make_views(amgc_hierarchy* h);
int precond_apply(amgc_hierarchy* h, const double* r, double* z);   // one V-cycle, FP64 in/out
bool staged_apply_in_use(const amgc_hierarchy* h);   // the FP32 cycle's fine K runs the staged kernel
void drop_cycle_graphs(amgc_hierarchy* h);            // forget captured cycles (their launches changed)
int set_row_mapping(amgc_hierarchy* h, int level, int matrix, int precision, int mapping);
int set_wait_limit(amgc_hierarchy* h, long long polls);
int nested_setup(amgc_hierarchy* h);   // dense K_c and S_hat inverses, work vectors (prec_kind 1)
// colouring, diagonal-block inverses and Schur ILU(0) of every smoothed level (smoother_kind != 0);
// schur_only: the Schur part alone (after an active-set change)
int block_smoother_setup(amgc_hierarchy* h, bool schur_only);
int dense_inverse(amgc_hierarchy* h, double* A, int n);   // in place, Gauss-Jordan (setup.cu)
int saddle_apply(amgc_hierarchy* h, int l, const double* x, double* y);
// FGMRES (krylov.cu)
int fgmres(amgc_hierarchy* h, const double* rhs, double* x, double tol, int* iters, double* relres);
// batched problems (batch.cu)
int fgmres_batched(amgc_hierarchy* h, int nrhs, const double* rhs, double* x, int* iters, double* relres);
// kMcCols columns at once (column stride rows[0], FP64 in and out): V-cycle, saddle apply
// (batch_cycle.cu); rows of instances q with live[q] == 0 are skipped when live (device) is given
int precond_apply_cols(amgc_hierarchy* h, const double* r, double* z, const int* live);
int saddle_apply_cols(amgc_hierarchy* h, const double* x, double* y, const int* live);
void mc_state_free(McState* st);
// gradients (grad.cu)
int grad_scatter(amgc_hierarchy* h, const double* adj, const double* x, double* gK, double* gB1, double* gB2);
// the element-gradient kernels with caller-provided scratch `lift` (3 ne doubles, used when gt != 0),
// enqueued on s without synchronising
int launch_grad_elements(int ne, const int* conn, const int* shape, const double* Khat, const int* node_free,
                         const double* adj, const double* x, const double* uD, const uint8_t* lift_mask,
                         const double* E, double* gE, double* gt, double* lift, cudaStream_t s);
int grad_elements(int ne, const int* conn, const int* shape, const double* Khat, const int* node_free,
                  const double* adj, const double* x, const double* uD, const uint8_t* lift_mask, const double* E,
                  double* gE, double* gt, cudaStream_t s);

}  // namespace amgc
