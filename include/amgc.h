/*
 * amgc -- fully coupled block algebraic multigrid for mortar-contact saddle-point systems
 * on one NVIDIA GB300 (sm_103a).
 *
 * The linear system is the linearised frictionless contact system of Sec. 2.3
 * (Eq. ch6_finalsaddlepointsystem, compact form Eq. ch6_finalsaddlepointsystem_comprehensive):
 *
 *        [ K   B1 ] [ u      ]   [ f ]
 *        [ B2  -Z ] [ lambda ] = [ g ]
 *
 * K: stiffness block in 3x3 nodal blocks; B1 = C1^T carries D^T (slave rows) and -M^T
 * (master rows); B2 = C2 carries the linearised weighted gap n^T(D u_s - M u_m) for active
 * slave nodes; -Z carries the frictionless tangential rows (active) or the identity (inactive).
 * Multipliers are Cartesian, three per slave interface node.
 *
 * The preconditioner is the paper's method: segregated aggregation with multiplier aggregates
 * derived from the slave displacement aggregates through D (Sec. 4, Algorithm 1), plain or
 * smoothed aggregation transfers (Sec. 3.1.2, Eq. ProlongatorSmoothing, Eq.
 * ch6_segregatedtransfers), Galerkin coarse operators, CheapSIMPLE level smoothing (Algorithm 4,
 * Sec. 5.2) in a V-cycle (Fig. mgalgorithm) with a direct coarsest solve, inside flexible GMRES
 * (Sec. 3; stopping rule Eq. ch7_linearstoppingcriterion).
 *
 * Conventions for every call:
 *  - Return value: AMGC_OK (0) or a negative AMGC_E* code; amgc_strerror() names it and
 *    amgc_last_error() gives the detail of the last failure in the calling thread.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default stream).  Every call
 *    orders its device work on that stream; calls that return host-visible results
 *    (sizes, iteration counts) synchronise that stream before returning.
 *  - Index arrays are int32, floating-point arrays are IEEE double unless stated.
 *  - Input pointers to amgc_setup may be host or device memory (unified addressing decides);
 *    they are copied and may be freed after the call.  Vector arguments of the apply calls are
 *    DEVICE pointers unless the call says otherwise.
 *  - The hierarchy is owned by the library until amgc_destroy().  A failed amgc_setup leaves
 *    *out == NULL and frees everything it allocated.
 *  - The library keeps per-device state for the life of the process (its memory pool, the device
 *    address of a static scratch array).  After cudaDeviceReset on a device that state is stale:
 *    do not call the library on that device again in the same process.
 */
#ifndef AMGC_H
#define AMGC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  AMGC_OK = 0,
  AMGC_EINVAL = -1,          /* malformed argument or input structure                         */
  AMGC_ESINGULAR = -2,       /* singular nodal block, rank-deficient aggregate or coarse pivot  */
  AMGC_NOT_CONVERGED = -3,   /* FGMRES reached maxit without meeting the tolerance              */
  AMGC_BREAKDOWN = -4,       /* non-finite value or Arnoldi breakdown                           */
  AMGC_TIMEOUT = -5,         /* a bounded device wait expired                                   */
  AMGC_ECUDA = -6,           /* CUDA runtime error                                              */
  AMGC_ENOMEM = -7           /* device allocation failed                                        */
};

/* Opaque hierarchy handle (library-owned; see amgc_setup / amgc_destroy). */
struct amgc_hierarchy;

/* Block-sparse row matrix: n_brow x n_bcol blocks of br x bc, row-major blocks,
 * rowptr[n_brow+1], col[nnzb] sorted ascending within each row, val[nnzb*br*bc]. */
typedef struct {
  int32_t n_brow, n_bcol, br, bc;
  const int32_t* rowptr;
  const int32_t* col;
  const double* val;
} amgc_bsr;

/* Scalar CSR matrix n_row x n_col (used for the mortar matrix M, slave x master). */
typedef struct {
  int32_t n_row, n_col;
  const int32_t* rowptr;
  const int32_t* col;
  const double* val;
} amgc_csr;

typedef struct {
  int32_t levels_max;        /* maximum number of levels (>= 1)                               */
  int32_t coarse_max_rows;   /* stop coarsening once the saddle system has fewer rows           */
  int32_t transfer;          /* 0 = plain aggregation (PA), 1 = smoothed aggregation for u (SA) */
  int32_t smoother_sweeps;   /* CheapSIMPLE sweeps, pre and post (>= 0)                        */
  int32_t jacobi_sweeps;     /* damped-Jacobi sweeps in the predictor (>= 1)                   */
  int32_t simplec;           /* 0: A~ = diag(K);  1: A~ = absolute row sums (SIMPLEC)          */
  int32_t precision;         /* 64: FP64 V-cycle; 32: FP32 storage and arithmetic in the cycle  */
  int32_t fgmres_restart;    /* Krylov subspace size m (1..256)                               */
  int32_t fgmres_maxit;      /* total FGMRES iterations allowed                                */
  uint32_t seed;             /* MIS-2 priority seed                                           */
  double sa_omega;           /* SA damping numerator: omega = sa_omega / lambda_max(D^-1 K)    */
  double jacobi_omega;       /* <= 0: (4/3) / lambda_max(D^-1 K) per level                     */
  double simple_alpha;       /* SIMPLE damping alpha of the multiplier correction              */
  double tol;                /* relative residual tolerance ||r_k|| / ||r_0||                  */
  int32_t autotune;          /* 1: time the row mappings of every level's K, P and R apply at
                                setup and keep the fastest (warp per row, SELL with one or two
                                threads per row), and the smoother fusion of every level (the
                                sweep's corrector and B1 update as two launches or one fused
                                single-CTA launch), separately for the FP64 and FP32 cycle  */
  int32_t schur_damping;     /* 0: the multiplier correction is damped by simple_alpha alone
                                (Sec. 5.2).  1: per level (per instance when batched) it is
                                damped by min(simple_alpha, (4/3) / rho), rho = spectral radius
                                of S_bd^-1 S_hat estimated by 30 power steps, which keeps the
                                block-diagonal Schur step a contraction where a slave mesh much
                                finer than its master couples many slave nodes through one
                                master node (rho >> 2)                                       */
  int32_t coarse_solver;     /* 0: explicit dense inverse of the merged coarsest matrix (the role
                                of the paper's LU, Sec. 6.2).  1: the level smoother's sweeps from
                                a zero guess on the coarsest level instead, with no merged matrix
                                (the alternative compared in Sec. 6.2; no dense-size limit).
                                Single hierarchies only; not with the transposed entry points */
} amgc_options;

typedef struct {
  int32_t n_levels;
  int32_t rows[16];          /* saddle rows per level                                          */
  int32_t disp_nodes[16];    /* displacement (super)nodes per level                            */
  int32_t lm_nodes[16];      /* multiplier nodes per level                                     */
  int32_t dofs_per_node[16]; /* 3 on level 0, 6 below                                          */
  int64_t nnz[16];           /* scalar nonzeros of the level's saddle matrix                   */
  double operator_complexity;
  double lambda_max[16];     /* estimate of lambda_max(D_K^-1 K) per level                     */
  double setup_ms;           /* wall time of the last amgc_setup                               */
  int32_t last_iters;        /* FGMRES iterations of the last solve                            */
  double last_relres;        /* true relative residual at the end of the last solve           */
  /* wall time of the setup phases, summed over levels (ms): 0 input copy and assembly,
   * 1 aggregation (MIS-2), 2 multiplier aggregation, 3 tentative transfers (QR),
   * 4 smoother data and lambda_max, 5 smoothed prolongator, 6 transpose, 7 Galerkin products,
   * 8 coarsest inverse, 9 fine-level SELL copies and views */
  double setup_phase_ms[10];
} amgc_stats_t;

/* Fills the defaults: levels_max 10, coarse_max_rows 5000, SA, 1 sweep, 1 Jacobi sweep,
 * SIMPLE (diag K), FP64, restart 50, maxit 1000, seed 0x5EED, sa_omega 4/3, jacobi_omega
 * automatic, alpha 0.8, tol 1e-8 (Sec. 6.2 settings, Eq. ch7_linearstoppingcriterion), autotune 0,
 * schur_damping 0, coarse_solver 0. */
void amgc_default_options(amgc_options* opts);

/* Builds the hierarchy (Sec. 4: segregated aggregation with Algorithm 1, transfers of
 * Sec. 3.1.2 / Eq. ch6_segregatedtransfers, Galerkin products, CheapSIMPLE data, coarsest
 * dense factorisation).
 *   K           n x n nodal 3x3 BSR, Dirichlet nodes already eliminated; every row must hold
 *               its diagonal block.
 *   D_diag      n_s diagonal entries of the dual-mortar D (slave node j <-> multiplier node j).
 *   M           n_s x n_m scalar CSR mortar matrix (slave rows, master columns); n_s >= 1:
 *               a system without a contact interface has no multiplier block and is refused
 *               (AMGC_EINVAL); every instance of a batch needs at least one slave node too.
 *   slave_node  n_s   K block row of slave interface node j.
 *   master_node n_m   K block row of master interface node l.
 *   triad       n_s x 3 x 3, rows (n, tau_xi, tau_eta) of each slave node, orthonormal.
 *   active      n_s   1 = active (normal gap row + tangential rows), 0 = inactive (lambda = 0).
 *   body_id     n     body of each K block row; couplings between bodies are dropped during
 *               aggregation (Sec. 4.2).
 *   nullspace   3n x 6 row-major rigid-body modes (t_x, t_y, t_z, r_x, r_y, r_z).
 * Errors: AMGC_EINVAL (sizes, indices out of range, missing diagonal block, nothing to
 * aggregate), AMGC_ESINGULAR (rank-deficient aggregate, singular Schur block or coarse pivot),
 * AMGC_ENOMEM, AMGC_ECUDA.  On error *out is NULL and nothing stays allocated. */
int amgc_setup(const amgc_bsr* K, const double* D_diag, const amgc_csr* M,
               const int32_t* slave_node, const int32_t* master_node,
               const double* triad, const uint8_t* active, const int32_t* body_id,
               const double* nullspace, const amgc_options* opts, void* stream,
               struct amgc_hierarchy** out);

/* Batched problems: n_inst independent contact systems concatenated block-diagonally in the
 * arrays of amgc_setup (instance q owns K block rows [node_ptr[q], node_ptr[q+1]) and slave /
 * multiplier nodes [lm_ptr[q], lm_ptr[q+1]); no coupling between instances; body_id must
 * separate the bodies of every instance).  One hierarchy serves all instances: MIS-2 keys use
 * instance-local node indices, lambda_max and the dampings are computed per instance, the
 * coarsest level is inverted per instance, and coarsening stops when the largest instance has
 * fewer than coarse_max_rows rows (or at levels_max).  Every instance therefore gets the
 * aggregates and transfers it would get alone.  node_ptr, lm_ptr: host arrays of n_inst + 1.
 * Other arguments, ownership and errors as amgc_setup. */
int amgc_setup_batched(const amgc_bsr* K, const double* D_diag, const amgc_csr* M,
                       const int32_t* slave_node, const int32_t* master_node,
                       const double* triad, const uint8_t* active, const int32_t* body_id,
                       const double* nullspace, int32_t n_inst, const int32_t* node_ptr, const int32_t* lm_ptr,
                       const amgc_options* opts, void* stream, struct amgc_hierarchy** out);

/* Solves the n_inst x nrhs independent systems of a batched hierarchy by FGMRES in lockstep,
 * one Krylov space, stopping test and iteration count per (instance, rhs) system.  rhs, x:
 * device arrays of nrhs columns of length rows[0] (column-major).  iters, relres: host arrays of
 * n_inst * nrhs entries, system q * nrhs + r (may be NULL).  Returns AMGC_NOT_CONVERGED when a
 * system reached fgmres_maxit. */
int amgc_solve_batched(struct amgc_hierarchy* h, int32_t nrhs, const double* rhs, double* x, int32_t* iters,
                       double* relres, void* stream);

/* z = V-cycle(r) with zero initial guess (Fig. mgalgorithm).  r, z: device vectors of
 * length rows[0] = 3n + 3 n_s, ordered [u; lambda].  r and z must not overlap.  With
 * precision 32 the cycle runs on FP32 copies of the level data (the inverted Schur blocks and
 * the coarsest inverse stay FP64); r and z are still FP64. */
int amgc_vcycle(struct amgc_hierarchy* h, const double* r, double* z, void* stream);

/* y = A x with the fine-level saddle operator [K B1; B2 -Z]; device vectors of length rows[0]. */
int amgc_apply(struct amgc_hierarchy* h, const double* x, double* y, void* stream);

/* Solves A x = rhs by right-preconditioned flexible GMRES with one V-cycle per iteration,
 * x_0 = 0, stopped when ||b - A x_k|| / ||b|| < tol (Eq. ch7_linearstoppingcriterion).
 * Arnoldi: classical Gram-Schmidt with re-orthogonalisation; the first projection's
 * coefficients come from FP32 copies of the basis, the updates and the second projection are
 * FP64, so the Hessenberg matrix and the Arnoldi relation hold to FP64 rounding.
 * rhs, x: device vectors of length rows[0]; iters / relres may be NULL.  Returns
 * AMGC_NOT_CONVERGED (x holds the last iterate) or AMGC_BREAKDOWN on failure. */
int amgc_solve(struct amgc_hierarchy* h, const double* rhs, double* x, int32_t* iters,
               double* relres, void* stream);

/* amgc_solve with the solution split into its two fields: u (3n displacements) and lam (3 n_s
 * Cartesian multipliers, three per slave node), the form (u, lambda) of the problem statement
 * (Sec. 2.3).  rhs: device vector of rows[0]; u, lam: host or device arrays (unified addressing
 * decides), not overlapping rhs.  Synchronises `stream`.  Results and errors as amgc_solve. */
int amgc_solve_split(struct amgc_hierarchy* h, const double* rhs, double* u, double* lam, int32_t* iters,
                     double* relres, void* stream);

/* Same as amgc_solve but rhs and x are HOST arrays: the call copies rhs to the device,
 * solves, and copies x back (synchronous with respect to the host). */
int amgc_solve_host(struct amgc_hierarchy* h, const double* rhs_host, double* x_host,
                    int32_t* iters, double* relres, void* stream);

/* Chooses the level smoother of the V-cycle (Sec. 5.1 block smoothers in the cheap forms of Sec. 5.2,
 * with the inner solvers of the paper's experiments, Sec. 6.1):
 *   kind 0: CheapSIMPLE (the default; Algorithm 4 with damped Jacobi and the nodal Schur blocks);
 *   kind 1: Uzawa (Algorithm 2):  du = SGS(K, f - K u - B1 lam) from 0,
 *           dlam = -ILU(S)^-1 (g - B2 u + Z lam - B2 du),  u += omega du,  lam += omega dlam;
 *   kind 2: Braess-Sarazin (Algorithm 3):  u_h = u + A~^-1 (f - K u - B1 lam) / omega,
 *           dlam = -ILU(S_w)^-1 (g + Z lam - B2 u_h),  lam += dlam,  u = u_h - A~^-1 B1 dlam / omega;
 *   kind 3: SIMPLE (Algorithm 4; SIMPLEC with opts.simplec):  u_h = SGS(K, f - B1 lam) from u,
 *           dlam = -ILU(S)^-1 (g + Z lam - B2 u_h),  lam += omega dlam,  u = u_h - omega A~^-1 B1 dlam;
 * with S = Z + B2 A~^-1 B1, S_w = Z + B2 A~^-1 B1 / omega assembled on the nodal 3x3 multiplier
 * blocks and factored by block ILU(0) (no fill; rows eliminated in natural order), and SGS =
 * sgs_sweeps damped (sgs_omega) symmetric Gauss-Seidel sweeps over the nodal blocks of K in the order
 * of a Jones-Plassmann colouring of K's node graph (colours ascending, then descending; priorities
 * fmix32(i ^ seed) * 2^32 + i as in the aggregation).  smoother_sweeps of the options sweeps run
 * pre and post.  The call builds, on every smoothed level, the colouring, the inverted diagonal
 * blocks of K and the ILU(0) factors (level-scheduled), drops the captured V-cycle graphs and
 * synchronises `stream`; amgc_update_active_set and amgc_pdass refactor the Schur part.  Kinds 1-3
 * need a single FP64 hierarchy; the transposed calls refuse them.  The ILU(0) substitutions run
 * level by level in one thread block, so these smoothers are for comparisons, not for speed.
 * Errors: AMGC_EINVAL (kind, omega <= 0, sgs_sweeps < 1, sgs_omega <= 0, batched or FP32
 * hierarchy), AMGC_ESINGULAR (singular diagonal block or ILU pivot), AMGC_ENOMEM, AMGC_ECUDA. */
int amgc_set_smoother(struct amgc_hierarchy* h, int32_t kind, double omega, int32_t sgs_sweeps, double sgs_omega,
                      void* stream);

/* Chooses the preconditioner that amgc_vcycle applies and amgc_solve / amgc_pdass use:
 *   kind 0: the fully coupled block AMG V-cycle (the paper's method; the default);
 *   kind 1: nested multigrid, the comparison approach of Sec. 3.2 (Fig. mgmphmodelsA): the
 *     coupling is treated on the finest level only, by `outer_sweeps` SIMPLE sweeps (Algorithm 4)
 *       u_h = u + V_K (f - K u - B1 lambda)
 *       dlambda = -S_hat^-1 (g + Z lambda - B2 u_h),  S_hat = Z + B2 A~^-1 B1 (exact, dense)
 *       lambda += omega dlambda,  u = u_h - omega A~^-1 B1 dlambda
 *     whose predictor V_K is one single-field AMG V-cycle on K: the displacement part of this
 *     hierarchy (its aggregates, transfers and Galerkin K_c), damped Jacobi with omega_J
 *     (smoother_sweeps pre and post), and the coarsest K_c by its dense inverse.
 * The first switch to kind 1 forms the dense inverses of the coarsest K_c and of S_hat (each at
 * most 16384 rows) and synchronises `stream`; amgc_update_active_set and amgc_pdass form S_hat
 * again.  Kind 1 needs a single FP64 hierarchy (precision 64, not batched); the transposed
 * calls keep the coupled cycle and refuse kind 1.  Errors: AMGC_EINVAL (kind, outer_sweeps < 1,
 * omega <= 0, batched or FP32 hierarchy, a dense size above the limit), AMGC_ESINGULAR,
 * AMGC_ENOMEM, AMGC_ECUDA. */
int amgc_set_preconditioner(struct amgc_hierarchy* h, int32_t kind, int32_t outer_sweeps, double omega, void* stream);

/* Replaces the hierarchy's active set (setup reuse across active-set changes, as in the Newton
 * steps of the paper's contact simulations, Sec. 6.3-6.4).  Only the constraint blocks depend on
 * the active set: B2 (the weighted-gap rows of active nodes) and Z (tangential rows of active
 * nodes, the identity of inactive ones).  The call forms B2 and Z anew on the finest level from
 * the interface data given to amgc_setup, the coarse B2_c = R^lambda B2 P and Z_c with the kept
 * transfers, the inverted nodal Schur blocks (and their damping), and the coarsest inverse (or the
 * coarsest smoother data); it keeps the aggregates, multiplier aggregates, transfers, lambda_max,
 * Jacobi data, coarse K and coarse B1, which the active set does not change (Sec. 4 aggregates
 * the displacement graph and derives the multiplier aggregates through D, not through B2).  The
 * result equals a fresh amgc_setup with the new set and the old aggregates.
 * active: n_s bytes (1 active, 0 inactive), host or device.  Single hierarchies only.  Drops the
 * captured V-cycle graphs and the transposed data (formed again when next needed).  Synchronises
 * `stream`.  Errors: AMGC_EINVAL (NULL argument, batched hierarchy), AMGC_ESINGULAR (singular Schur
 * block or coarse pivot), AMGC_ENOMEM, AMGC_ECUDA. */
int amgc_update_active_set(struct amgc_hierarchy* h, const uint8_t* active, void* stream);

/* Primal-dual active set strategy (PDASS, Sec. 2.2) for frictionless contact with an initial
 * normal gap: from the hierarchy's current active set, solves the saddle system of the set with
 * FGMRES (amgc_solve's method and tolerance), right-hand side f on the displacement rows and, on an
 * active node's normal row, D_jj g0_j (zero on every other multiplier row); then takes as next set
 *     active_j  <=>  lambda_n,j - c g_j(u) > 0,   lambda_n,j = n_j . lambda_j,
 *     g_j(u) = D_jj g0_j - n_j^T (D_jj u_s,j - sum_l M_jl u_m,l)   (weighted gap, Eq. ch4_discretenormalcontact),
 * with n_j the first row of node j's triad, and updates the hierarchy as amgc_update_active_set
 * does; it stops when a solve leaves the set unchanged (the contact conditions then hold at the
 * solve's accuracy).
 *   f: device, 3n displacement right-hand side; g0: device, n_s initial normal gaps; c > 0 the
 *   complementarity parameter; max_steps >= 1 solves at most; x: device, rows[0]: the last solve's
 *   solution [u; lambda].  active_out: host (or device) n_s bytes for the final set, or NULL;
 *   steps: solves run; total_iters: FGMRES iterations over all solves (both may be NULL).
 * Returns AMGC_NOT_CONVERGED if a solve failed to converge or the set still changed after
 * max_steps solves (x and the hierarchy then hold the last step's), AMGC_EINVAL for bad
 * arguments or a batched hierarchy; other errors as amgc_solve and amgc_update_active_set. */
int amgc_pdass(struct amgc_hierarchy* h, const double* f, const double* g0, double c, int32_t max_steps, double* x,
               uint8_t* active_out, int32_t* steps, int32_t* total_iters, void* stream);

/* Adjoint calls (transposed system).  The first one builds, once, the transposed data of every
 * level (B1^T, B2^T, blockwise transposes of Z and of the Schur-block inverses, the transposed
 * coarsest inverse).  They run in FP64, with the coupled V-cycle and CheapSIMPLE smoothing
 * (AMGC_EINVAL after amgc_set_smoother or amgc_set_preconditioner chose another kind, for a
 * batched hierarchy, or with coarse_solver 1).
 *
 * amgc_apply_transposed:  y = A^T x.
 * amgc_vcycle_transposed: z = M^T r, M the V-cycle of amgc_vcycle.  Since K is symmetric, M^T
 *   is the V-cycle on A^T with each CheapSIMPLE sweep transposed (multiplier update
 *   w = -alpha S^-T (e_lambda - B1^T A~^-1 e_u) first, then u += J^T (e_u - B2^T w) with J the
 *   predictor's jacobi_sweeps damped Jacobi steps in residual form,
 *   J^T = sum_{i<jacobi_sweeps} omega D^-1 (I - omega K D^-1)^i), unchanged transfers and the
 *   transposed coarsest inverse, so <M x, y> = <x, M^T y>.
 * amgc_solve_transposed:  FGMRES on A^T x = rhs preconditioned by M^T, stopped at
 *   ||r_k|| / ||r_0|| < tol (tol <= 0: the setup tolerance).  Device vectors, as amgc_solve. */
int amgc_apply_transposed(struct amgc_hierarchy* h, const double* x, double* y, void* stream);
int amgc_vcycle_transposed(struct amgc_hierarchy* h, const double* r, double* z, void* stream);
int amgc_solve_transposed(struct amgc_hierarchy* h, const double* rhs, double* x, double tol, int32_t* iters,
                          double* relres, void* stream);

/* Outer-product scatter of the adjoint: for x = A^{-1} b and adj = A^{-T} (dJ/dx),
 * dJ/dK = -adj_u (x) x_u on every stored 3x3 block of the fine K (same order as the K given to
 * amgc_setup), dJ/dB1 = -adj_u (x) lambda on B1's blocks, dJ/dB2 = -adj_lambda (x) u on B2's
 * blocks, and dJ/db = adj.  gK: nnzb(K)*9 doubles; gB1, gB2: nnzb*9 doubles or NULL (block
 * counts from amgc_export).  All device pointers; adj, x of length rows[0]. */
int amgc_grad_scatter(struct amgc_hierarchy* h, const double* adj, const double* x, double* gK, double* gB1,
                      double* gB2, void* stream);

/* Element-level gradients for K = sum_e E_e Khat_e and the lifted right-hand side
 * f = -K_fD u_D:
 *   gE[e] = dJ/dE_e = -adj_e^T Khat_e u_e   (u_e: solution at free nodes, u_D at prescribed ones;
 *                                            adj_e: adjoint at free nodes, 0 at prescribed ones)
 *   gt[c] = dJ/dt_c for a uniform prescribed displacement t on the nodes flagged in lift_mask:
 *           -sum_e E_e sum_{flagged nodes a of e} (Khat_e adj_e)_(a,c)   (gt may be NULL)
 * conn: ne x 8 node ids (full numbering), shape: ne indices into Khat (n_shape x 24 x 24, unit
 * modulus, DOF order node-major), node_free: full node -> free node (K block row) or -1,
 * adj, x: length-rows[0] vectors, uD: n_all x 3 prescribed values, lift_mask: n_all bytes (or
 * NULL), E: ne moduli.  All device pointers.  The reduction into gt is deterministic. */
int amgc_grad_elements(int32_t ne, const int32_t* conn, const int32_t* shape, const double* Khat,
                       const int32_t* node_free, const double* adj, const double* x, const double* uD,
                       const uint8_t* lift_mask, const double* E, double* gE, double* gt, void* stream);

/* amgc_grad_elements without any device allocation, for callers that cannot allocate when
 * they need the gradients: code that owns all device memory up front (a framework's memory
 * pool with a hard cap leaves no room for the library's own allocations), or a latency-bound
 * loop that must stay out of the driver's allocator and its implicit synchronisation.  The
 * paper has no counterpart; this is a property of the library.
 * Same arguments and results as amgc_grad_elements, except that this call is asynchronous: it
 * only enqueues its two kernels on `stream` and returns (amgc_grad_elements waits for its stream
 * before it frees its scratch); read gE and gt after synchronising that stream.  With gt == NULL
 * no scratch is used at all, and ne == 0 returns at once.  Its scratch is one file-scope device
 * array of 3 x 262144 doubles (6 MiB) that every GPU loading the library holds until the
 * process exits: ne above 262144 is rejected with AMGC_EINVAL.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) with the device current, so make
 * that first call before any stream capture.  All calls share the array and each call
 * overwrites the part it reads, so calls that overlap on the GPU (different streams, no
 * ordering between them) race: order them. */
int amgc_grad_elements_noalloc(int32_t ne, const int32_t* conn, const int32_t* shape, const double* Khat,
                               const int32_t* node_free, const double* adj, const double* x, const double* uD,
                               const uint8_t* lift_mask, const double* E, double* gE, double* gt, void* stream);

/* Copies the hierarchy's summary (levels, sizes, operator complexity, lambda_max per level, setup
 * time and phase times, the last solve's iterations and residual) into *out.  Host only; no
 * device work.  Errors: AMGC_EINVAL (null argument). */
int amgc_stats(const struct amgc_hierarchy* h, amgc_stats_t* out);

/* Copies one internal array of level `level` to the host buffer dst (capacity `bytes`).
 * what: see AMGC_EXPORT_*.  Returns the number of bytes the array holds (>= 0) or an error;
 * with dst == NULL only the size is returned.  Used by the parity tests. */
enum {
  AMGC_EXPORT_AGG = 1,        /* int32[disp_nodes]   displacement aggregate of each node       */
  AMGC_EXPORT_LAGG = 2,       /* int32[lm_nodes]     multiplier aggregate of each node         */
  AMGC_EXPORT_P_ROWPTR = 3,   /* int32  prolongator (u) BSR of this level -> next             */
  AMGC_EXPORT_P_COL = 4,
  AMGC_EXPORT_P_VAL = 5,      /* double bu x 6 blocks                                          */
  AMGC_EXPORT_K_ROWPTR = 6,   /* K block of this level                                         */
  AMGC_EXPORT_K_COL = 7,
  AMGC_EXPORT_K_VAL = 8,
  AMGC_EXPORT_B1_ROWPTR = 9,
  AMGC_EXPORT_B1_COL = 10,
  AMGC_EXPORT_B1_VAL = 11,
  AMGC_EXPORT_B2_ROWPTR = 12,
  AMGC_EXPORT_B2_COL = 13,
  AMGC_EXPORT_B2_VAL = 14,
  AMGC_EXPORT_Z = 15,         /* double[lm_nodes*9]                                            */
  AMGC_EXPORT_SINV = 16,      /* double[lm_nodes*9]  inverted nodal blocks of S_hat            */
  AMGC_EXPORT_NULLSPACE = 17, /* double[dofs*6]                                                */
  AMGC_EXPORT_PL_W = 18,      /* double[lm_nodes]    multiplier tentative-transfer weights     */
  AMGC_EXPORT_ATINV = 19,     /* double[dofs]        A~^-1                                     */
  AMGC_EXPORT_OMEGA = 20,     /* double[2]           (lambda_max, omega_J)                     */
  AMGC_EXPORT_COARSE_INV = 21, /* double[rows*rows]  inverse of the coarsest saddle matrix
                                 (batched: the instances' inverses one after the other)   */
  AMGC_EXPORT_SCHUR_RHO = 22, /* double[instances]  rho of S_bd^-1 S_hat (schur_damping = 1;
                                 empty otherwise); SINV then holds the blocks already scaled
                                 by min(alpha, (4/3)/rho) / alpha                          */
  AMGC_EXPORT_COLOR = 23      /* int32[disp_nodes]  Jones-Plassmann colour of each node (block
                                 smoothers with SGS; empty otherwise)                      */
};
int64_t amgc_export(const struct amgc_hierarchy* h, int32_t level, int32_t what, void* dst,
                    int64_t bytes);

/* Diagnostic timing of the dominant kernel family: the fine-level K-block applies (residual,
 * Jacobi predictor and saddle apply, one launch each).  With enable != 0 every such launch is
 * bracketed by CUDA events recorded on the launching stream; amgc_profile_read synchronises
 * that stream and returns the accumulated device time (ms), the number of launches, the
 * algorithmic bytes those launches move (matrix values and indices once, every vector once) and
 * their algorithmic floating-point operations (two per stored matrix value).
 * enable is a mask: 1 times the FP64 applies, 2 the FP32 applies, 3 both, 0 stops timing.
 * Enabling resets the counters.  Not for production runs: each launch adds two event records. */
int amgc_profile(struct amgc_hierarchy* h, int32_t enable);
int amgc_profile_read(struct amgc_hierarchy* h, double* total_ms, int64_t* launches, double* bytes,
                      double* flops);

/* Overrides the row mapping of one sparse apply of the cycle, or the smoother fusion of a level (the
 * choices the setup-time autotuner makes when opts.autotune = 1).  level: 0 .. n_levels-1; matrix:
 * 0 = the level's K (with its B1 coupling), 1 = its prolongator P, 2 = its restriction R (P and R:
 * not on the coarsest level), 3 = the form of the CheapSIMPLE sweep's multiplier corrector and B1
 * update (mapping 0: two launches after the sweep's Jacobi step; 1: one fused launch of one thread
 * block, which the autotuner picks on levels with few multiplier rows, with the arithmetic of
 * form 0; 2: split, the interface rows (B1's rows and B2's columns) take the last Jacobi step of
 * the sweep, the corrector and the B1 update on a second stream beside the Jacobi step of the
 * other rows, equal to form 0 up to the summation order of the interface rows' K products; -1:
 * the default, form 0; the autotuner times the forms a level has and keeps the fastest);
 * precision: 64 = the FP64 views (the Krylov operator apply and the FP64 cycle), 32 = the FP32
 * cycle (hierarchies set up with precision 32 only); mapping: -1 = the default, 0 = one warp per
 * block row, 1 / 2 = SELL-32 with one / two threads per block row, 3 = the shared-memory staged
 * FP32 kernel with bounded waits (level 0, K, precision 32 only).  Builds the SELL copy of the
 * matrix if it has none and drops the captured V-cycle graphs (recaptured on the next cycle).
 * Synchronises the hierarchy's last stream.  Errors: AMGC_EINVAL (argument out of range, or a
 * mapping the matrix has no form for), AMGC_ENOMEM, AMGC_ECUDA.  (Library mechanics; the paper
 * has no counterpart.) */
int amgc_set_row_mapping(struct amgc_hierarchy* h, int32_t level, int32_t matrix, int32_t precision,
                         int32_t mapping);

/* Sets how many times each bounded device wait of the hierarchy's kernels (the mbarrier waits of
 * the staged FP32 apply) tests its barrier before giving up: polls < 0 restores the default (2^26
 * tests, about a second); 0 makes every such wait give up without testing (the give-up path on
 * demand, for tests of the error handling); up to 2^32 - 1 otherwise.  A wait that gives up makes
 * its warp stop, lets the copies the warp started land (waiting for them with the default limit),
 * and sets a status bit: amgc_vcycle and amgc_solve then return AMGC_TIMEOUT (amgc_last_error says
 * which call), and the output vector is incomplete.  The status is cleared when it is reported, so
 * the next call runs normally.  Drops the captured V-cycle graphs.  Synchronises the hierarchy's
 * last stream.  Errors: AMGC_EINVAL (h NULL, polls above 2^32 - 1), AMGC_ECUDA.  (Library
 * mechanics; the paper has no counterpart.) */
int amgc_set_wait_limit(struct amgc_hierarchy* h, int64_t polls);

/* Waits for the hierarchy's stream (and its auxiliary setup stream), then frees every device and
 * host resource the hierarchy owns (device memory goes back to the library's pool).  NULL is
 * accepted.  The handle must not be used afterwards. */
void amgc_destroy(struct amgc_hierarchy* h);
/* Static description of a status code (never NULL). */
const char* amgc_strerror(int code);
/* Detail of the last failure in the calling thread (empty string if none); valid until the
 * thread's next failing call. */
const char* amgc_last_error(void);

/* Number of CUDA kernels this library has launched in the calling process so far. */
int64_t amgc_launch_count(void);

/* Device memory of the library comes from a stream-ordered memory pool per device: buffers are
 * allocated and freed in order on the stream of the call (no device synchronisation on free),
 * and freed memory stays in the pool for later calls.  amgc_trim_memory waits for the current
 * device to finish its work and returns the pool's unused memory to the driver.  (Library
 * mechanics; the paper has no counterpart.)  Errors: AMGC_ECUDA. */
int amgc_trim_memory(void);

/* y[i] = x[i] rounded to FP32, to nearest with ties to even (the value a C cast gives), for
 * i < n: the conversion that feeds the FP32 cycle its input and forms the FP32 copies of the
 * hierarchy and of the Krylov basis.  x, y: device arrays of n elements, not overlapping; the
 * work is enqueued on stream (NULL: the default stream).  (Library mechanics; the paper has no
 * counterpart.)  Errors: AMGC_EINVAL for n < 0 or a NULL array with n > 0; AMGC_ECUDA. */
int amgc_f64_to_f32(int64_t n, const double* x, float* y, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* AMGC_H */
