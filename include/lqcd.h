/*
 * lqcd.h — C ABI of the GB300 (sm_103a) factorized-quark-propagator library.
 *
 * Method: Ce, Giusti, Schaefer, "Domain decomposition and multilevel
 * integration for fermions" (arXiv:1612.06424).  The library computes, on
 * one GPU, the Dirac-operator work of that method:
 *   - the Wilson(-clover) operator D, normalised as 2 kappa D = 1 - kappa D_hop
 *     (Sec. 5, definition below eq. stochastic_estimator), clover term
 *     c_sw (i/4) sum_{mu,nu} sigma_mu_nu Fhat_mu_nu(x) added to its diagonal;
 *   - its domain (block) operators D_L on time slabs with Dirichlet boundaries,
 *     the exact sub-blocks of D of eq. block_inverse (Sec. 3) and Sec. 5;
 *   - solves of D_L psi = eta and D psi = eta (Sec. 5: "solutions of the
 *     Dirac equation", and its cost counted in Dirac-operator inversions);
 *   - the factorized propagator of Sec. 3 (eqs. quark_prop_I, quark_prop_II)
 *     and its correction, corr = D^{-1} - fact (eq. observable_factorization);
 *   - the link force of S = phi^dag (D_L^dag D_L)^{-1} phi, the domain-local
 *     pseudofermion action the multilevel scheme needs for independent domain
 *     updates (Sec. 2.1, eq. action_decomposition; the paper defers its
 *     construction to its Ref. Ce:2016ajy).
 *
 * Conventions shared by every call
 *   dims        {T, L1, L2, L3}; x0 is time (slowest).  All four even, L3 >= 2.
 *   site index  i = ((x0*L1 + x1)*L2 + x2)*L3 + x3   ("natural order")
 *   gauge field U[i][mu][a][b], complex128 (re, im interleaved), mu = 0 time.
 *   spinor      psi[i][s][c], complex128, spin s = 0..3, colour c = 0..2,
 *               chiral gamma basis, gamma_5 = g0 g1 g2 g3 = diag(1, 1, -1, -1),
 *               g0 = [[0,-1],[-1,0]], g_k = [[0,-i s_k],[i s_k,0]] in 2x2 blocks.
 *   hopping     (D_hop psi)(x) = sum_mu (1 - g_mu) U_mu(x) psi(x+mu)
 *                                     + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu).
 *   time BC     LQCD_BC_OPEN (the paper's open BC, Sec. 5: no hop between
 *               x0 = T-1 and x0 = 0, and the clover leaves through that
 *               missing link vanish), LQCD_BC_PERIODIC, LQCD_BC_ANTIPERIODIC.
 *               Space is periodic.
 *   slab        {t0, t1}: the inclusive time range t0..t1.  A slab vector is
 *               the natural-order slice of a full-lattice vector over sites
 *               t0*L1*L2*L3 .. (t1+1)*L1*L2*L3 - 1 (time is slowest), i.e.
 *               (t1-t0+1)*L1*L2*L3*12 complex128 values.
 *   pointers    every data pointer is a DEVICE pointer unless the argument
 *               says otherwise; the caller owns it.  The library owns its
 *               internal even-odd, compressed and reduced-precision copies.
 *   stream      a cudaStream_t passed as void*; NULL means the legacy default
 *               stream.  Calls are stream-ordered; those that return solver
 *               statistics synchronise the stream before returning.
 *   errors      0 on success, a negative LQCD_E* code on failure, with a
 *               message from lqcd_last_error().  Nothing aborts or traps.
 *               A failed call leaves caller buffers in an unspecified state.
 */
#ifndef LQCD_H
#define LQCD_H

#ifdef __cplusplus
extern "C" {
#endif

#define LQCD_OK 0
#define LQCD_EBADARG (-1)      /* argument out of range or inconsistent        */
#define LQCD_ENOMEM (-2)       /* device allocation failed                      */
#define LQCD_ENONUNITARY (-3)  /* set_gauge: a link is not SU(3) to 1e-10       */
#define LQCD_ENOTCONVERGED (-4)/* a solve hit max_iter above its tolerance      */
#define LQCD_EBREAKDOWN (-5)   /* Krylov breakdown that restarts did not cure   */
#define LQCD_ENAN (-6)         /* NaN or Inf in a residual                      */
#define LQCD_ECUDA (-7)        /* a CUDA runtime call failed                    */
#define LQCD_ENOFIELD (-8)     /* field index not loaded                        */
#define LQCD_ERANK (-9)        /* vectors to orthonormalise are linearly dependent */

#define LQCD_BC_OPEN 0
#define LQCD_BC_PERIODIC 1
#define LQCD_BC_ANTIPERIODIC 2

#define LQCD_MEM_DEVICE 0
#define LQCD_MEM_HOST 1

typedef struct lqcd_lattice lqcd_lattice; /* opaque, owned by the library */

typedef struct {
  int t0, t1; /* inclusive time range */
} lqcd_slab;

/* Two-region split of Sec. 2.1 / 3: Gamma, the overlap DeltaGamma (a subset
 * of Gamma* adjacent to Gamma; empty when delta.t1 < delta.t0) and Gamma*.
 * Gamma u Gamma* must be the whole time range, Gamma first; Gammabar =
 * Gamma u DeltaGamma. */
typedef struct {
  lqcd_slab gamma, delta, gamma_star;
} lqcd_split;

typedef struct {
  double tol;            /* target relative true residual ||eta - D psi|| / ||eta||   */
  int max_iter;          /* bound on Krylov iterations per system (all cycles)        */
  int precision;         /* 64: FP64 throughout; 32: FP32 inner solves with FP64
                            defect correction; 16: FP16 vectors (per-site FP32 norm)
                            and FP16 links in the inner solves, FP64 correction      */
  double inner_tol;      /* relative residual reduction per inner cycle (0: default,
                            3e-6 for FP32, 2e-2 for FP16) */
  int check_every;       /* iterations between host convergence checks (0: default) */
  int max_wave;          /* systems solved together at most (0: as many as fit in free
                            device memory; larger batches run in consecutive waves)  */
} lqcd_solver_params;

typedef struct {
  int iters;             /* inner Krylov iterations summed over cycles                */
  int cycles;            /* FP64 defect-correction cycles (true residual evaluations) */
  int status;            /* LQCD_OK, LQCD_ENOTCONVERGED, LQCD_EBREAKDOWN or LQCD_ENAN */
  double true_residual;  /* ||eta - D psi||_2 / ||eta||_2 recomputed in FP64 from the
                            final iterate (even-odd: the odd half b^_o - D^ psi_o; the
                            reconstructed even half is exact up to rounding)          */
  double seconds;        /* wall time of the call that produced this entry           */
} lqcd_solver_stats;

/* Create a lattice of the given dims with time boundary condition bc_t.
 * *out receives an opaque handle owned by the library.  Selects the current
 * CUDA device.  Errors: LQCD_EBADARG (an extent odd or below 2; V/2 * 72 at
 * or above 2^31, since site indices of the packed link / clover arrays are
 * 32-bit; V/2 * max(L1, L2, L3/2) at or above 2^32, since site coordinates
 * are recovered with one multiply-high per division). */
int lqcd_create_lattice(const int dims[4], int bc_t, lqcd_lattice **out);

/* Free every device buffer of the lattice; the handle becomes invalid. */
int lqcd_destroy_lattice(lqcd_lattice *lat);

/* Load n_fields gauge fields U[n_fields][V][4][3][3] (complex128, natural
 * order; host memory if mem == LQCD_MEM_HOST, else device memory) with the
 * operator parameters kappa and c_sw (c_sw = 0: plain Wilson, Sec. 5).
 * Builds, per field, the even-odd packed links in FP64 / FP32 / FP16 (the
 * reduced copies keep the first two rows, the third is rebuilt as
 * conj(row0 x row1)), the clover blocks A(x) on every site and their
 * inverses on even sites.  Replaces any fields loaded before.
 * Errors: LQCD_ENONUNITARY when a link deviates from SU(3) by > 1e-10
 * (max |U U^dag - 1| or |det U - 1|), LQCD_ENOMEM. */
int lqcd_set_gauge(lqcd_lattice *lat, int n_fields, const double *U, double kappa, double c_sw, int mem,
                   void *stream);

/* out = D_L in (dagger = 0) or D_L^dag in (dagger = 1) for the slab dom
 * (NULL: the whole lattice, with the lattice's time BC) on field `field`,
 * evaluated in `precision` (64, 32 or 16) through the even-odd packed data.
 * in / out: device slab vectors (see "slab" above) in complex128.
 * Sec. 3 eq. block_inverse: D_L is the sub-block of D on the slab's sites. */
int lqcd_dslash(lqcd_lattice *lat, int field, const lqcd_slab *dom, int dagger, int precision, const double *in,
                double *out, void *stream);

/* Batched solve of D_{L_k} psi_k = eta_k for k < n_sys, system k on slab
 * doms[k] of field field_ids[k].  src / sol: device slab vectors of the
 * systems packed back to back in the order k = 0..n_sys-1 (system k starts
 * after the slab vectors of systems 0..k-1).  sol is overwritten.
 * All systems advance together in the same kernels (even-odd preconditioned
 * BiCGStab, FP64 defect correction).  stats: host array of n_sys entries or
 * NULL.  Returns LQCD_ENOTCONVERGED if any system stopped above tol. */
int lqcd_solve_block(lqcd_lattice *lat, int n_sys, const lqcd_slab *doms, const int *field_ids, const double *src,
                     double *sol, const lqcd_solver_params *params, lqcd_solver_stats *stats, void *stream);

/* Batched full-lattice solve D psi_k = eta_k (the correction solve of
 * Sec. 3.2); src / sol are n_sys full-lattice vectors back to back. */
int lqcd_solve_full(lqcd_lattice *lat, int n_sys, const int *field_ids, const double *src, double *sol,
                    const lqcd_solver_params *params, lqcd_solver_stats *stats, void *stream);

/* Batched point-source propagators: system k solves D_{L_k} psi_k = eta_k on
 * slab doms[k] of field field_ids[k] with the point source
 * eta_k(y) = delta(y, x_k) delta(s, s_k) delta(c, c_k), x_k = x_src[4k..4k+3]
 * (inside the slab), column cols[k] = 3 s_k + c_k.  The sources are built on
 * the device (no source arrays).  sol: device slab vectors back to back as in
 * lqcd_solve_block.  Systems beyond free device memory run in consecutive
 * waves (params->max_wave caps a wave).  stats: host array of n_sys or NULL. */
int lqcd_point_propagators(lqcd_lattice *lat, int n_sys, const lqcd_slab *doms, const int *field_ids,
                           const int *x_src, const int *cols, double *sol, const lqcd_solver_params *params,
                           lqcd_solver_stats *stats, void *stream);

/* The 12-source factorized propagator of Sec. 3 for point sources at x_src
 * (x_src[0] inside Gamma), on field `field`:
 *   y in Gamma:  fact(y,x) = D_Gamma^{-1}(y,x)                        eq. quark_prop_I
 *   y in Gamma*: fact(y,x) = -[D_Gamma*^{-1} D_dGamma* D_Gammabar^{-1}](y,x)  eq. quark_prop_II
 * with D_dGamma* the block of D from Gamma to Gamma* (eq. block_inverse).
 * fact: device [12][V][4][3] complex128, column col = 3*s0 + c0 of the
 * source.  corr: device [12][V][4][3] receiving D^{-1} - fact (the full
 * solve on the lattice), or NULL to skip it.  stats: host array of
 * 4 entries (Gamma, Gammabar, Gamma*, full) aggregated over the 12
 * columns (max iterations, max residual, worst status), or NULL. */
int lqcd_factorized_propagator(lqcd_lattice *lat, const lqcd_split *split, const int x_src[4], int field,
                               double *fact, double *corr, const lqcd_solver_params *params,
                               lqcd_solver_stats *stats, void *stream);

/* lqcd_factorized_propagator for n_fields gauge fields at once (the level-1
 * fields of Sec. 2.2 eq. multilevel_estimator, whose factors the two-level
 * average needs field by field): field_ids[j] < loaded fields, j < n_fields.
 * fact: device [n_fields][12][V][4][3] complex128; corr: the same shape or
 * NULL; stats: host array of 4 n_fields entries, stats[4 j + k] as in
 * lqcd_factorized_propagator for field j, or NULL.  The 12 n_fields systems
 * of each kind are solved in one batch (consecutive waves when they exceed
 * free device memory), in four stages: Gamma; Gammabar started from the
 * Gamma solution (zero on DeltaGamma); Gamma* from the boundary source; the
 * full lattice started from fact.  A starting iterate changes iteration
 * counts only: every system stops at ||eta - D psi|| <= tol ||eta|| in FP64.
 * Errors: LQCD_EBADARG, LQCD_ENOFIELD, LQCD_ENOMEM, LQCD_ENOTCONVERGED,
 * LQCD_ECUDA. */
int lqcd_factorized_propagators(lqcd_lattice *lat, const lqcd_split *split, const int x_src[4], int n_fields,
                                const int *field_ids, double *fact, double *corr, const lqcd_solver_params *params,
                                lqcd_solver_stats *stats, void *stream);

/* The boundary source of eq. quark_prop_II on its own (Sec. 3 eq.
 * block_inverse: D_dGamma* is the block of D from Gamma to Gamma*):
 *   chi_k = P_Gamma* D P_Gamma psi_k,  k < n,
 * for psi_k a device slab vector on Gammabar (e.g. D_Gammabar^{-1} eta from
 * lqcd_point_propagators), on field field_ids[k].  chi: device [n][2][L1 L2
 * L3][4][3] complex128, overwritten: slot 0 the first slice of Gamma* (the
 * backward time hop from the last slice of Gamma), slot 1 the last slice
 * x0 = T-1 (the wrapping hop to x0 = 0; zero for the open time boundary).
 * With lqcd_schur_solve it splits a factorized propagator between processes
 * that exchange chi alone (L1 L2 L3 x 12 complex per source and slot).
 * Synchronises.  Errors: LQCD_EBADARG, LQCD_ENOFIELD, LQCD_ECUDA. */
int lqcd_schur_boundary(lqcd_lattice *lat, const lqcd_split *split, int n, const int *field_ids, const double *psi,
                        double *chi, void *stream);

/* The Gamma* half of eq. quark_prop_II: fact_k = -D_Gamma*^{-1} chi_k on
 * field field_ids[k], k < n, with chi in the layout of lqcd_schur_boundary.
 * fact_gs: device [n] slab vectors on Gamma* back to back, overwritten.
 * stats: host array of n entries or NULL.  Errors: LQCD_EBADARG,
 * LQCD_ENOFIELD, LQCD_ENOMEM, LQCD_ENOTCONVERGED, LQCD_ECUDA. */
int lqcd_schur_solve(lqcd_lattice *lat, const lqcd_split *split, int n, const int *field_ids, const double *chi,
                     double *fact_gs, const lqcd_solver_params *params, lqcd_solver_stats *stats, void *stream);

/* Nucleon correlators of point-source propagators (the two Wick
 * contractions whose factorized form is Sec. 4.2 eq. nucleon_prop_factorized),
 * summed over the sink sites y of each time slice t0 .. t0+n_t-1:
 *   W[p][t][0] = W1 = sum_y eps^{abc} eps^{a'b'c'} (C g5)_{mu nu} (C g5)_{mu' nu'}
 *                (g5 P_-)_{gam del} S^{ab'}_{mu nu'} S^{ba'}_{nu mu'} S^{cc'}_{del gam}
 *   W[p][t][1] = W2 = the same with S^{ab'}_{mu nu'} S^{bc'}_{nu gam} S^{ca'}_{del mu'}
 * with S = S_p(y, x)[(sink spin, colour), (source spin, colour)] =
 * prop[p][3 s0 + c0][y][s][c], C = g0 g2, P_- = (1 - g0)/2; the correlator is
 * W1 - W2.  prop: device [n_prop][12][V][4][3] complex128 (e.g. fact or
 * fact + corr of lqcd_factorized_propagators); W: device [n_prop][n_t][2]
 * complex128.  FP64, one warp per site, block sums in a fixed order.
 * Stream-ordered.  Errors: LQCD_EBADARG, LQCD_ENOMEM, LQCD_ECUDA. */
int lqcd_nucleon_point(lqcd_lattice *lat, int n_prop, const double *prop, int t0, int n_t, double *W, void *stream);

/* The hierarchy of Sec. 6 eq. nucleon_prop_hierarchical for the 12 point
 * sources at x_src on field `field`: C^(d) is the nucleon correlator
 * (lqcd_nucleon_point, W1 - W2) of the factorized propagator with the overlap
 * DeltaGamma_d = gamma.t1+1 .. delta_t1[d] (nested: gamma.t1 < delta_t1[0] <
 * ... < delta_t1[n_d-1] < T-1; split->delta is ignored), C that of the full
 * propagator.  All overlaps run in one batched set of solves (Gamma and the
 * full lattice once, the n_d Gammabar and Gamma* stages together).
 * C: host [n_d + 2][T] complex128, row k < n_d+1 the k-th term of
 *   C = C^(0) + [C^(1) - C^(0)] + ... + [C^(n_d-1) - C^(n_d-2)] + [C - C^(n_d-1)],
 * the last term C^(rest); row n_d+1 the full C.  stats: host array of 4
 * entries (Gamma, Gammabar, Gamma*, full; each the worst over columns and
 * overlaps) or NULL.  Synchronises.  Errors: LQCD_EBADARG, LQCD_ENOFIELD,
 * LQCD_ENOMEM, LQCD_ENOTCONVERGED, LQCD_ECUDA. */
int lqcd_nucleon_hierarchy(lqcd_lattice *lat, const lqcd_split *split, int n_d, const int *delta_t1,
                           const int x_src[4], int field, double *C, const lqcd_solver_params *params,
                           lqcd_solver_stats *stats, void *stream);

/* Link force of S = phi^dag (D_L^dag D_L)^{-1} phi for the slab dom on field
 * `field`: force[i][mu][a] = dS/domega for U_mu(x_i) -> exp(i omega T_a)
 * U_mu(x_i), T_a = lambda_a / 2 (Gell-Mann), i.e.
 *   F = -2 Re <Y, (dD_L/domega) X>,  Y = D_L^{-dag} phi,  X = D_L^{-1} Y,
 * hopping and clover terms included.  phi: device slab vector on dom;
 * force: device [V][4][8] float64, every link of the lattice (links outside
 * the slab reached by the clover leaves of its sites are included; the rest
 * are 0), or NULL to compute the action alone (one D^dag solve).
 * action: host double receiving S = ||Y||^2, or NULL.
 * stats: host array of 2 entries (the D^dag and D solves) or NULL.  X and Y
 * are recomputed on every call, never cached. */
int lqcd_link_force(lqcd_lattice *lat, const lqcd_slab *dom, int field, const double *phi, double *force,
                    double *action, const lqcd_solver_params *params, lqcd_solver_stats *stats, void *stream);

/* Projection vectors of the quark-line cut (Sec. 6: N_m orthonormal vectors
 * from inverse iterations of the Dirac operator on a slab around the
 * boundary).  Starting from v0 (device, n_modes slab vectors on dom back to
 * back), each of the n_iter iterations solves D_L w_i = v_i (L = dom, all
 * i together) and orthonormalises the w_i (Cholesky QR, twice: the unique
 * orthonormal basis W with V = W R, R upper triangular with positive real
 * diagonal).  Then phi = the same orthonormalisation of P_+ v_i restricted
 * to time slice g1 (P_+ = (1 + g0)/2, the half of a spinor that the
 * boundary block D_dGamma* reads when g1 is the last slice of Gamma; the
 * span is the 6 L1 L2 L3-dimensional space of Sec. 3.3).
 * phi: device [n_modes][L1 L2 L3][4][3] complex128, overwritten.
 * Limits: 1 <= n_modes <= min(1024, 6 L1 L2 L3); g1 inside dom.
 * stats: host, one entry aggregated over every solve, or NULL.
 * Errors: LQCD_EBADARG, LQCD_ENOFIELD, LQCD_ERANK (v0 or its slice part
 * linearly dependent), LQCD_ENOTCONVERGED, LQCD_ECUDA. */
int lqcd_boundary_modes(lqcd_lattice *lat, const lqcd_slab *dom, int g1, int field, int n_modes, int n_iter,
                        const double *v0, double *phi, const lqcd_solver_params *params, lqcd_solver_stats *stats,
                        void *stream);

/* The two factors of the projected quark line (Sec. 3.3 eq.
 * quark_prop_II_proj) for projection vectors phi_i (device [n_modes][L1 L2
 * L3][4][3], living on the last slice g1 of Gamma), on field `field`:
 *   xi_i  = D_Gammabar^{-dag} phi_i   (so [phi_i^dag D_Gammabar^{-1}](x) = xi_i(x)^dag;
 *                                      the paper's xi_i^T is xi_i^dag)
 *   eta_i = D_Gamma*^{-1} D_dGamma* phi_i
 * xi: device [n_modes] slab vectors on Gammabar; eta: device [n_modes] slab
 * vectors on Gamma*.  Open time boundary only (LQCD_EBADARG otherwise).
 * stats: host array of 2 entries (the Gammabar and the Gamma* solves) or NULL.
 * Errors: LQCD_EBADARG, LQCD_ENOFIELD, LQCD_ENOTCONVERGED, LQCD_ECUDA. */
int lqcd_projected_factors(lqcd_lattice *lat, const lqcd_split *split, int field, int n_modes, const double *phi,
                           double *xi, double *eta, const lqcd_solver_params *params, lqcd_solver_stats *stats,
                           void *stream);

/* The projected factorized propagator on Gamma* (eq. quark_prop_II_proj,
 * case II) for the 12 point sources at x_src (x_src[0] inside Gamma):
 *   fact[b](y)[a] = - sum_i eta_i(y)[a] conj(xi_i(x)[b]),  b = 3 s0 + c0,
 * from factors of lqcd_projected_factors (xi and eta may come from different
 * gauge fields: the n1^2 pairs of the two-level average).  fact: device
 * [12][V][4][3]; only the sites of Gamma* are written.  Synchronises.
 * Errors: LQCD_EBADARG (1 <= n_modes <= 1024), LQCD_ECUDA. */
int lqcd_projected_propagator(lqcd_lattice *lat, const lqcd_split *split, int n_modes, const double *xi,
                              const double *eta, const int x_src[4], double *fact, void *stream);

/* Nucleon blocks of the factorized nucleon propagator (Sec. 4.2 eq.
 * nucleon_prop_factorized) for n fields s_i (device [n] slab vectors on
 * `slab`, complex128; conj = 1 uses conj(s_i), e.g. the xi of
 * lqcd_projected_factors, whose conjugate is the paper's row xi_i^T), for the
 * time slices t0 .. t0+n_t-1 (inside the slab):
 *   B[t][i][j][k][alpha] = sum_{xvec} eps^{abc} {[s_i^T]^a(x) C g5 [s_j]^b(x)} [s_k]^c_alpha(x)
 * with C = g0 g2 (C g_mu C^{-1} = -g_mu^T in the basis above).  B: device
 * [n_t][n][n][n][4] complex128, overwritten.  Arithmetic (default, the tensor
 * cores): the inputs rounded to FP32 once, the diquark in FP32, the (x, c)
 * contraction as a real GEMM on tcgen05 in three TF32 passes (hi*hi + hi*lo +
 * lo*hi of each operand's split into an 11-bit head and an FP32 remainder),
 * accumulated in FP32 per 64 sites and then in FP32 running sums; relative
 * error at most about (16 + 288 + L1 L2 L3 / 64) 2^-24 of the sum of |terms|;
 * stored as FP64.  Scratch: one FP32 copy of the fields on up to about 2 GB
 * worth of slices at a time (stream-ordered allocation).  The call waits for
 * its kernels (it reads back the status of their bounded waits on the tensor
 * pipeline).  With the environment variable LQCD_NUCLEON_TC=0: the FP32-FMA
 * kernel (partial sums over 64 sites, then their running sum; relative error
 * about (200 + L1 L2 L3 / 64) 2^-24 of the sum of |terms|), stream-ordered,
 * no synchronisation.  1 <= n <= 1024.
 * Errors: LQCD_EBADARG, LQCD_ENOMEM, LQCD_ECUDA (also when a tensor-core
 * wait timed out). */
int lqcd_nucleon_blocks(lqcd_lattice *lat, const lqcd_slab *slab, int n, const double *s, int conj, int t0, int n_t,
                        double *B, void *stream);

/* The two factorized Wick contractions for every pair (source slice ix of
 * B_xi, sink slice iy of B_eta) (eq. nucleon_prop_factorized):
 *   W[ix][iy][0] = W1 = -sum_ijk B_xi[ix][j][i][k]^T g5 P_- B_eta[iy][i][j][k]
 *   W[ix][iy][1] = W2 = -sum_ijk B_xi[ix][k][i][j]^T g5 P_- B_eta[iy][i][j][k]
 * with P_- = (1 - g0)/2, in FP64; C_N^(f)(y0, x0) = (W1 - W2) / (L1 L2 L3).
 * B_xi: device [n_x][n][n][n][4], B_eta: device [n_y][n][n][n][4] complex128
 * (level-1 averages of blocks may be passed for the two-level estimator);
 * W: device [n_x][n_y][2] complex128.  Errors: LQCD_EBADARG, LQCD_ECUDA. */
int lqcd_nucleon_contract(int n, int n_x, const double *B_xi, int n_y, const double *B_eta, double *W, void *stream);

/* Level-1 average of the two-level estimator (Sec. 2.2 eq.
 * multilevel_estimator): out[e] = (1/count) sum_{j<count} in[j*size + e] for
 * count arrays of `size` complex128 entries stored back to back (device), in
 * FP64 and in j order.  Averaging the blocks (or factors) of each region over
 * its n1 level-1 fields before contracting gives the product of the two
 * level-1 averages.  Errors: LQCD_EBADARG, LQCD_ECUDA. */
int lqcd_level_mean(long long size, int count, const double *in, double *out, void *stream);

/* Stochastic estimator of the disconnected traces of Sec. 4.1 (eq.
 * stochastic_estimator of Sec. 5) on each slab L_d = doms[d], d < n_doms, of field
 * `field` (Dirichlet blocks of Sec. 3, or the whole lattice for doms[d] =
 * 0..T-1), all sources and slabs solved together:
 *   trace[i][d][x0] = sum_{xvec} eta_i^dag(x) [(kappa D_hop)^8 D_L^{-1} g5 eta_i](x)
 * for x0 in L_d (0 elsewhere), with kappa D_hop = 1 - 2 kappa D_L on the
 * slab, g5 = diag(1, 1, -1, -1) in spin.  Its mean over i estimates
 * sum_{xvec} tr{g5 D_L^{-1}(x,x)}; the eighth power (exact for Wilson
 * quarks: every closed path shorter than 8 hops has a vanishing g5 trace)
 * only lowers the noise.  Wilson operator only: the lattice's c_sw must be 0
 * (else LQCD_EBADARG).
 * eta: device [n_src][V][4][3] complex128, sources on the whole lattice
 *   (only each slab's part enters; the caller draws them, e.g. Gaussian).
 * trace: device [n_src][n_doms][T] complex128, overwritten.
 * mean: device [n_doms][T] complex128 receiving (1/n_src) sum_i trace[i],
 *   or NULL.
 * D_L^{-1} g5 eta_i is solved to params->tol (relative residual); the eight
 * hops and the contraction run in FP64.  stats: host array of n_doms
 * entries (each aggregated over the sources), or NULL.  Solutions are not
 * kept: systems run in waves that fit in free device memory.
 * Errors: LQCD_EBADARG, LQCD_ENOFIELD, LQCD_ECUDA, LQCD_ENOTCONVERGED. */
int lqcd_disconnected_trace(lqcd_lattice *lat, int n_doms, const lqcd_slab *doms, int field, int n_src,
                            const double *eta, double *trace, double *mean, const lqcd_solver_params *params,
                            lqcd_solver_stats *stats, void *stream);

/* Timing hook of the stencil (no counterpart in the paper: a measurement
 * aid).  Builds the batch of systems (slab doms[k] on field field_ids[k]),
 * fills two synthetic vectors, and launches `reps` times the hop kernel the
 * solver uses for the second half of the even-odd operator,
 *   out_o = A_oo y_o - 1/4 D_hop x_e     (precision 64, 32 or 16),
 * after 3 untimed launches, timed with CUDA events on `stream`.
 * ms_per_launch: mean launch duration (ms).  bytes_per_launch: algorithmic
 * bytes = 3 spinors per system site + (8 links + 1 clover block) per distinct
 * site of each field's slabs.  flops_per_launch: (1320 hop + 504 clover + 72)
 * per system site.  Any output pointer may be NULL. */
int lqcd_dslash_bench(lqcd_lattice *lat, int n_sys, const lqcd_slab *doms, const int *field_ids, int precision,
                      int reps, double *ms_per_launch, double *bytes_per_launch, double *flops_per_launch,
                      void *stream);

/* Timing hook of one kernel of the solver's BiCGStab iteration (no
 * counterpart in the paper: a measurement aid), on the batch of systems
 * (slab doms[k] on field field_ids[k]) with synthetic vectors, in the
 * solver's launch shape, timed like lqcd_dslash_bench.  kernel:
 *   0  out_o = A_oo y_o - 1/4 D_hop x_e            (3 spinor passes)
 *   1  out_e = A_ee^{-1} D_hop x_o                 (2 passes; first half of D^)
 *   2  kernel 0 with the reduction <r0, out>       (4 passes)
 *   3  kernel 0 with <out, y> and |out|^2          (3 passes)
 *   4  s = r - alpha v                             (3 passes)
 *   5  x += alpha p + omega s, r = s - omega t, <r0, r>, |r|^2   (7 passes)
 *   6  p = r + beta (p - omega v)                  (4 passes)
 * bytes_per_launch: algorithmic bytes = passes x spinor bytes per system
 * site, plus (8 links + 1 clover block) per distinct field site of the
 * slabs for kernels 0-3.  flops_per_launch: per system site, hop 1320 +
 * site-diagonal block (504 with clover, else 24) + epilogue / reductions
 * (kernels 0-3), or the vector arithmetic (kernels 4-6).  Errors:
 * LQCD_EBADARG, LQCD_ENOFIELD, LQCD_ENOMEM, LQCD_ECUDA. */
int lqcd_stencil_bench(lqcd_lattice *lat, int n_sys, const lqcd_slab *doms, const int *field_ids, int precision,
                       int kernel, int reps, double *ms_per_launch, double *bytes_per_launch,
                       double *flops_per_launch, void *stream);

/* Measured FMA throughput of the current GPU in TFLOP/s (bits = 64 or 32;
 * no counterpart in the paper: the ALU roofline of the FP64 kernels).  One
 * launch of 8 independent FMA chains per thread on 8 blocks per SM, timed
 * with CUDA events on `stream`; synchronises.  Errors: LQCD_EBADARG. */
int lqcd_fma_peak(int bits, double *tflops, void *stream);

/* Size of the device scratch array of lqcd_dslash_noalloc (16 MiB). */
#define LQCD_NOALLOC_SCRATCH_BYTES (16 * 1024 * 1024)

/* Allocation-free variant of lqcd_dslash in FP64 (no counterpart in the
 * paper: an integration aid).  Same operation, arguments and layouts as
 * lqcd_dslash with precision 64: out = D_L in (dagger = 0) or D_L^dag in
 * (dagger = 1) on the slab dom (NULL: whole lattice) of field `field`.
 * For callers that cannot allocate device memory while they run -- an
 * application whose own allocator owns the GPU's memory, or a latency-
 * critical path where an allocation's cost or failure is not acceptable --
 * it calls no cudaMalloc / cudaFree or allocating library routine: its
 * scratch (even / odd copies of in and out, the system descriptor, a
 * pointer table) lives in one file-scope device array of
 * LQCD_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits.  The caller still owns and passes in / out (device).
 * Limit: the scratch needs 512 + 768 n bytes for a slab of n sites per
 * parity, so the slab may hold at most 2 floor((LQCD_NOALLOC_SCRATCH_BYTES -
 * 512) / 768) = 43 688 sites (e.g. a 16^3 x 10 slab); larger slabs return
 * LQCD_EBADARG.  The descriptor and the in / out pointers reach the scratch
 * array as kernel arguments of a one-thread set-up kernel.
 * The first call on a device looks up the array's device address (with that
 * device current) and caches it.  All calls share the one array and it
 * keeps the last call's contents (every word a call reads is written by
 * that call first): calls that overlap on the GPU -- on different streams
 * or host threads without ordering between them -- race and must not be
 * issued.  Stream-ordered; does not synchronise.  Errors: LQCD_EBADARG, LQCD_ENOFIELD, LQCD_ECUDA. */
int lqcd_dslash_noalloc(lqcd_lattice *lat, int field, const lqcd_slab *dom, int dagger, const double *in, double *out,
                        void *stream);

/* Message of the last failing call on this host thread ("" if none). */
const char *lqcd_last_error(void);

/* Number of kernels this library has launched since load (all streams);
 * a host-side counter for accounting, not synchronised with the device. */
long long lqcd_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* LQCD_H */
