/* qcd.h - C-ABI of the GB300 Wilson-clover AMA library.
 *
 * The library solves the Dirac equation D psi = eta for O(a)-improved
 * Wilson-clover quarks with a Schwarz-alternating-procedure (SAP)
 * preconditioned flexible GCR solver, and forms the nucleon two-point
 * function and its all-mode-averaging (AMA) estimate from point-source
 * propagators (arXiv:1605.00564, Sec. 2).  Everything is computed by CUDA
 * kernels on the caller's GPU; there is no CPU fallback.
 *
 * Conventions (all entry points):
 *  - dims = {T, X, Y, Z}.  Site index s = ((t*Z + z)*Y + y)*X + x (x fastest).
 *  - Canonical FP64 layouts, complex numbers as interleaved (re, im) doubles:
 *      spinor     [rhs][site][spin 4][colour 3]
 *      gauge      [site][mu 4][row 3][col 3], mu = 0 time, 1 x, 2 y, 3 z;
 *                 U_mu(x) is the link from x to x + mu-hat
 *      propagator the 12 spinors of one point source, rhs = 3*spin + colour
 *  - The operator (kappa normalisation, chiral Euclidean gamma basis,
 *    gamma_5 = diag(1,1,-1,-1), sigma_{mu nu} = (i/2)[g_mu, g_nu]):
 *      D psi(x) = psi(x) - kappa sum_mu [(1 - g_mu) U_mu(x) psi(x+mu)
 *                                      + (1 + g_mu) U_mu(x-mu)^+ psi(x-mu)]
 *               + i kappa c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x) psi(x)
 *    F_{mu nu} = (Q_{mu nu} - Q_{mu nu}^+)/8 from the four plaquette leaves
 *    Q_{mu nu}; periodic in space, time_bc (+1 / -1) on hops across t = 0.
 *  - Tolerances are relative: ||eta - D psi||_2 / ||eta||_2, evaluated in FP64.
 *  - Ownership: the caller owns every buffer it passes; the library owns the
 *    context and its internal copies and workspaces.  "device" pointers are
 *    CUDA global memory of the context's device; "host" pointers are CPU
 *    memory (pinned or pageable).  Work is ordered on the context's stream;
 *    calls that return results to host memory synchronise that stream.
 *  - Errors: every call returns a qcd_status; nothing throws across the ABI.
 *    qcd_last_error() gives a message for the most recent failure of the
 *    calling thread.  Argument errors are detected before any launch.
 */
#ifndef QCD_GB300_H
#define QCD_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qcd_ctx qcd_ctx; /* opaque, library-owned */

typedef enum {
  QCD_OK = 0,
  QCD_ERR_ARG = 1,            /* invalid argument (checked before any launch) */
  QCD_ERR_CUDA = 2,           /* a CUDA runtime call failed */
  QCD_ERR_OOM = 3,            /* device allocation failed */
  QCD_ERR_NOT_CONVERGED = 4,  /* solver hit max_outer; psi holds the best iterate */
  QCD_ERR_BREAKDOWN = 5,      /* a Gram-Schmidt norm vanished */
  QCD_ERR_NONFINITE = 6,      /* NaN or Inf in an input or a residual */
  QCD_ERR_TIMEOUT = 7,        /* a bounded device wait gave up */
  QCD_ERR_STATE = 8           /* call out of order (e.g. solve before load_gauge) */
} qcd_status;

/* Precision of a computation.  QCD_PREC_F64 is the plain double-precision
 * path; QCD_PREC_F32 stores and computes in single precision. */
typedef enum { QCD_PREC_F64 = 0, QCD_PREC_F32 = 1 } qcd_precision;

/* Solver parameters (Sec. 2.2: block size and n_cy are the SAP tunables;
 * the GCR restart length and stopping rule are the outer solver's).
 *   block       SAP block extents {T, X, Y, Z}; each must divide the lattice
 *               and give an even number of blocks per direction
 *               (checkerboard colouring of the blocks).  Block volume <= 1024.
 *   ncy         SAP cycles per preconditioner application (paper: 5).
 *   nmr         minimal-residual steps per block solve.
 *   nkv         GCR Krylov vectors per restart cycle (<= 32).
 *   max_outer   cap on GCR iterations (preconditioner applications) per RHS.
 *   restart_drop  a restart cycle ends when the recursive residual fell by
 *               this factor (0 = only at nkv); the true residual is then
 *               recomputed.  Used with the mixed-precision policy.
 *   precision   QCD_PREC_F32: FP64 outer vectors and true residuals, FP32 SAP
 *               and Krylov basis (mixed precision, Sec. 2.2 last paragraph);
 *               QCD_PREC_F64: everything in FP64.
 *   rhs_tile    right-hand sides solved together (0 = library choice).
 *   dfl         1 = use the deflated preconditioner once qcd_deflation_setup
 *               has built the subspace (FP32 inner precision only):
 *               M rho = Phi A^-1 Phi^+ rho + M_SAP(P_L rho), Sec. 2.2 local
 *               deflation; the deflation blocks are the SAP blocks.
 *   dfl_little_iters  steps of the block-Jacobi preconditioned GCR that
 *               approximates A^-1 on the little vectors.
 *   graphs      1 = each SAP application (its 2 n_cy sweep launches) is replayed
 *               from a CUDA graph captured on first use for the same buffers
 *               and parameters (needs a non-default stream; otherwise, and with
 *               0, the launches are issued one by one).
 *   dfl_gen_iters  subspace generation: 0 = every inverse-iteration round
 *               applies M_SAP; k > 0 = the first round applies M_SAP and the
 *               later rounds k iterations of the deflated SAP-GCR solver.
 *   sap_half    FP32 SAP only: 1 = the block's links and clover term are held
 *               as 16-bit copies in shared memory during a block solve (the
 *               preconditioner changes by their rounding; the outer flexible
 *               GCR is unaffected in what it converges to); 2 = in addition the
 *               block residual read by neighbouring sites is held as bf16;
 *               0 = FP32 copies.
 *   basis_half  QCD_PREC_F32 only: 1 = the GCR images chi_k = D phi_k are
 *               stored as FP16 with one FP32 scale per site (52 bytes per site
 *               instead of 96; arithmetic stays FP32).  The recursive residual
 *               then carries the FP16 rounding (about 3e-4 relative), so it is
 *               meant for sloppy tolerances; convergence is still decided by
 *               the true residual.  qcd_ama_nucleon_2pt applies it to the
 *               sloppy solves only.  0 = FP32 storage.  Ignored for QCD_PREC_F64.
 *   resid_f32_tol  QCD_PREC_F32 only: a tile of right-hand sides whose every
 *               tolerance is >= resid_f32_tol evaluates its true residuals
 *               eta - D psi with the FP32 operator (psi rounded to FP32, the
 *               difference taken in FP64).  The rounding of D psi, about
 *               1e-7 |D| |psi|, stays far below such a stopping tolerance,
 *               while FP64 arithmetic runs at 1/64 of the FP32 rate on this
 *               GPU.  0 = FP64 true residuals always (the default).  A value
 *               below 1e-4 is rejected.
 */
typedef struct {
  int block[4];
  int ncy;
  int nmr;
  int nkv;
  int max_outer;
  double restart_drop;
  int precision;
  int rhs_tile;
  int sap_half;
  int dfl;
  int dfl_little_iters;
  int dfl_gen_iters;
  int graphs;
  int basis_half;
  double resid_f32_tol;
} qcd_solver_params;

/* Per right-hand-side outcome of a solve. */
typedef struct {
  int status;                 /* QCD_OK or QCD_ERR_NOT_CONVERGED / ..._NONFINITE */
  int outer_iters;            /* GCR iterations (preconditioner applications) */
  int restarts;               /* true-residual recomputations */
  double true_rel_residual;   /* ||eta - D psi|| / ||eta|| at exit (FP64 sums;
                                 D psi in FP64, or FP32 under resid_f32_tol) */
} qcd_rhs_stats;

/* Message for a status code (static string). */
const char* qcd_status_string(qcd_status s);
/* Message of the last failure in this thread (static per-thread buffer). */
const char* qcd_last_error(void);

/* Create a context for a lattice dims = {T, X, Y, Z} on the current CUDA
 * device (library plumbing; no counterpart in the paper).  cuda_stream is a cudaStream_t (NULL = legacy default stream).
 * Each extent must be >= 2; T*X*Y*Z < 2^31. */
qcd_status qcd_create(qcd_ctx** out, const int dims[4], void* cuda_stream);
void qcd_destroy(qcd_ctx* ctx);

/* Load the gauge field and the operator's couplings (Sec. 2.2, the Dirac
 * equation D psi = eta for O(a)-improved Wilson quarks).  U is canonical
 * FP64, on the device when U_on_device != 0, else host.  The clover term is
 * built on the device from the plaquette leaves.  time_bc is +1 or -1. */
qcd_status qcd_load_gauge(qcd_ctx* ctx, const double* U, int U_on_device, double csw, double kappa,
                          int time_bc);

/* The solver's tunables (Sec. 2.2 and the struct above).
 * Default parameters: block 4^4, ncy 5, nmr 4, nkv 16, max_outer 2000,
 * restart_drop 1e-5, precision F32, rhs_tile 0, sap_half 0, dfl 1,
 * dfl_little_iters 16, dfl_gen_iters 0, graphs 1, basis_half 0, resid_f32_tol 0. */
void qcd_default_params(qcd_solver_params* p);
qcd_status qcd_set_params(qcd_ctx* ctx, const qcd_solver_params* p);

/* The operator of the Dirac equation D psi = eta (Sec. 2.2; O(a)-improved
 * Wilson quarks): out = D in (dagger = 0) or D^+ in (dagger = 1) for nrhs
 * canonical spinors on the device, computed in the given precision (inputs are rounded to it;
 * the output is written back in FP64).  in and out must not overlap. */
qcd_status qcd_apply_dirac(qcd_ctx* ctx, const double* in, double* out, int nrhs, int dagger, int precision);

/* psi = M_SAP eta: n_cy SAP cycles from psi = 0 with nmr MR steps per block
 * solve (Sec. 2.2, M_SAP = K sum_{nu<n_cy} (1 - D K)^nu, inexact blocks).
 * Device canonical spinors, precision F64 or F32. */
qcd_status qcd_apply_sap(qcd_ctx* ctx, const double* eta, double* psi, int nrhs, int precision);

/* Solve D psi = eta for nrhs device canonical spinors with SAP-preconditioned
 * flexible GCR (Sec. 2.2: D M_SAP phi = eta, psi = M_SAP phi).  psi holds the
 * initial guess on entry (zeros for none).  rel_tol is a host array of nrhs
 * tolerances.  stats (host, nrhs entries) may be NULL.  Returns QCD_OK when
 * every RHS converged, else QCD_ERR_NOT_CONVERGED (psi = best iterates). */
qcd_status qcd_solve(qcd_ctx* ctx, const double* eta, double* psi, int nrhs, const double* rel_tol,
                     qcd_rhs_stats* stats);

/* Several lattices (contexts of different sizes) solved in one call: each
 * context's solve runs from its own host thread on its own stream, so the
 * lattices' kernels overlap on the GPU.  Arrays of nctx entries; eta[i],
 * psi[i] device canonical spinors of ctxs[i], rel_tol[i] host arrays of
 * nrhs[i] tolerances, stats[i] host arrays or stats == NULL.  With nctx > 1
 * every context needs a non-default stream.  Returns the first non-OK status
 * in context order.  Errors of a context do not stop the others. */
qcd_status qcd_solve_multi(qcd_ctx* const* ctxs, int nctx, const double* const* eta, double* const* psi,
                           const int* nrhs, const double* const* rel_tol, qcd_rhs_stats* const* stats);

/* Nucleon two-point function (eq. Nop, N = eps^{abc} (u^a^T C g5 d^b) u^c,
 * C = g0 g2, u = d) from one point-source propagator prop (device,
 * canonical, 12 spinors rhs = 3*spin + colour) with source src = {t,x,y,z}:
 *   corr[p][t][re/im], p = 0: tr[P+ G], p = 1: tr[P- G], P+- = (1 +- g0)/2,
 *   G(t) = sum_{x-vec} <N(x,t) N-bar(src)>, t relative to the source time;
 *   a sink time that wraps past T is multiplied by time_bc^3.
 * corr is host memory of 2*T*2 doubles.  precision selects FP64 or FP32
 * arithmetic. */
qcd_status qcd_nucleon_2pt(qcd_ctx* ctx, const double* prop, const int src[4], double* corr, int precision);

/* AMA estimate of the nucleon two-point function (eqs. caa1, caa2):
 *   O_AMA = (1/N_org) sum_f [O^f - O_appx^f] + (1/N_G) sum_g O_appx^g.
 * For each of n_src source positions src[4*i..] the 12 spin-colour point
 * sources are solved to sloppy_tol; the first n_exact positions are also
 * solved to exact_tol (the bias correction, N_org = n_exact).  Positions must
 * be multiples of the SAP block extents, and differ from the first source by
 * an even number of blocks, so that the translations map each of the SAP
 * domains Omega and Omega* onto itself (Sec. 2.2, end).  The exact solve of a
 * source starts from its sloppy solution (its iteration counts in stats are
 * the additional iterations).
 *   corr_ama  host [2][T][2]          the AMA estimate
 *   corr_all  host [n_src + n_exact][2][T][2] or NULL: sloppy correlators
 *             of every source, then exact correlators of the first n_exact
 *   stats     host [(n_src + n_exact) * 12] or NULL, same order. */
qcd_status qcd_ama_nucleon_2pt(qcd_ctx* ctx, const int* src, int n_src, int n_exact, double sloppy_tol,
                               double exact_tol, double* corr_ama, double* corr_all, qcd_rhs_stats* stats);

/* Nucleon three-point functions with the isovector insertions of the
 * axial, scalar and tensor charges (Sec. 2.3, eqs. R_A, R_S, R_T):
 *   C3_O(t) = sum_{x at t_s, y at t} tr[P <N(x) O(y) N-bar(src)>],
 *   O = u-bar Gamma u - d-bar Gamma d (connected insertions, u = d),
 * for O = A_3 (Gamma = g3 g5, P = P53 = P g5 g3), S (Gamma = 1, P) and T_12
 * (Gamma = sigma_12, P53), with P = P+ = (1 + g0)/2 for direction = +1
 * (sink at src_t + t_sep) and P = P- = (1 - g0)/2 for direction = -1 (sink at
 * src_t - t_sep, the backward-propagating nucleon), times modulo T.
 * Method: sequential propagators through the sink (12 solves per projector,
 * 24 in all, to the relative tolerance tol with the context's solver).
 * Point sink (smeared sinks: qcd_ama_nucleon with qcd_set_smearing).
 *   prop   device, canonical FP64: the 12 spinors of the point source at src
 *          (rhs = 3 spin + colour), solutions of D psi = eta as qcd_solve
 *          returns them (kappa normalisation).
 *   t_sep  source-sink separation, 1 <= t_sep < T.
 *   corr3  host [3][T][2]: insertion (A_3, S, T_12), operator time relative to
 *          the source, re/im.  Times and the boundary sign follow
 *          qcd_nucleon_2pt: a sink earlier than the source in absolute time is
 *          multiplied by time_bc^3, so C3 / C2 pairs values of one convention;
 *          the ratios of Wilson-normalised propagators are
 *          R = 2 kappa C3(t) / C2(t_sep), C2 from qcd_nucleon_2pt (P+ or P-).
 *   stats  host, 24 entries (sequential solves: P, then P53) or NULL.
 * Returns QCD_ERR_NOT_CONVERGED if a sequential solve did not converge (corr3
 * is still written). */
qcd_status qcd_nucleon_3pt(qcd_ctx* ctx, const double* prop, const int src[4], int t_sep, int direction, double tol,
                           double* corr3, qcd_rhs_stats* stats);

/* All-mode averaging of the nucleon two- and three-point functions
 * (Sec. 2.1, eqs. caa1, caa2), with the sloppy solves either to a relative
 * tolerance or, as in the paper's production runs (Sec. 3, Table 3), with a
 * fixed number N_iter of GCR iterations, separately for the point-source
 * propagators (2pt) and the sequential propagators (3pt).
 *   n_exact     N_org: the first n_exact source positions are also solved to
 *               exact_tol (the bias correction); their point-source solves
 *               start from the sloppy solutions.
 *   sloppy_tol, exact_tol   relative tolerances in (0, 1); sloppy_tol is used
 *               where the corresponding n_iter is 0.
 *   n_iter_2pt  > 0: every sloppy point-source solve runs exactly this many
 *               GCR iterations (no tolerance; not an error).
 *   n_iter_3pt  > 0: every sloppy sequential solve likewise.
 *   t_sep       0: two-point functions only; 1 <= t_sep < T: also the
 *               three-point functions of qcd_nucleon_3pt with this separation.
 *   direction   +1 / -1: sink at src_t +- t_sep (P+ / P-), as qcd_nucleon_3pt. */
typedef struct {
  int n_exact;
  double sloppy_tol;
  double exact_tol;
  int n_iter_2pt;
  int n_iter_3pt;
  int t_sep;
  int direction;
} qcd_ama_params;

/* src: host [n_src][4] source positions (multiples of the SAP block extents,
 * differing from src[0] by an even number of blocks, as qcd_ama_nucleon_2pt).
 *   c2_ama  host [2][T][2]          AMA estimate of the two-point function
 *                                   (P+, P-; layout of qcd_nucleon_2pt)
 *   c3_ama  host [3][T][2] or NULL  AMA estimate of the three-point functions
 *                                   (needed when t_sep > 0; layout of qcd_nucleon_3pt)
 *   c2_all  host [n_src + n_exact][2][T][2] or NULL: sloppy correlators of
 *           every position, then exact ones of the first n_exact
 *   c3_all  host [n_src + n_exact][3][T][2] or NULL, same order
 *   stats   host [n_src + n_exact][12 (+ 24 with t_sep)] or NULL: point-source
 *           solves, then the sequential solves of each position
 * Work is stream-ordered on the context's stream; the call returns after the
 * correlators are on the host.  Returns the first non-OK status of a solve
 * (a fixed-iteration solve that stops at N_iter counts as OK). */
qcd_status qcd_ama_nucleon(qcd_ctx* ctx, const int* src, int n_src, const qcd_ama_params* p, double* c2_ama,
                           double* c3_ama, double* c2_all, double* c3_all, qcd_rhs_stats* stats);

/* The error model of the AMA estimator (eqs. ama1-ama3; host computation,
 * no device work) from measurements of one observable on n_conf gauge
 * configurations: exact [n_conf][n_org] (O^f), appx_org [n_conf][n_org]
 * (O_appx^f at the same positions), appx [n_conf][n_g] (O_appx^g).  With
 * sample covariances over the configurations,
 *   out[0] = Delta r = (1/N_org - 1/N_G) (1 - (1/N_org) sum_f corr(O^f, O_appx^f))
 *   out[1] = R = (1/N_G^2) sum_{g != g'} corr(O_appx^g, O_appx^g')
 *   out[2] = sqrt(1/N_G + 2 Delta r + R), the model of sigma_AMA / sigma
 *   out[3] = the measured std(O_AMA) / sqrt(mean_f var(O^f)).
 * QCD_ERR_ARG if n_conf < 2, n_org > n_g or a measurement has zero variance. */
qcd_status qcd_ama_error_model(const double* exact, const double* appx_org, const double* appx, int n_conf,
                               int n_org, int n_g, double* out);

/* Smeared sources and sinks (Sec. 2.3: Gaussian smearing at source and sink
 * with APE-smeared links in the Laplacian; the paper takes the parameters
 * from earlier work, so they are the caller's).
 * qcd_smear_links: APE-smeared spatial links from the loaded gauge field,
 *   n_ape steps of U'_k(x) = Proj_SU(3)[U_k(x) + alpha sum_{j != k spatial}
 *   (U_j(x) U_k(x+j) U_j(x+k)^+ + U_j(x-j)^+ U_k(x-j) U_j(x-j+k))], Proj_SU(3)
 *   the unitary polar factor divided by the principal cube root of its
 *   determinant; time links unchanged.  Kept in the context (FP64); loading a
 *   new gauge field does not update them.  alpha >= 0, 0 <= n_ape <= 1000.
 * qcd_set_smearing: Gaussian kernel K = [(1 + kappa_g H) / (1 + 6 kappa_g)]^n_gauss,
 *   H the spatial hopping term on the smeared links (spin untouched,
 *   periodic in space); qcd_ama_nucleon then smears its point sources and
 *   the sink index of its propagators (n_gauss = 0: point source and sink).
 *   Needs qcd_smear_links first when n_gauss > 0.
 * qcd_smear_gaussian: out = K in for nrhs device canonical spinors.
 * qcd_get_smeared_links: the smeared links as a device canonical FP64 gauge
 *   field [site][mu][3][3]. */
qcd_status qcd_smear_links(qcd_ctx* ctx, double alpha, int n_ape);
qcd_status qcd_set_smearing(qcd_ctx* ctx, double kappa_g, int n_gauss);
qcd_status qcd_smear_gaussian(qcd_ctx* ctx, const double* in, double* out, int nrhs);
qcd_status qcd_get_smeared_links(qcd_ctx* ctx, double* out);

/* The site-diagonal part A(x) = 1 + i kappa c_sw sum sigma F of the operator
 * (the O(a)-improvement (clover) term of Sec. 2.2's Wilson-clover operator)
 * as [site][chirality 2][6][6] complex FP64 (device), chirality block 0 acting
 * on spins 0,1 and block 1 on spins 2,3, index 3*(spin & 1) + colour. */
qcd_status qcd_get_clover(qcd_ctx* ctx, double* out);

/* Differentiable nucleon correlator (Feynman-Hellmann).  Wilson normalisation:
 * D_w = D / (2 kappa), kappa = 1 / (2 m0 + 8), S = D_w^-1; the isovector axial
 * coupling adds +lambda g3 g5 to D_w for u and -lambda g3 g5 for d (the
 * zero-momentum A_3 insertion of R_A, Sec. 2.3), taken at lambda = 0.
 * qcd_fh_forward: solves the 12 point sources at src to tol, writes S (device,
 * canonical FP64, 12 spinors) and C = tr[P+- <N N-bar>] (host [2][T][2], FP64,
 * from S) as qcd_nucleon_2pt; stats: 12 entries or NULL.
 * qcd_fh_gradient: for the upstream gradient gcorr (host [2][T][2]: dL/dRe C,
 * dL/dIm C) of a real loss L, returns grad = {dL/dm0, dL/dlambda} (host) by the
 * adjoint method: H = dL/dS from the contraction, Y = (D_w^+)^-1 H
 * = 2 kappa g5 D^-1 g5 H (24 solves: u and d), dL/dtheta = -Re sum tr[Y^+ dD_w S].
 * prop is the S returned by qcd_fh_forward; stats: 24 entries or NULL. */
qcd_status qcd_fh_forward(qcd_ctx* ctx, const int src[4], double tol, double* prop, double* corr,
                          qcd_rhs_stats* stats);
qcd_status qcd_fh_gradient(qcd_ctx* ctx, const double* prop, const int src[4], const double* gcorr, double tol,
                           double* grad, qcd_rhs_stats* stats);

/* Autotuner (no counterpart in the paper; implementation parameters only).
 * Times a solve of the nrhs device canonical sources eta to tol for each
 * candidate SAP block shape (4^4, 8x4^3, 4^3x8, 4x8x4^2 where they tile the
 * lattice), 16- or 32-bit SAP block copies, nkv in {16, 32} and rhs_tile in
 * {nrhs, nrhs/2}, keeping ncy, nmr, precision and deflation as set; the
 * fastest converged candidate becomes the context's parameters and is
 * written to *best (may be NULL).  cache_path (may be NULL): a text file of
 * earlier results, keyed by lattice, couplings, tolerance, nrhs and GPU name;
 * a hit skips the timing.  Changing the block shape discards a deflation
 * subspace.  Allocates one nrhs-spinor work buffer for the duration of the
 * call. */
qcd_status qcd_autotune(qcd_ctx* ctx, const double* eta, int nrhs, double tol, const char* cache_path,
                        qcd_solver_params* best);

/* Allocation-free nucleon two-point function (no counterpart in the paper:
 * an interface for callers that cannot allocate device memory where they
 * need the correlator - inside a stream capture, under a host application's
 * own device allocator or fixed arena, or in a loop that must not take an
 * allocation's implicit synchronisation).  It computes what qcd_nucleon_2pt
 * computes, needs no context, and calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *   dims {T, X, Y, Z}; time_bc +1 / -1; prop: device, canonical FP64, the 12
 *   spinors of a point source (rhs = 3*spin + colour); src {t, x, y, z};
 *   corr: DEVICE memory of 2*T*2 doubles, [p][t][re/im] as in qcd_nucleon_2pt;
 *   precision QCD_PREC_F64 or QCD_PREC_F32; cuda_stream: the stream to use.
 * The work is only enqueued on cuda_stream; corr is ready when it completes.
 * Scratch: a fixed 4 MiB device array inside the library (resident on every
 * GPU that loads it until the process exits) holds the per-CTA partial sums,
 * which limits the lattice to V / ns <= 131072, ns being the largest power of
 * two <= 32 dividing X*Y*Z (e.g. up to 4,194,304 sites when 32 divides X*Y*Z);
 * larger lattices return QCD_ERR_ARG before any launch.  The first call on a
 * device looks up the array's device address (and sets kernel attributes); make
 * that first call before capturing a stream.  All calls share the array:
 * calls that overlap on the GPU (different streams, not ordered) race on it
 * and give wrong results. */
qcd_status qcd_nucleon_2pt_noalloc(const int dims[4], int time_bc, const double* prop, const int src[4],
                                   double* corr, int precision, void* cuda_stream);

/* Local deflation (Sec. 2.2).  Builds the deflation subspace on the SAP
 * blocks from ns random global fields init (device, canonical FP64, ns
 * spinors; the caller draws them): block Gram-Schmidt, then n_inv rounds of
 * the inverse iteration phi -> M_SAP phi followed by block Gram-Schmidt; then
 * the little Dirac operator A = (phi_k^b, D phi_l^b') (eq. little) on the
 * block and its 8 neighbours (tensor-core GEMMs, FP32-accurate products,
 * compensated sums, FP64 storage), and the FP64 Gauss-Jordan inverses of its
 * diagonal blocks; FP32 copies of both serve the little solve of the
 * deflated preconditioner.  QCD_ERR_TIMEOUT if the tensor-core build gave up
 * waiting for its matrix multiplies (a bounded wait; nothing is left
 * running).  1 <= ns <= 32; SAP block extents >= 2 in every direction.  Setting new parameters with a different block size discards
 * the subspace.  Returns QCD_ERR_BREAKDOWN if a diagonal block is singular. */
qcd_status qcd_deflation_setup(qcd_ctx* ctx, const double* init, int ns, int n_inv);
/* The deflation fields as ns canonical FP64 spinors (device). */
qcd_status qcd_deflation_fields(qcd_ctx* ctx, double* out);
/* The little Dirac operator (stored in FP64) as host FP64 complex
 * [block][9][ns][ns]: part 0
 * couples a block to itself, 1 + 2 mu to its neighbour at +mu, 2 + 2 mu to
 * the one at -mu; blocks are numbered ((bt*nbz + bz)*nby + by)*nbx + bx. */
qcd_status qcd_deflation_little_matrix(qcd_ctx* ctx, double* out);
/* Little vectors (host FP64 complex [n][block][ns], rounded to FP32 on the
 * device): mode 0: out = A in with the FP64 A (FP64 sums); mode 1: out = the
 * m-step block-Jacobi preconditioned GCR approximation of A^-1 in that the
 * preconditioner uses (FP32 copies of A and the block inverses). */
qcd_status qcd_deflation_little(qcd_ctx* ctx, const double* in, double* out, int n, int mode, int m);

/* Kernel timing (no counterpart in the paper; measurement support).  While
 * enabled, every kernel launch of the library on the context's stream is
 * bracketed by CUDA events.  qcd_profile_read synchronises the stream and
 * returns, per kernel family, the launches, their summed device time and
 * the algorithmic bytes they had to move (each input word read once, each
 * output word written once), then clears the records.
 * Families: "dslash_f64", "dslash_f32", "sap_f64", "sap_f32", "blas",
 * "layout", "contract", "deflation". */
typedef struct {
  char name[24];
  int launches;
  double ms;
  double bytes;
  double flops;
} qcd_kernel_time;

qcd_status qcd_profile_enable(qcd_ctx* ctx, int on);
/* out: host array of max entries; *n receives the number of families filled. */
qcd_status qcd_profile_read(qcd_ctx* ctx, qcd_kernel_time* out, int max, int* n);

#ifdef __cplusplus
}
#endif

#endif /* QCD_GB300_H */
