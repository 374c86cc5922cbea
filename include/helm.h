/*
 * helm.h -- C ABI of the GB300 frequency-domain FWI library.
 *
 * The library evaluates the reduced least-squares objective of the paper
 * (Da Silva & Herrmann, "A Unified 2D/3D Large Scale Software Environment for
 * Nonlinear Inverse Problems", Sec. 2, eq. (mainprob))
 *
 *     f(m) = sum_{w} sum_{s} 1/2 || P_r H_w(m)^{-1} q_{s,w} - d_{s,w} ||^2
 *
 * and its adjoint-state gradient (Appendix A, eqs. (dU2), (dH), (dHadj);
 * Table derivstuff; Listing pdefunc, OBJ branch)
 *
 *     u = H^{-1} q,   v = -H^{-H} P_r^T (P_r u - d),   g = E^T sum w^2 Re(conj(u) v),
 *
 * where H(m,w) = Lap_eta + w^2 diag(m) is the 7-point (5-point in 2D) finite-
 * difference Helmholtz operator of Sec. 2 (eq. (helmholtz) on the extended
 * domain with damping layers), m = 1/v^2, and E copies the physical model
 * into the layers along the normal direction (its adjoint E^T sums back).
 * Solves are matrix-free: restarted FGMRES (Sec. 4) with the multi-level
 * ML-GMRES preconditioner of Sec. 4 (Alg. vcycle; Fig. mlgmres) or damped
 * Jacobi, in FP64 or with complex64 inner solves under FP64 iterative
 * refinement.  Around the objective the library offers the operator and
 * preconditioner applies, forward and adjoint modelling, the linearised
 * products of Table derivstuff (J dm, J^T dD, the Gauss-Newton and the full
 * Hessian-vector products) and 2.5D modelling (Sec. 3).
 *
 * Conventions for every call
 *  - Bulk arrays are DEVICE pointers owned by the caller; the library never
 *    allocates, frees or keeps them.  Scalars, option structs, frequency lists
 *    and report arrays are HOST memory.
 *  - Complex values are interleaved (re, im): complex128 = two doubles,
 *    complex64 = two floats.
 *  - Grid fields are x-fastest: physical [nz][ny][nx] (n_phys values) and
 *    computational [Nz][Ny][Nx] (n_comp values, layers included).  2D uses
 *    ny = 1.  Node indices are PHYSICAL linear indices ix + nx*(iy + ny*iz).
 *  - Multi-field arrays are [nfreq][nsrc][...] (frequency slowest).
 *  - `workspace` is caller-allocated device scratch of at least the size that
 *    helm_workspace_size() reports for the same call and sizes, 256-byte aligned.
 *  - Calls are enqueued on `stream` but BLOCK the host: the solvers read
 *    per-RHS convergence state between restart cycles, so every output is
 *    complete when a call returns.  Calls on one plan must not overlap.
 *  - Return value: HELM_OK or a negative helm_status.  HELM_E_NOCONV still
 *    writes every output; the per-RHS reports say which solves fell short.
 */
#ifndef HELM_H
#define HELM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t-compatible handle (NULL = the legacy default stream). */
typedef struct CUstream_st* helm_stream_t;

typedef enum {
  HELM_OK = 0,
  HELM_E_INVAL = -1,     /* bad sizes, options, pointers or node indices */
  HELM_E_NOMEM = -2,     /* workspace smaller than helm_workspace_size() */
  HELM_E_CUDA = -3,      /* a CUDA runtime call or kernel launch failed */
  HELM_E_NOCONV = -4,    /* some solve missed its tolerance (outputs written) */
  HELM_E_NONFINITE = -5, /* NaN/Inf met in a residual */
  HELM_E_TIMEOUT = -6,   /* a kernel gave up on a bounded wait for its bulk copies; outputs are void */
  HELM_E_BOUNDS = -7     /* debug build (HELM_DEBUG) only: a kernel wrote into the guard band after a
                            workspace array, or a slot index was out of range; outputs are void */
} helm_status;

typedef enum { HELM_FP64 = 0, HELM_MIXED = 1 } helm_precision;
/* Element type of stored forward fields (helm_misfit / helm_gradient). */
typedef enum { HELM_FIELD_C128 = 0, HELM_FIELD_C64 = 1 } helm_field_type;
typedef enum { HELM_PRECOND_NONE = 0, HELM_PRECOND_JACOBI = 1, HELM_PRECOND_MLGMRES = 2 } helm_precond;
typedef enum {
  HELM_CALL_APPLY = 0, HELM_CALL_FORWARD = 1, HELM_CALL_ADJOINT = 2, HELM_CALL_MISFIT_GRAD = 3,
  HELM_CALL_MISFIT = 4, HELM_CALL_GRADIENT = 5, HELM_CALL_PRECOND = 6, HELM_CALL_BORN = 7,
  HELM_CALL_BORN_ADJOINT = 8, HELM_CALL_GN_HESSVEC = 9, HELM_CALL_HESSVEC = 10, HELM_CALL_MISFIT_GRAD_25D = 11,
  HELM_CALL_WRI = 12
} helm_call;

/* Geometry of the extended domain (Sec. 2: Omega' contains Omega; "PDEopts"
 * of Sec. 3 carries the layer width).  The damping profile is
 * sigma(x) = sigma_max (dist(x)/W)^2 across a layer of width W, and the
 * stretched derivative is (1/eta) d/dx with eta = 1 + i sigma / w. */
typedef struct {
  int dim;               /* 2 or 3 */
  int n[3];              /* physical nodes along x, y, z (dim 2: n[1] = 1) */
  double h;              /* node spacing [m] */
  int npml[3];           /* damping-layer cells on each side (dim 2: npml[1] = 0) */
  double v_ref;          /* velocity [m/s] setting the default sigma_max */
  double sigma_max[3];   /* 0 selects 3 v_ref ln(1000) / (2 npml h) */
  int levels;            /* 1..3 grid levels; with levels > 1 extra high-side layer
                            cells make N_d + 1 divisible by 2^(levels-1) */
} helm_grid;

/* Solver options ("LinSolveOpts" of Sec. 3; ML-GMRES parameters
 * (k_so, k_si, k_co, k_ci) of Sec. 4). */
typedef struct {
  int precision;         /* helm_precision */
  int precond;           /* helm_precond */
  int k_inner;           /* Krylov length of one outer FGMRES restart cycle (1..32) */
  int max_cycles;        /* outer restart cycles per solve (per refinement step) */
  double tol;            /* target ||q - H u|| / ||q||, checked in FP64 */
  double tol_inner;      /* MIXED: residual reduction asked of each complex64 solve */
  int max_refine;        /* MIXED: iterative-refinement steps */
  int k_so, k_si;        /* ML-GMRES smoother GMRES: cycles, Krylov length */
  int k_co, k_ci;        /* ML-GMRES coarse FGMRES: cycles, Krylov length */
  double jacobi_omega;   /* damped-Jacobi weight */
  int jacobi_sweeps;     /* damped-Jacobi sweeps per preconditioner application */
  int max_batch;         /* right-hand sides solved together (0 = all at once) */
  int reorth;            /* 1: Gram-Schmidt with one re-orthogonalisation pass (CGS2);
                            0: a single classical Gram-Schmidt pass */
  int sstep;             /* 1: the fixed-cycle GMRES solves (ML-GMRES smoothers and the
                            last-level coarse solve) build their Krylov basis with s = k
                            operator applications and solve the same minimal-residual
                            problem through its Gram matrix (s-step GMRES; k <= 8);
                            0: Arnoldi with Gram-Schmidt for every solve */
} helm_solve_opts;

/* One report per right-hand side (frequency-major, like the fields). */
typedef struct {
  int status;            /* HELM_OK, HELM_E_NOCONV or HELM_E_NONFINITE */
  int iters;             /* outer Krylov iterations summed over refinement steps */
  int refinements;       /* MIXED: refinement steps taken (FP64: 1) */
  double rel_resid;      /* final ||q - H u|| / ||q|| in FP64 */
} helm_rhs_report;

typedef struct helm_plan helm_plan;

/* Fill `opts` with the defaults: MIXED, ML-GMRES (3,5,3,5) with s-step
 * smoothers, outer FGMRES(10) with CGS2, tol 1e-10, tol_inner 0.1 (about one
 * complex64 FGMRES cycle per FP64 refinement step), max_refine 60.
 * Returns HELM_OK. */
int helm_default_opts(helm_solve_opts* opts);

/* Validate `grid` and `opts` and build a host-side plan (no device memory).
 * HELM_E_INVAL on a bad field; *plan is NULL then. */
int helm_plan_create(const helm_grid* grid, const helm_solve_opts* opts, helm_plan** plan);
void helm_plan_destroy(helm_plan* plan);

/* Computational sizes N[3] (layers and padding included), n_comp = N0*N1*N2
 * and n_phys = n0*n1*n2. */
int helm_plan_dims(const helm_plan* plan, int N[3], size_t* n_comp, size_t* n_phys);

/* Device workspace in bytes needed by `call` for the given sizes
 * (n_rhs = nfreq*nsrc fields; nrec receivers). */
int helm_workspace_size(const helm_plan* plan, int call, int nfreq, int nsrc, int nrec,
                        size_t* bytes);

/* y = H(m, w) x, or y = H(m, w)^H x when `adjoint` != 0, for `nrhs` fields on
 * the computational grid sharing m and w = 2 pi freq_hz (Sec. 2 operator; its
 * adjoint is the conjugate transpose, Sec. 5.1 adjoint test).  precision
 * HELM_FP64: x, y complex128; HELM_MIXED: x, y complex64 (FP32 arithmetic).
 * m_phys: float64 [n_phys].  x and y must not overlap. */
int helm_apply(helm_plan* plan, const double* m_phys, double freq_hz, int adjoint, int precision,
               const void* x, void* y, int nrhs, void* workspace, size_t ws_bytes,
               helm_stream_t stream);

/* z = M^{-1} x: one application of the plan's preconditioner to each of
 * `nrhs` fields at one frequency (Sec. 4): with HELM_PRECOND_MLGMRES one
 * ML-GMRES V-cycle from a zero guess (pre-smoothing by k_so restarted cycles of
 * GMRES(k_si), the residual restricted by full weighting, the rediscretised
 * coarse problem at spacing 2h solved by k_co cycles of (F)GMRES(k_ci) --
 * preconditioned by the next level's V-cycle when there is one -- its
 * solution prolonged by linear interpolation and added, post-smoothing as
 * before); with HELM_PRECOND_JACOBI `jacobi_sweeps` damped Jacobi sweeps from
 * zero; with HELM_PRECOND_NONE a copy.  `adjoint` != 0 preconditions H^H
 * instead (the same cycle on the adjoint operators).  Fields are in the
 * plan's precision: complex128 [nrhs][n_comp] for HELM_FP64, complex64 for
 * HELM_MIXED (the same types as helm_apply).  x is read only; z is written.
 * The cycle is a nonlinear function of x when its smoothers are GMRES.
 * Workspace: helm_workspace_size(plan, HELM_CALL_PRECOND, 1, nrhs, 0, ...);
 * max_batch bounds the fields processed together. */
int helm_precond_apply(helm_plan* plan, const double* m_phys, double freq_hz, int adjoint, const void* x,
                       void* z, int nrhs, void* workspace, size_t ws_bytes, helm_stream_t stream);

/* Forward modelling (Listing pdefunc, FORW_MODEL): for every frequency k and
 * source s solve H(m, w_k) u = q with q = wavelet[k] sum_j Q[j, s] delta_h(x - x_j),
 * delta_h = 1/h^dim at the node src_idx[j], then D = P_r u (u sampled at rec_idx).
 *   m_phys   float64 [n_phys]
 *   freqs_hz HOST float64 [nfreq]
 *   src_idx  int32 [n_srcloc]; Q complex128 [n_srcloc][nsrc]
 *   wavelet  complex128 [nfreq] or NULL (all ones)
 *   rec_idx  int32 [nrec]
 *   U0       complex128 [nfreq][nsrc][n_comp] or NULL: initial guesses (a warm
 *            start, e.g. the fields of a nearby model, as when an inversion
 *            moves on between model updates or frequency bands); the solves
 *            start from zero when NULL.  A guess whose residual already meets
 *            the tolerance is returned unchanged after no iteration.  U0 may
 *            be the same array as U_out.
 *   U_out    complex128 [nfreq][nsrc][n_comp] or NULL
 *   D_out    complex128 [nfreq][nsrc][nrec] or NULL
 *   reports  HOST [nfreq*nsrc] or NULL */
int helm_forward(helm_plan* plan, const double* m_phys, const double* freqs_hz, int nfreq,
                 const int32_t* src_idx, int n_srcloc, const void* Q, int nsrc,
                 const void* wavelet, const int32_t* rec_idx, int nrec, const void* U0,
                 void* U_out, void* D_out, void* workspace, size_t ws_bytes,
                 helm_rhs_report* reports, helm_stream_t stream);

/* Adjoint solve: V = H(m, w_k)^{-H} P_r^T R for every frequency and source
 * (the adjoint wavefield of Table derivstuff without its minus sign).
 *   R_in  complex128 [nfreq][nsrc][nrec];  V_out complex128 [nfreq][nsrc][n_comp] */
int helm_adjoint(helm_plan* plan, const double* m_phys, const double* freqs_hz, int nfreq,
                 const int32_t* rec_idx, int nrec, const void* R_in, int nsrc, void* V_out,
                 void* workspace, size_t ws_bytes, helm_rhs_report* reports,
                 helm_stream_t stream);

/* Misfit and gradient (Sec. 2 eq. (mainprob); Appendix A; Listing pdefunc OBJ):
 *   f = sum_{k,s} 1/2 ||P_r u_{k,s} - d_{k,s}||^2,
 *   g = E^T sum_{k,s} w_k^2 Re(conj(u_{k,s}) v_{k,s}),  v = -H^{-H} P_r^T (P_r u - d),
 * over the (k, s) pairs whose mask byte is non-zero (all when mask is NULL; the
 * paper's batch-mode source/frequency subsets, Sec. 3).
 *   d_obs   complex128 [nfreq][nsrc][nrec]
 *   mask    uint8 [nfreq][nsrc] or NULL
 *   f_out   float64 [1];  g_out float64 [n_phys] (overwritten) */
int misfit_and_gradient(helm_plan* plan, const double* m_phys, const double* freqs_hz, int nfreq,
                        const int32_t* src_idx, int n_srcloc, const void* Q, int nsrc,
                        const void* wavelet, const int32_t* rec_idx, int nrec,
                        const void* d_obs, const uint8_t* mask, double* f_out, double* g_out,
                        void* workspace, size_t ws_bytes, helm_rhs_report* reports,
                        helm_stream_t stream);

/* Linearised modelling (Appendix A eqs. (dU2), (dH), (dHadj) with A = I;
 * Table derivstuff).  For every selected (k, s) pair the state
 * u = H(m, w_k)^{-1} q_{k,s} is solved first (sources, wavelet and receivers as
 * in helm_forward, mask as in misfit_and_gradient; masked-out pairs
 * contribute nothing), then:
 *
 * helm_born:          dD = J dm = P_r du with H du = -w_k^2 (E dm) u
 *                     (two solves per pair).
 *     dm_phys  float64 [n_phys];  dD_out complex128 [nfreq][nsrc][nrec]
 *     (rows of masked-out pairs are zero)
 * helm_born_adjoint:  g = J^T dD = E^T sum_{k,s} w_k^2 Re(conj(u) v),
 *                     v = -H^{-H} P_r^T dD_{k,s} (two solves per pair; with
 *                     dD = P_r u - d it is the misfit gradient).
 *     dD_in    complex128 [nfreq][nsrc][nrec];  g_out float64 [n_phys]
 * helm_gn_hessvec:    Hdm = J^T J dm, the Gauss-Newton Hessian applied to dm
 *                     (three solves per pair).
 *     dm_phys  float64 [n_phys];  Hdm_out float64 [n_phys]
 *
 * J is taken with respect to the physical m (real), so J^T is the adjoint
 * for the real inner product Re<J dm, dD> = <dm, J^T dD>.  reports (HOST,
 * [nfreq*nsrc] or NULL) add the iterations of the pair's solves and keep the
 * worst residual and status.  Workspace: helm_workspace_size with
 * HELM_CALL_BORN / HELM_CALL_BORN_ADJOINT / HELM_CALL_GN_HESSVEC. */
int helm_born(helm_plan* plan, const double* m_phys, const double* freqs_hz, int nfreq,
              const int32_t* src_idx, int n_srcloc, const void* Q, int nsrc, const void* wavelet,
              const int32_t* rec_idx, int nrec, const double* dm_phys, const uint8_t* mask,
              void* dD_out, void* workspace, size_t ws_bytes, helm_rhs_report* reports,
              helm_stream_t stream);
int helm_born_adjoint(helm_plan* plan, const double* m_phys, const double* freqs_hz, int nfreq,
                      const int32_t* src_idx, int n_srcloc, const void* Q, int nsrc,
                      const void* wavelet, const int32_t* rec_idx, int nrec, const void* dD_in,
                      const uint8_t* mask, double* g_out, void* workspace, size_t ws_bytes,
                      helm_rhs_report* reports, helm_stream_t stream);
int helm_gn_hessvec(helm_plan* plan, const double* m_phys, const double* freqs_hz, int nfreq,
                    const int32_t* src_idx, int n_srcloc, const void* Q, int nsrc,
                    const void* wavelet, const int32_t* rec_idx, int nrec, const double* dm_phys,
                    const uint8_t* mask, double* Hdm_out, void* workspace, size_t ws_bytes,
                    helm_rhs_report* reports, helm_stream_t stream);

/* Full Hessian of the misfit applied to dm (Table derivstuff, last row;
 * Appendix A with A = I and the least-squares phi, whose Hessian is the
 * identity).  Four solves per selected (k, s) pair:
 *   u  = H^{-1} q,   v = -H^{-H} P_r^T (P_r u - d),   du = -H^{-1} w^2 (E dm) u,
 *   dv = H^{-H} ( -w^2 (E dm) v - P_r^T P_r du ),
 *   Hdm = E^T sum_{k,s} w_k^2 Re( conj(du) v + conj(u) dv ).
 * Arguments as helm_gn_hessvec plus d_obs (complex128 [nfreq][nsrc][nrec], as
 * misfit_and_gradient).  At zero data residual it equals helm_gn_hessvec.
 * Workspace: helm_workspace_size with HELM_CALL_HESSVEC. */
int helm_hessvec(helm_plan* plan, const double* m_phys, const double* freqs_hz, int nfreq,
                 const int32_t* src_idx, int n_srcloc, const void* Q, int nsrc, const void* wavelet,
                 const int32_t* rec_idx, int nrec, const void* d_obs, const double* dm_phys,
                 const uint8_t* mask, double* Hdm_out, void* workspace, size_t ws_bytes,
                 helm_rhs_report* reports, helm_stream_t stream);

/* 2.5D misfit and gradient (Sec. 3, 2.5D): a model invariant in y on a 2D
 * plan (dim = 2, the grid is (x, z)); the y-Fourier transform turns each
 * frequency into 2D problems H(k_i) u~_i = q with H(k) = H(m, w) - k^2 I (no
 * layer in y), and the data are the quadrature sum
 *   D_{k,s} = sum_i ck[i] P_r u~_{k,s,i},
 * with ck[i] = (quadrature weight) cos(k_i dy) / pi supplied by the caller
 * (e.g. Gauss-Legendre on [0, p w / v_min], dy = receiver y - source y).
 *   f = sum_{k,s} 1/2 ||D_{k,s} - d_{k,s}||^2,
 *   g = E^T sum_{k,s,i} w_k^2 Re(conj(u~_i) v_i),  v_i = -H(k_i)^{-H} P_r^T (ck[i] r_{k,s}).
 *   ky, ck   HOST float64 [nk] (wavenumbers in rad/m, weights)
 *   d_obs    complex128 [nfreq][nsrc][nrec]; wavelet as helm_forward
 *   f_out    float64 [1]; g_out float64 [n_phys] of the 2D plan
 *   reports  HOST [nfreq][nsrc][nk] or NULL
 * The nk solves of one (frequency, source) run in the same batch, so
 * max_batch must be 0 or at least nk.  Workspace: helm_workspace_size with
 * HELM_CALL_MISFIT_GRAD_25D and nfreq*nk in place of nfreq. */
int helm_misfit_and_gradient_25d(helm_plan* plan, const double* m_phys, const double* freqs_hz, int nfreq,
                                 const double* ky, const double* ck, int nk, const int32_t* src_idx,
                                 int n_srcloc, const void* Q, int nsrc, const void* wavelet,
                                 const int32_t* rec_idx, int nrec, const void* d_obs, double* f_out,
                                 double* g_out, void* workspace, size_t ws_bytes, helm_rhs_report* reports,
                                 helm_stream_t stream);

/* Waveform Reconstruction Inversion objective and gradient (Sec. 3 penalty
 * method, eqs. (wri), (wrifieldeq); Appendix B).  For every (k, s) pair the
 * field u minimises ||P_r u - d||^2 + lambda^2 ||H u - q||^2; with
 * u0 = H^{-1} q it is u = u0 + lambda^-2 H^{-1} H^{-H} P_r^T z, where z solves
 * the receiver-space system (I + lambda^-2 P_r H^{-1} H^{-H} P_r^T) z = d - P_r u0
 * by conjugate gradients (Hermitian positive definite; two solves per
 * iteration, to a relative residual cg_tol or cg_maxit iterations).  Then
 *   f = sum 1/2 ||P_r u - d||^2 + lambda^2/2 ||H u - q||^2,
 *   g = E^T sum lambda^2 w^2 Re(conj(u) (H u - q))   (variable projection).
 * Arguments as misfit_and_gradient (no mask) plus lambda > 0, cg_tol > 0 and
 * cg_maxit >= 1.  Pairs whose CG misses cg_tol report HELM_E_NOCONV.
 * Workspace: helm_workspace_size with HELM_CALL_WRI. */
int helm_wri_misfit_and_gradient(helm_plan* plan, const double* m_phys, const double* freqs_hz, int nfreq,
                                 const int32_t* src_idx, int n_srcloc, const void* Q, int nsrc,
                                 const void* wavelet, const int32_t* rec_idx, int nrec, const void* d_obs,
                                 double lambda, double cg_tol, int cg_maxit, double* f_out, double* g_out,
                                 void* workspace, size_t ws_bytes, helm_rhs_report* reports,
                                 helm_stream_t stream);

/* Misfit alone (Table derivcosts: one PDE per source and frequency):
 *   f = sum_{k,s} 1/2 ||P_r u_{k,s} - d_{k,s}||^2,  u = H(m, w_k)^{-1} q_{k,s},
 * over the (k, s) pairs whose mask byte is non-zero (all when mask is NULL).
 * Optionally keeps what the gradient needs later (the forward-field store
 * policy of a differentiable objective):
 *   R_out  complex128 [nfreq][nsrc][nrec] or NULL: data residuals P_r u - d
 *          (rows of masked-out pairs are set to zero)
 *   U_out  [nfreq][nsrc][n_comp] or NULL: forward fields (masked-out pairs
 *          are not written), complex128 when u_type is HELM_FIELD_C128 or
 *          complex64 when it is HELM_FIELD_C64 (each part of the FP64 field
 *          rounded to nearest: half the memory, a relative perturbation of
 *          at most 2^-24 per part, which the gradient inherits)
 * The misfit itself always uses the FP64 field.  Other arguments as
 * misfit_and_gradient.  f_out float64 [1]. */
int helm_misfit(helm_plan* plan, const double* m_phys, const double* freqs_hz, int nfreq,
                const int32_t* src_idx, int n_srcloc, const void* Q, int nsrc, const void* wavelet,
                const int32_t* rec_idx, int nrec, const void* d_obs, const uint8_t* mask, double* f_out,
                void* R_out, void* U_out, int u_type, void* workspace, size_t ws_bytes,
                helm_rhs_report* reports, helm_stream_t stream);

/* Adjoint-state gradient from stored forward fields (Appendix A; Table
 * derivstuff, grad f = T* V): for every unmasked (k, s),
 *   v = -H(m, w_k)^{-H} P_r^T R_{k,s},   g = E^T sum w_k^2 Re(conj(U_{k,s}) v),
 * with U and R as written by helm_misfit (U [nfreq][nsrc][n_comp] of type
 * u_type, R complex128 [nfreq][nsrc][nrec]).  g_out float64 [n_phys]
 * (overwritten).  helm_misfit followed by helm_gradient with complex128
 * fields equals misfit_and_gradient. */
int helm_gradient(helm_plan* plan, const double* m_phys, const double* freqs_hz, int nfreq,
                  const int32_t* rec_idx, int nrec, const void* R_in, int nsrc, const void* U_in,
                  int u_type, const uint8_t* mask, double* g_out, void* workspace, size_t ws_bytes,
                  helm_rhs_report* reports, helm_stream_t stream);

/* One model's misfit_and_gradient request for helm_misfit_and_gradient_batch
 * (the paper's distribution over models, sources and frequencies, Sec. 3).
 * Fields mean what the arguments of misfit_and_gradient mean; `status` is
 * written with that call's return value. */
typedef struct {
  helm_plan* plan;
  const double* m_phys;
  const double* freqs_hz;   /* HOST */
  int nfreq;
  const int32_t* src_idx;
  int n_srcloc;
  const void* Q;
  int nsrc;
  const void* wavelet;
  const int32_t* rec_idx;
  int nrec;
  const void* d_obs;
  const uint8_t* mask;
  double* f_out;
  double* g_out;
  void* workspace;
  size_t ws_bytes;
  helm_rhs_report* reports; /* HOST or NULL */
  helm_stream_t stream;     /* each item on its own stream */
  int status;               /* out */
} helm_batch_item;

/* Evaluate every item (models of any size; each with its own plan, data and
 * workspace).  A work queue hands items to `nworkers` host threads; each
 * runs misfit_and_gradient on its item's stream, so the kernels of several
 * models are in flight on the GPU together.  Blocks until all items are done
 * and returns the worst status (HELM_E_INVAL if items is NULL or nworkers < 1).
 * Items whose streams or workspaces alias must not be in the same batch. */
int helm_misfit_and_gradient_batch(helm_batch_item* items, int nitems, int nworkers);

/* helm_apply without a workspace argument (the paper has no counterpart: this
 * is an interface convenience).  For callers that cannot allocate device
 * memory where they apply the operator: hosts whose framework owns every
 * device allocation through its own pool and forbids raw cudaMalloc, and
 * serving loops that must not allocate per request.  The scratch helm_apply
 * takes from its workspace (extended model, damping tables, slot lists)
 * lives instead in one static device array of HELM_NOALLOC_SCRATCH_BYTES
 * inside the library, present on every GPU that loads the library until the
 * process exits.  Enough for fields of up to about 1.3 million computational
 * nodes; larger problems return HELM_E_NOMEM (use helm_apply with a
 * workspace).  The first call on a device looks up the array's device address
 * with that device current.  Like helm_apply, the call copies small host
 * arrays to the device and synchronises `stream` before it returns, so it
 * cannot be recorded into a CUDA graph by stream capture.  All calls share
 * the array and it keeps the last call's contents: calls whose GPU work
 * overlaps (other streams or host threads) race and must be serialised.  The
 * call allocates nothing.  Arguments and results are those of helm_apply. */
#define HELM_NOALLOC_SCRATCH_BYTES (16u << 20)
int helm_apply_noalloc(helm_plan* plan, const double* m_phys, double freq_hz, int adjoint,
                       int precision, const void* x, void* y, int nrhs, helm_stream_t stream);

/* Tile shapes of the operator apply (no counterpart in the paper: the
 * paper's stencil is a CPU loop).  The complex64 apply has
 * helm_stencil_variant_count() shapes -- columns per block, z-planes per tile
 * and the blocks per SM its register budget is sized for, as
 * helm_stencil_variant_info() reports.  Every shape computes every node with
 * the same arithmetic, so results do not depend on the shape.  By default
 * the first apply on a grid of at least 200000 nodes times each shape three
 * times on that call's own fields (synchronising the stream once) and keeps
 * the fastest for the grid; the complex128 apply and smaller grids use shape
 * 0.  helm_stencil_select(v) forces shape v for every later apply (-1 goes
 * back to tuning); HELM_E_INVAL for a shape out of range.
 * helm_stencil_tuned() reports the shape tuned for a plan's grid level
 * (plain apply when residual is 0, residual form b - H x otherwise) and the
 * fastest launch time in microseconds, or HELM_E_INVAL when that grid has not
 * been tuned.  The settings are process-wide. */
int helm_stencil_variant_count(void);
int helm_stencil_variant_info(int variant, int* threads, int* zplanes, int* min_blocks);
int helm_stencil_select(int variant);
int helm_stencil_tuned(const helm_plan* plan, int level, int residual, int* variant, double* us);

/* Diagnostic (no counterpart in the paper): checks, on the device of the
 * current context, how the library reports a bounded device wait that runs
 * out.  One thread waits -- with the same bounded wait the streamed kernels
 * use on their bulk copies -- on an mbarrier phase that nothing completes;
 * after about half a second (2^30 SM cycles) it gives up and the call returns
 * HELM_E_TIMEOUT, with the CUDA context still usable.  HELM_OK would mean
 * the wait completed (never expected); HELM_E_CUDA a launch or copy error.
 * Blocks the host for the duration of the wait. */
int helm_check_bounded_wait(helm_stream_t stream);

/* Debug build (libhelm_debug.so, compiled with HELM_DEBUG; no counterpart in
 * the paper).  That build leaves a 256-byte guard band filled with 0xA5 after
 * every array it lays out in a workspace, checks on the host that every slot
 * index it hands to the kernels is in range, and ends every entry point by
 * checking the bands: HELM_E_BOUNDS reports a write past the end of an array
 * (workspace sizes grow by the bands).  helm_debug_guard_selftest arms the
 * bands of an operator-apply workspace (sized by helm_workspace_size with
 * HELM_CALL_APPLY, nfreq = nsrc = 1), checks them (HELM_OK expected), then
 * changes one byte of the first band from the host and checks again:
 * HELM_E_BOUNDS is the expected result.  Not exported by the release build. */
#ifdef HELM_DEBUG
int helm_debug_guard_selftest(helm_plan* plan, void* workspace, size_t ws_bytes, helm_stream_t stream);
#endif

/* Static description of a status code. */
const char* helm_status_string(int status);

/* Number of kernels this library launched since the process started (a
 * monotonically increasing host counter). */
uint64_t helm_kernel_launch_count(void);

/* Instrumentation (no counterpart in the paper): per-kernel-class timing.
 * While enabled, every launch of a class is bracketed by CUDA events on its
 * own stream and the algorithmic bytes it moves (inputs read once, outputs
 * written once) are summed.  helm_profile_enable(on) clears the counters and
 * switches recording on or off; helm_profile_read() waits for the recorded
 * events and returns launches, summed device milliseconds and bytes. */
typedef enum {
  HELM_PROF_STENCIL_C64 = 0,  /* stencil / residual, complex64 */
  HELM_PROF_STENCIL_C128 = 1, /* stencil / residual, complex128 */
  HELM_PROF_KRYLOV_C64 = 2,   /* fused Gram-Schmidt / norm / update passes, complex64 */
  HELM_PROF_KRYLOV_C128 = 3,  /* the same in complex128 */
  HELM_PROF_SMALL = 4,        /* unused (reductions are folded into the producing kernels); kept for stable numbering */
  HELM_PROF_TRANSFER = 5,     /* restriction / prolongation */
  HELM_PROF_FWI = 6,          /* sources, receivers, misfit, gradient, extension */
  HELM_PROF_MISC = 7,         /* conversions, zero fills, Jacobi */
  HELM_PROF_STENCIL_C64_COARSE = 8, /* complex64 stencil launches on grids below 200000 nodes */
  HELM_PROF_KRYLOV_C64_COARSE = 9,  /* complex64 vector passes on grids below 200000 nodes */
  HELM_PROF_GRAM_C64 = 10,    /* s-step Gram passes, complex64, fine grids */
  HELM_PROF_UPDATE_C64 = 11,  /* solution updates (and recursive residuals), complex64, fine grids */
  HELM_PROF_NCLASS = 12
} helm_prof_class;
int helm_profile_enable(int on);
int helm_profile_read(int cls, uint64_t* launches, double* ms, double* bytes);

#ifdef __cplusplus
}
#endif
#endif /* HELM_H */
