/*
 * ibdl.h — C ABI of the GB300 (sm_103a) implementation of the Immersed Boundary Double Layer
 * (IBDL) operator and its GMRES solve (Leathers 2022, arXiv 2210.07403).
 *
 * The problem (Sec. 5.1, Sec. 6.1): find the boundary density Q of the second-kind system
 *
 *     L u + S̃ Q = 0 in the periodic box C,      S* u + ½ Q = U_b on Γ,
 *
 * with L = Δ − λ (screened Poisson, λ ≥ 0, Sec. 5.1.1) or the Stokes system
 * μΔu − ∇p + μ∇·(S A) = 0, ∇·u + S(Q·n) = 0 (Sec. 6.1.1, interior domain, η = 0). Eliminating
 * u gives the Schur operator applied at every GMRES iteration (Sec. 5.3.2, Eq. "ibdl schur
 * again"; Sec. 6.3.3):
 *
 *     A Q = −S* L⁻¹ S̃ Q + ½ Q.
 *
 * Data layout (all entry points):
 *   - boundary arrays are structure-of-arrays, FP64: X and normals are [dim][n_points]
 *     (x coordinates first), weights [n_points]; densities and data are [c][n_points] with
 *     c = 1 (scalar) or c = dim (Stokes: Q_x[M] then Q_y[M]).
 *   - grid fields are row-major with x fastest: u[z][y][x].
 *   - the grid is cubic: n nodes per axis on [origin, origin + box)^dim, h = box / n,
 *     node i at origin + i·h (Sec. 2.2.1).
 *
 * Ownership: the caller owns every pointer it passes. ibdl_create_geometry copies X, normals
 * and weights and owns all workspace (grid spectra, sorted point tables, twiddles, Krylov
 * basis); nothing the caller passes is retained after a call returns.
 *
 * Streams: every call enqueues its work on the CUDA stream given (a cudaStream_t passed as
 * void*; NULL = the legacy default stream). ibdl_apply, ibdl_adjoint and ibdl_evaluate_field
 * are asynchronous. ibdl_solve synchronises the stream before returning its status.
 *
 * Errors: every call returns an ibdl_status and never aborts the process. On failure,
 * ibdl_last_error() returns a message describing the last error on the calling thread.
 *
 * Threads: a geometry may be used by one thread at a time; distinct geometries are independent.
 *
 * Environment (read once per process; for experiments, none is needed for correct results):
 *   IBDL_NO_PDL=1            launch kernels without programmatic dependent launch;
 *   IBDL_UNROLL=u (1..16)    GMRES iterations per body of a cycle's captured while loop (8);
 *   IBDL_ARNOLDI_CLUSTER=8   run the Arnoldi step on 8-CTA clusters even where 16 fit;
 *   IBDL_PLAN_R, IBDL_PLAN_C, IBDL_THREADS   2-D launch shape before autotuning (rows per CTA of
 *                            the row kernels, columns per CTA of the column pass, least threads
 *                            per CTA of the row kernels);
 *   IBDL_PLAN3_R, IBDL_PLAN3_C, IBDL_PLAN3_CZ   the same for the 3-D kernels;
 *   IBDL_BATCH_PERSISTENT=1  batched column passes of the scalar operator on persistent CTAs
 *                            that load the next unit before transforming the current one,
 *                            instead of one CTA per unit (read when a batch is created);
 *   IBDL_COL_STAGED=0|1      FP32 column pass with direct loads (0) or staged in shared memory by
 *                            tensor-memory-accelerator copies (1), read when a geometry or batch
 *                            is created; unset, the direct pass runs until ibdl_autotune /
 *                            ibdl_batch_autotune choose the faster one;
 *   IBDL_COL_STAGES=2..4     stages (units copied ahead) of the staged column pass (3).
 *
 * IBDL_ERR_TIMEOUT: the staged column pass bounds each wait for its copies (1 s); a wait that
 * runs out stops that CTA and sets a flag, reported by the next solve or application on the
 * geometry (a batch: by its next solve).
 */
#ifndef IBDL_H
#define IBDL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IBDL_OK = 0,
  IBDL_ERR_INVALID_ARG = 1,   /* a null pointer, an out-of-range size or option          */
  IBDL_ERR_CUDA = 2,          /* a CUDA runtime call failed (message has the CUDA error) */
  IBDL_ERR_NO_MEMORY = 3,     /* device or pinned host allocation failed                 */
  IBDL_ERR_NOT_CONVERGED = 4, /* GMRES hit maxit; Q holds the best iterate               */
  IBDL_ERR_NONFINITE = 5,     /* NaN/Inf in the inputs or in a residual                  */
  IBDL_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up                      */
  IBDL_ERR_UNSUPPORTED = 7    /* a valid combination this build does not implement       */
} ibdl_status;

/* PDE on the periodic box */
enum { IBDL_PDE_SCALAR = 0, /* L = Δ − λ (Sec. 5.1.1); λ = 0 uses the mean-zero Δ₀⁻¹ (Sec. 2.2.4) */
       IBDL_PDE_STOKES = 1  /* μΔu − λu − ∇p, interior, η = 0: Stokes for λ = 0 (Sec. 6.3.3),
                               Brinkman for λ = k² > 0 (Sec. 6.3.2); dim = 2 only             */ };

/* boundary condition of the scalar problem */
enum { IBDL_BC_DIRICHLET = 0, /* S*u + ½Q = U_b (Sec. 5.1.1)                                       */
       IBDL_BC_NEUMANN = 1    /* S*u = ½U_b with U_b the unknown, ∂u/∂n = V_b (Sec. 5.2): the
                                 operator is (−S*L⁻¹S̃ − ½) and the right-hand side S*L⁻¹S V_b
                                 is −ibdl_single_layer(V_b) (scalar PDE only)                    */ };

/* one-dimensional 4-point kernel φ of δ_h = h^-d Π φ(x_j/h) (Sec. 2.2.2) */
enum { IBDL_DELTA_COS = 0,  /* φ(r) = (1 + cos(πr/2))/4, |r| < 2                            */
       IBDL_DELTA_SQRT = 1  /* Peskin's 4-point kernel with square roots (Sec. 2.2.2)         */ };

/* discretisation of the dipole spread S̃Q = ∇·(S(Q n)) (Sec. 5.1.1, Sec. 5.3.1) */
enum { IBDL_DIPOLE_ANALYTIC = 0,     /* exact gradient of δ_h: one scalar field (Stokes: 3)   */
       IBDL_DIPOLE_SPECTRAL_DIV = 1  /* spread Q n, divergence by the derivative symbol       */ };

/* Fourier symbols of the differential operators (Sec. 2.2.1, Sec. 2.3.1, Sec. 5.3.1) */
enum { IBDL_SYMBOL_SPECTRAL = 0, /* −Δ ↦ |k|², ∂ ↦ ik (0 at the Nyquist index)             */
       IBDL_SYMBOL_FD2 = 1       /* 5-point Laplacian and centred first differences         */ };

/* arithmetic of the grid work inside one operator application */
enum { IBDL_FP64 = 0, IBDL_FP32 = 1,
       IBDL_MIXED = 2,  /* solve only: FP32 applies, FP64 Arnoldi, refinement residual as chosen by
                           ibdl_solve_opts.residual                                           */
       IBDL_FP32X2 = 3  /* float-float: every value of the FFT and Fourier stage an unevaluated
                           sum of two FP32 numbers (about 48 significand bits, an application
                           within about 1e-13 of FP64), the point work in FP64; operator
                           applications (A and Aᵀ; 2-D grids to 4096², every 3-D grid) and the
                           refinement residual                                                */ };

typedef struct ibdl_geometry ibdl_geometry; /* opaque, library-owned */

typedef struct {
  int dim;              /* 2 or 3                                                          */
  int n;                /* grid nodes per axis: a power of two, 16..8192 (2-D), 16..256 (3-D);
                           every 2-D operator runs to 8192 in FP64 and FP32 (one field per
                           launch where a band's or column's fields do not fit shared memory
                           together) and to 4096 in float-float; a float-float call at 8192
                           returns IBDL_ERR_UNSUPPORTED                                       */
  double box;           /* side length of the periodic box, > 0                             */
  double origin[3];     /* lower corner of the box (unused entries ignored)                 */
  int64_t n_points;     /* M ≥ 1                                                           */
  const double* X;      /* [dim][M] boundary points                                         */
  const double* normals;/* [dim][M] unit normals pointing out of Ω; NULL (2-D): estimated      */
  const double* weights;/* [M] quadrature weights Δs_i (arclength, Sec. 2.2.2); NULL (2-D):  */
                        /* estimated. Estimates (Sec. 5.3.1) treat the points as one closed
                           curve in order: n_i ∝ (Y_{i+1} − Y_{i−1}, −(X_{i+1} − X_{i−1})), to the
                           right of the direction of travel (order an interior boundary
                           counter-clockwise, an exterior one clockwise), Δs_i = ‖X_{i+1} − X_i‖,
                           differences by minimum image                                      */
  int pde;              /* IBDL_PDE_*                                                       */
  double lambda;        /* λ ≥ 0: L = Δ − λ (scalar); L = μΔ − λ (Stokes λ = 0, Brinkman λ > 0) */
  double mu;            /* viscosity μ > 0 for IBDL_PDE_STOKES (cancels from A when λ = 0)   */
  int delta;            /* IBDL_DELTA_*                                                     */
  int dipole;           /* IBDL_DIPOLE_*                                                    */
  int symbol;           /* IBDL_SYMBOL_*                                                    */
  int inputs_on_device; /* nonzero: X, normals, weights are device pointers                 */
  int bc;               /* IBDL_BC_* (0, Dirichlet, for a zero-initialised descriptor)      */
  double eta;           /* completed method, η > 0 (0: not completed); see below          */
} ibdl_geometry_desc;

/* Completed method (Sec. 5.3.3 Poisson, Sec. 6.1.3 and Sec. 6.3.3 Stokes): for exterior domains
 * (and wherever the double layer alone cannot represent the flow) the sources gain the
 * single layer ηSQ and, because λ = 0 leaves the mean of u free, the unknowns gain ū, one mean
 * per component: the system is
 *     S*u₀ + ū·1 + ½Q = U_b − (forcing term),    η Σ_i Δs_i Q_i = h^d Σ_g g̃,
 * u₀ the mean-zero grid field of (S̃ + ηS)Q (Stokes: the projected source is (η/μ)SQ + ∇·(SA)).
 * With η > 0 (2-D, λ = 0, analytic dipole, Dirichlet data; IBDL_ERR_UNSUPPORTED otherwise)
 * every boundary vector of ibdl_apply, ibdl_solve and ibdl_evaluate_field has c·M + c entries:
 * the density [c][M], then ū[c]; the last c entries of a right-hand side are h^d Σ g̃ per
 * component, and the grid field written by ibdl_evaluate_field is u₀ + ū. The net force on the
 * boundary is −η Σ_i Δs_i Q_i (Sec. 6.1.3). Transposes, derivatives, probes, the single layer,
 * batches and ibdl_apply_noalloc do not take completed geometries. */

typedef struct {
  double rtol;          /* stop when ‖U_b − A Q‖₂ ≤ rtol·‖U_b‖₂ (relative Euclidean residual)  */
  int restart;          /* Krylov subspace size m before a restart, 1..64                    */
  int maxit;            /* maximum total Krylov iterations (all restarts and sweeps)         */
  int precision;        /* IBDL_FP64 (plain), IBDL_FP32 or IBDL_MIXED (FP32 inner, FP64 outer) */
  double inner_rtol;    /* IBDL_MIXED: relative tolerance of each inner FP32-apply GMRES      */
  int max_refine;       /* IBDL_MIXED: maximum refinement sweeps whose inner cycle converged
                           (a sweep whose inner cycle stops at the restart length is followed
                           by an FP64 residual restart and does not count)                    */
  int io_on_host;       /* nonzero: U_b and Q are host pointers (copied inside the call)     */
  int residual;         /* IBDL_MIXED: arithmetic of the refinement residual's application,
                           IBDL_FP64 (0) or IBDL_FP32X2 (float-float, for 2-D grids to 4096²
                           and every 3-D grid; 8192² grids use FP64); the residual's
                           subtraction and norm are FP64 either way                           */
} ibdl_solve_opts;

typedef struct {
  int iterations;       /* Krylov iterations, all cycles and sweeps                          */
  int fp64_applies;     /* operator applications with FP64 grid arithmetic                   */
  int fp32_applies;     /* operator applications with FP32 grid arithmetic                   */
  int sweeps;           /* refinement sweeps (IBDL_MIXED), restart cycles otherwise          */
  double rel_residual;  /* final ‖U_b − AQ‖₂/‖U_b‖₂ with an FP64 (or, IBDL_MIXED with residual */
                        /* IBDL_FP32X2, float-float) application (plain: the GMRES estimate  */
                        /* of the last cycle)                                                */
  double seconds;       /* wall time of the call                                             */
  int64_t kernel_launches; /* CUDA kernels this call launched (including ones that found the  */
                        /* solve already converged and returned at once)                     */
  int fp32x2_applies;   /* operator applications with float-float grid arithmetic            */
} ibdl_solve_info;

/* Stage timing (off by default). When enabled, every operator application records CUDA events
 * on the caller's stream around each of its kernels, and every Arnoldi step around its kernel.
 * ibdl_get_stage_times synchronises the device, adds up the device milliseconds and the
 * launches of every stage recorded since the previous call, writes them to ms[] and launches[]
 * (IBDL_STAGE_COUNT entries each), and resets the record. At most 16384 events are kept; later
 * launches are not timed. */
enum { IBDL_STAGE_SPREAD_ROWFFT_FP64 = 0, IBDL_STAGE_COLUMN_FP64 = 1, IBDL_STAGE_ROWIFFT_GATHER_FP64 = 2,
       IBDL_STAGE_SPREAD_ROWFFT_FP32 = 3, IBDL_STAGE_COLUMN_FP32 = 4, IBDL_STAGE_ROWIFFT_GATHER_FP32 = 5,
       IBDL_STAGE_ARNOLDI = 6, IBDL_STAGE_OTHER = 7, IBDL_STAGE_COUNT = 8 };
ibdl_status ibdl_set_stage_timing(ibdl_geometry* geom, int enable);
ibdl_status ibdl_get_stage_times(ibdl_geometry* geom, double* ms, int64_t* launches);

/* Build the geometry: copy the boundary, bucket points by stencil cell, precompute the kernel
 * weights (FP64 and FP32) and FFT twiddles, allocate all workspace. Points may lie outside
 * the box; they wrap periodically. Errors: IBDL_ERR_INVALID_ARG (sizes, non-unit normals,
 * non-positive weights, non-finite coordinates), IBDL_ERR_UNSUPPORTED (Stokes in 3-D),
 * IBDL_ERR_NO_MEMORY, IBDL_ERR_CUDA. Synchronises `stream`. */
ibdl_status ibdl_create_geometry(const ibdl_geometry_desc* desc, void* stream, ibdl_geometry** out);

/* Release all device and host memory of the geometry. Safe on NULL. Synchronises the device. */
ibdl_status ibdl_destroy_geometry(ibdl_geometry* geom);

/* Y = A Q = S*u + ½Q with u = −L⁻¹S̃Q (scalar, Sec. 5.3.2 Eq. "ibdl schur again") or the
 * Stokes velocity of Sec. 6.3.3. Q and Y are device FP64 arrays [c][M] (they may not alias);
 * `precision` (IBDL_FP64, IBDL_FP32 or IBDL_FP32X2) selects the grid
 * arithmetic. Asynchronous on `stream`. */
ibdl_status ibdl_apply(ibdl_geometry* geom, int precision, const double* Q, double* Y, void* stream);

/* Z = A* W, the adjoint of A with respect to the Δs-weighted boundary inner product
 * Σ_i Δs_i a_i b_i: A* W = ½W + (S̃)* (−L⁻¹) S W, where S* is the adjoint of S under the weighted
 * products (Sec. 2.1, Sec. 2.2.4). Scalar PDE only (IBDL_ERR_UNSUPPORTED for Stokes). Device
 * FP64 arrays [M]; asynchronous. */
ibdl_status ibdl_adjoint(ibdl_geometry* geom, int precision, const double* W, double* Z, void* stream);

/* Solve A Q = U_b by GMRES from a zero initial guess (Sec. 5.1.2 step 1 and Sec. 5.3.2 with
 * g̃ = 0). IBDL_FP64: restarted GMRES(m), FP64 everything. IBDL_MIXED: iterative refinement,
 * each sweep one inner GMRES cycle with FP32 applications and FP64 Arnoldi/Hessenberg to
 * max(inner_rtol·‖r‖, ½·rtol·‖U_b‖), then Q += correction and the FP64 residual U_b − A₆₄Q; the
 * host reads the status once per sweep (once per cycle in FP64). U_b and Q are [c][M] FP64,
 * device pointers unless opts->io_on_host.
 * Returns IBDL_ERR_NOT_CONVERGED (Q = best iterate) when maxit is reached. `info` may be NULL. */
ibdl_status ibdl_solve(ibdl_geometry* geom, const double* Ub, double* Q, const ibdl_solve_opts* opts,
                       ibdl_solve_info* info, void* stream);

/* A source term g̃ on the box (Sec. 5.1.2, Eq. "ibdl schur again"; Sec. 6.1.1, Eq. "ibdl stokes"):
 * L u + S̃Q = g̃ (scalar) or L u − ∇p + μ∇·(SA) = g̃ with ∇·u + S(Q·n) = 0 (Stokes, Brinkman). Its
 * response alone is u_g = L⁻¹g̃ (scalar) or û_g = −P̂ĝ/(μ|k|² + λ) (Stokes: the operator's own
 * projection and symbols); for λ = 0 the mean of g̃ does not enter u_g. Then
 *   ibdl_solve_forced:          A Q = U_b − S*u_g (U_b the Dirichlet data; for the Neumann problem
 *                               −ibdl_single_layer(V_b)), solved as ibdl_solve does; for the
 *                               completed method the c constraint rows become h^d Σ_g g̃_l (the
 *                               last c entries of U_b are ignored);
 *   ibdl_evaluate_field_forced: u_grid = the field of Q (ibdl_evaluate_field) + u_g.
 * g_grid: device FP64 [c][n^dim] (c = 1 scalar, 2 Stokes; 2-D and 3-D); NULL makes both calls
 * their unforced counterparts. u_grid may not overlap g_grid. The geometry allocates its
 * source-term workspace (about (c + 3)·n^dim + c·M doubles) on the first forced call. */
ibdl_status ibdl_solve_forced(ibdl_geometry* geom, const double* Ub, const double* g_grid, double* Q,
                              const ibdl_solve_opts* opts, ibdl_solve_info* info, void* stream);
ibdl_status ibdl_evaluate_field_forced(ibdl_geometry* geom, const double* Q, const double* g_grid, double* u_grid,
                                       void* stream);

/* Z = S*(−L⁻¹)(S V): the single-layer operator of the scalar method (the constraint method's
 * Schur complement up to sign, Sec. 2.2.3), with S the Δs-weighted spread and S* the
 * interpolation. It carries Neumann data into the right-hand side of the Neumann equation
 * (Sec. 5.2, Eq. "Neumann saddle point", g̃ = 0): rhs = −Z(V_b). Scalar PDE, 2-D; V and Z are
 * device FP64 [M] that may not alias; `precision` IBDL_FP64 or IBDL_FP32; asynchronous. */
ibdl_status ibdl_single_layer(ibdl_geometry* geom, int precision, const double* V, double* Z, void* stream);

/* Differentiation. The paper states no derivative; these follow from the operators of
 * Sec. 5.3.2 and Sec. 6.3.3 by the adjoint method. Both operators are
 * A Q = S*(K[sources(Q)]) + ½Q with K a Fourier multiplier (−L⁻¹, or the Stokes multiplier
 * û = (i k̃ ŝ + P̂ ĝ)/|k|²). For Q = A⁻¹U_b and an objective J(Q) with G = ∂J/∂Q:
 *   λ = A⁻ᵀ G,   ∂J/∂U_b = λ,   ∂J/∂p = −∂(λᵀ A(X, n, Δs) Q)/∂p  for p = X, n, Δs.
 * The normals and weights are independent inputs; a caller whose n and Δs depend on X adds
 * their chain rule. Derivatives in X use φ'' of the delta kernel, which jumps where a point
 * sits at a whole-number offset from a node (√-Peskin |r| = 1, 2; cosine |r| = 2): A is not
 * differentiable in X there and the value returned is that of the piece containing the offset.
 * Stokes derivatives and transposes need the analytic dipole (IBDL_ERR_UNSUPPORTED otherwise).
 *
 * ibdl_apply_transpose: Z = Aᵀ G (Euclidean transpose; [c][M] FP64 device arrays that may not
 * alias). Scalar: Aᵀ = W A* W⁻¹ (W = diag Δs, A* as in ibdl_adjoint) = ½G + (Δs/h^d)(S̃)*(−L⁻¹)ψ,
 * ψ = Σ_j G_j Φ(x − X_j). Stokes: ½G + the spread transpose of Kᵀψ, ψ_l = Σ_j G_{l,j} Φ(x − X_j),
 * K̂ᵀ the conjugate symbol. `precision` as ibdl_apply. Asynchronous.
 *
 * ibdl_solve_transpose: solve Aᵀ λ = G with the GMRES of ibdl_solve (same options, precision
 * modes, graphs and convergence rule, on ‖G − Aᵀλ‖ ≤ rtol‖G‖). G and lambda are [c][M] FP64,
 * device pointers unless opts->io_on_host. Synchronises `stream`.
 *
 * ibdl_solve_vjp: given Q (the solution of A Q = U_b) and λ (of Aᵀλ = G), writes
 *   dX[dim][M] = ∂J/∂X,  dn[dim][M] = ∂J/∂n,  dw[M] = ∂J/∂Δs
 * (any may be NULL: not computed), in the boundary layout of ibdl_create_geometry. FP64: the
 * grid fields u = K[sources(Q)] and v = Kᵀψ (ψ = Σ_j λ_j Φ(x − X_j)), then per point the value,
 * gradient and Hessian gathers of δ_h against them. Outputs may not overlap each other or the
 * inputs. Asynchronous; the first derivative call allocates grid fields held by the geometry.
 *
 * Probes (2-D): values of the grid solution at n_probes points P[2][n_probes] (device FP64,
 * wrapped periodically), u(p) = Σ_g u_g δ_h(x_g − p) h^d, with the geometry's delta kernel.
 * ibdl_probe_evaluate: U[c][n_probes] = E Q, u the grid field of Q (scalar u or the Stokes
 * velocity). ibdl_probe_vjp: for ν[c][n_probes] = ∂J/∂U, writes dQ[c][M] = Eᵀν and
 * dX, dn, dw = ∂(νᵀ E(X, n, Δs) Q)/∂(X, n, Δs) with P fixed (each may be NULL). A full gradient
 * of J(U) with U = E Q(U_b) adds these to the solve's: pass G = dQ to ibdl_solve_transpose, then
 * ibdl_solve_vjp. Outputs may not overlap each other or the inputs. Asynchronous. */
ibdl_status ibdl_apply_transpose(ibdl_geometry* geom, int precision, const double* G, double* Z, void* stream);
ibdl_status ibdl_solve_transpose(ibdl_geometry* geom, const double* G, double* lambda, const ibdl_solve_opts* opts,
                                 ibdl_solve_info* info, void* stream);
ibdl_status ibdl_solve_vjp(ibdl_geometry* geom, const double* Q, const double* lambda, double* dX, double* dn,
                           double* dw, void* stream);
ibdl_status ibdl_probe_evaluate(ibdl_geometry* geom, const double* P, int n_probes, const double* Q, double* U,
                                void* stream);
ibdl_status ibdl_probe_vjp(ibdl_geometry* geom, const double* P, int n_probes, const double* Q, const double* nu,
                           double* dQ, double* dX, double* dn, double* dw, void* stream);

/* Post-processing of a grid solution.
 *
 * ibdl_indicator (Sec. 5.3.5): flags the grid nodes enclosed by the discrete boundary. χ solves
 * Δχ = −S̃1, the IBDL grid field of the unit density for the Laplace problem (mean-zero inverse),
 * with the geometry's delta kernel, dipole spread and symbol whatever its PDE, λ or η; in the
 * continuum χ is the indicator of the enclosed region minus its area fraction. The call writes
 * chi = χ − χ(box corner, node 0) (≈ 1 enclosed, ≈ 0 outside; ≈ −1 enclosed when the normals
 * point into the enclosed region) and flags = 1 where |chi| > ½, else 0. Several disjoint curves
 * are flagged at once. chi: device FP64 [n^dim]; flags: device uint8 [n^dim]; they may not
 * overlap. 2-D and 3-D. Asynchronous. The geometry keeps a post-processing workspace (one FP64
 * grid field plus, in 2-D, 5 bytes per node), allocated by the first post-processing call.
 *
 * ibdl_near_boundary (Sec. 5.3.4, 2-D): replaces the grid values near Γ by linear interpolation.
 * Every node x_p with omega[x_p] ≠ 0 whose nearest boundary point lies closer than m1·h gets
 *     u(x_p) = u_A |x_B − x_p|/|x_B − x_A| + u_B |x_A − x_p|/|x_B − x_A|,
 * x_A the point of the chord between its two nearest boundary points x_1, x_2 closest to x_p (if
 * that point falls off the chord: the chord between the two of the three nearest points lying
 * farthest apart, the point clamped to it), u_A = U_b(x_1)|x_A − x_2|/|x_2 − x_1| +
 * U_b(x_2)|x_A − x_1|/|x_2 − x_1|, x_B = x_A + m2·h (x_p − x_A)/|x_p − x_A| and u_B the bilinear
 * interpolation of u at the four nodes around x_B. A node on the chord takes u_A; all other nodes
 * are copied. Distances are minimum-image; nearness and the nearest points are decided on FP64
 * squared distances, equal ones ordered by point index. The paper's settings: m1 = 6, m2 = 8 with
 * IBDL_SYMBOL_FD2; m1 = 2(log₂n − 4), m2 = m1 + 2 with IBDL_SYMBOL_SPECTRAL.
 *   Ub     device FP64 [c][M] boundary values (Dirichlet data; for a Neumann solve, its Q; for a
 *          completed geometry the first c·M entries of the right-hand side)
 *   u      device FP64 [c][n][n] grid solution (ibdl_evaluate_field)
 *   omega  device uint8 [n][n], nonzero on the PDE domain Ω: the flags of ibdl_indicator for an
 *          interior problem, their complement for an exterior one
 *   m1     0 < m1 < n/2; m2 > 0 (meshwidths)
 *   out    device FP64 [c][n][n], may not overlap the inputs
 * Needs M ≥ 3 (IBDL_ERR_INVALID_ARG) and dim = 2 (IBDL_ERR_UNSUPPORTED otherwise). Asynchronous. */
ibdl_status ibdl_indicator(ibdl_geometry* geom, double* chi, uint8_t* flags, void* stream);
ibdl_status ibdl_near_boundary(ibdl_geometry* geom, const double* Ub, const double* u, const uint8_t* omega, double m1,
                               double m2, double* out, void* stream);

/* The grid solution of a density (Sec. 5.1.2 step 2 with g̃ = 0): scalar u = −L⁻¹S̃Q written
 * to u_grid[n^dim]; Stokes velocity written to u_grid[dim][n^dim]. FP64 device arrays;
 * asynchronous. */
ibdl_status ibdl_evaluate_field(ibdl_geometry* geom, const double* Q, double* u_grid, void* stream);

/* Default solve options: rtol 1e-8, restart 50, maxit 200, IBDL_FP64, inner_rtol 1e-4,
 * max_refine 6, device I/O, float-float refinement residual. */
void ibdl_default_solve_opts(ibdl_solve_opts* opts);

/* Autotuner (2-D; 3-D shapes follow a fixed volume rule): time candidate launch shapes of the
 * operator application on this geometry (rows per row band 2–64 with a least thread count of the
 * row kernels of 0, 256 or 512, then kx columns per column group 1–32, within 512 threads and the
 * shared memory of a CTA) with CUDA events and keep the fastest, for FP64 (precision_mask bit
 * 0), FP32 (bit 1) and/or float-float (bit 2). The choice is cached in the process per grid size,
 * field counts, PDE, dipole form and precision; geometries created later with the same key start
 * from it. Allocates and frees a small scratch vector. Synchronises `stream`. */
ibdl_status ibdl_autotune(ibdl_geometry* geom, int precision_mask, void* stream);

/* Geometry facts: number of density components c and points M. */
ibdl_status ibdl_geometry_sizes(const ibdl_geometry* geom, int* ncomp, int64_t* n_points);

/* The 2-D launch plan of one grid arithmetic (IBDL_FP64, IBDL_FP32 or IBDL_FP32X2; the paper has no
 * counterpart: this reports the library's own choices, e.g. after ibdl_autotune): rows per row
 * band, kx columns per column group, least threads per CTA of the row kernels, whether FP32
 * column passes are staged by tensor-memory-accelerator copies (0/1) and whether applications
 * run one field per launch (0/1). Any output pointer may be NULL. IBDL_ERR_UNSUPPORTED for 3-D
 * geometries. No device work. */
ibdl_status ibdl_launch_plan(const ibdl_geometry* geom, int precision, int* rows, int* cols, int* threads,
                             int* staged, int* split);

/* ---- batches of independent 2-D problems -------------------------------------------------
 * A batch holds `count` problems with the same pde and dipole form and any grid size, point
 * count, λ, delta and symbol. Boundary vectors of all problems are concatenated in problem order
 * (problem b occupies [offsets[b], offsets[b+1]) of every Q, Y, U_b array; see ibdl_batch_sizes).
 * Every stage of an application is one launch for the whole batch; a batched solve runs one
 * GMRES per problem, all advancing together in one captured graph per restart cycle. There is
 * no counterpart in the paper beyond solving each problem as in Sec. 5.3.2. */
typedef struct ibdl_batch ibdl_batch; /* opaque, library-owned */

/* Create the geometries of `count` 2-D problems (each as ibdl_create_geometry) and the batched
 * launch tables. Errors: IBDL_ERR_INVALID_ARG (count outside [1, 65536], mixed pde or dipole
 * forms, any per-problem error, reported with the problem index), IBDL_ERR_UNSUPPORTED (3-D). */
ibdl_status ibdl_create_batch(const ibdl_geometry_desc* descs, int count, void* stream, ibdl_batch** out);
ibdl_status ibdl_destroy_batch(ibdl_batch* batch);

/* Number of problems, the offsets (count + 1 entries, may be NULL) and the total length of the
 * concatenated boundary vectors. */
ibdl_status ibdl_batch_sizes(const ibdl_batch* batch, int* count, int64_t* offsets, int64_t* total);

/* Autotune a batch: time the whole batched application for each pair of candidate FFT volumes
 * per CTA, one for the row kernels and one for the column kernel (512 to 8192 complex elements
 * each; every problem's rows per band and columns per group follow from them) and each least
 * thread count of the row kernels (0 or 256), keep the fastest per precision (precision_mask
 * bits as ibdl_autotune), and rebuild the batched launch tables. Allocates and frees a scratch
 * vector. Synchronises `stream`. */
ibdl_status ibdl_batch_autotune(ibdl_batch* batch, int precision_mask, void* stream);

/* Y = A Q for every problem of the batch (concatenated device FP64 arrays; FP64, FP32 or
 * float-float grid arithmetic). Asynchronous. */
ibdl_status ibdl_batch_apply(ibdl_batch* batch, int precision, const double* Q, double* Y, void* stream);

/* Solve every problem (options as ibdl_solve; maxit bounds the longest problem's iterations).
 * `infos` (count entries, may be NULL) receives per-problem results. Returns
 * IBDL_ERR_NOT_CONVERGED if any problem missed rtol. Synchronises `stream`. */
ibdl_status ibdl_batch_solve(ibdl_batch* batch, const double* Ub, double* Q, const ibdl_solve_opts* opts,
                             ibdl_solve_info* infos, void* stream);

/* Y = A Q for a 2-D problem without allocating any memory (the paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc, e.g. a latency-bound loop that must
 * not take the allocator's locks, or a plug-in whose host application owns all device memory
 * through its own allocator; such callers cannot create an ibdl_geometry, which allocates its
 * tables and work buffers). `desc` describes the geometry as for
 * ibdl_create_geometry, with X, normals and weights in device memory (inputs_on_device = 1); the
 * descriptor's scalars are checked as there, the arrays' values are not (finite coordinates, unit
 * normals and positive weights are the caller's responsibility). Q and Y are device FP64 arrays [c][M]; `precision` is IBDL_FP64 or IBDL_FP32.
 * All work space comes from one fixed 8 MiB array inside the library, per GPU, held from library
 * load to process exit: problems needing more (about nf·n²·8 bytes of spectra with nf = 1 to 4
 * fields, plus about 250 bytes per point) are rejected with IBDL_ERR_INVALID_ARG and a message
 * giving the size. The first call on each GPU looks up that array's device address (a one-time
 * set-up that makes no stream call); make that first call before any stream capture begins. Every
 * call rebuilds the point tables in the shared array, so calls whose GPU work overlaps (other
 * streams or threads) race and give wrong results. Asynchronous on `stream`. */
ibdl_status ibdl_apply_noalloc(const ibdl_geometry_desc* desc, int precision, const double* Q, double* Y,
                               void* stream);

/* Message for the last failed call on this thread ("" if none). Valid until the next call. */
const char* ibdl_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* IBDL_H */
