/*
 * spuma.h -- C ABI of the GB300 LDU pressure-solve library.
 *
 * The library solves A x = b for the pressure equation of a finite-volume
 * mesh stored in OpenFOAM's face-addressed LDU format ("LDUorderedCOO",
 * paper Sec. 2.1): per internal face f an owner lower_addr[f] and a
 * neighbour upper_addr[f] with lower_addr[f] < upper_addr[f], faces sorted by
 * (lower, upper); coefficients diag[n_cells] and upper[n_faces] (the matrix
 * is symmetric, so lower == upper).  Sign convention: A is the NEGATIVE of
 * OpenFOAM's laplacian matrix, so A is symmetric positive definite
 * (diag > 0, upper < 0).
 *
 * Conventions shared by every entry point
 *  - All array arguments are DEVICE pointers (cudaMalloc'ed or torch tensor
 *    storage on the current device), owned by the caller, unless stated
 *    otherwise.  The library never allocates device memory: all scratch and
 *    all derived topology live in the caller's workspace.
 *  - stream is a cudaStream_t (passed as void*); NULL means the legacy
 *    default stream.  Calls are asynchronous with respect to the host except
 *    where stated.
 *  - Arguments are checked on the host before anything is launched; a bad
 *    argument returns an error status and launches nothing.
 *  - Errors found on the device (non-finite input, a non-positive DIC pivot,
 *    a grid-barrier timeout) never trap: they are written to the solver
 *    report (spuma_solver_perf.status) on the device, and
 *    spuma_ldu_device_status() reads them back.
 *  - Non-convergence is not an error (OpenFOAM semantics): status OK with
 *    converged == 0.
 *  - Integers are int32: n_faces < 2^31.
 */
#ifndef SPUMA_H
#define SPUMA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spuma_ldu* spuma_ldu_t;
typedef struct spuma_batch* spuma_batch_t;
typedef void* spuma_stream_t;

typedef enum {
    SPUMA_OK = 0,
    SPUMA_ERR_INVALID_ARG = 1,           /* NULL pointer, negative size, bad enum      */
    SPUMA_ERR_NOT_UPPER_TRIANGULAR = 2,  /* l >= u, index out of range, faces unsorted */
    SPUMA_ERR_CUDA = 3,                  /* a CUDA runtime call failed (see last error) */
    SPUMA_ERR_WORKSPACE_TOO_SMALL = 4,
    SPUMA_ERR_SINGULAR = 5,              /* |p.Ap| / normFactor < 1e-300               */
    SPUMA_ERR_NOT_SPD = 6,               /* a DIC pivot is <= 0                         */
    SPUMA_ERR_NONFINITE = 7,             /* NaN or Inf among the coefficients or b      */
    SPUMA_ERR_DEVICE_TIMEOUT = 8,        /* a grid barrier waited past its time limit   */
    SPUMA_ERR_HOST = 9                   /* a host allocation or thread failed          */
} spuma_status;

typedef enum { SPUMA_F64 = 0, SPUMA_MIXED = 1, SPUMA_F32 = 2, SPUMA_MIXED_RESTART = 3 } spuma_precision;
typedef enum {
    SPUMA_PRECOND_NONE = 0,
    SPUMA_PRECOND_DIAGONAL = 1,
    SPUMA_PRECOND_DIC = 2,
    SPUMA_PRECOND_DILU = 3 /* asymmetric matrices, spuma_pbicg_solve only */
} spuma_precond;

/* spuma_workspace_bytes() flags */
#define SPUMA_WORKSPACE_ASYMMETRIC 1 /* room for spuma_pbicg_solve (asymmetric matrices) */

/* Solver controls, after OpenFOAM's fvSolution entries (paper appendix,
 * fvSolution listing: solver PCG, preconditioner, tolerance, relTol, maxIter,
 * minIter).  Residuals are OpenFOAM's normalised L1 residual
 * sum|b - A x| / normFactor.
 *  precision SPUMA_MIXED: FP32 PCG inside FP64 refinement by reliable
 *    updates: whenever the FP32 residual has dropped by the factor
 *    inner_rel_tol since the last update (or claims convergence, or max_iter
 *    is reached) the FP32 correction is added to the FP64 solution and the
 *    FP64 residual b - A x replaces the FP32 one; the search direction is
 *    kept (no Krylov restart).  max_iter bounds the FP32 iterations.
 *  precision SPUMA_MIXED_RESTART: FP64 iterative refinement around restarted
 *    FP32 inner solves: inner_rel_tol is the inner solve's relative
 *    tolerance, max_outer the maximum number of refinement steps, max_iter
 *    bounds each inner solve.
 *  block_threads: 0 = library default (or the tuned value for batches).   */
typedef struct {
    int32_t precond;        /* spuma_precond                              */
    int32_t precision;      /* spuma_precision (SPUMA_F32 only for Amul)  */
    double tolerance;       /* absolute normalised residual               */
    double rel_tol;         /* relative to the initial residual, 0 = off  */
    double inner_rel_tol;   /* mixed form only                             */
    int32_t max_iter;
    int32_t min_iter;
    int32_t max_outer;      /* mixed form only                             */
    int32_t block_threads;
} spuma_solver_controls;

/* Solver report (OpenFOAM's solverPerformance), written to DEVICE memory by
 * the solve so that solves can be queued and captured without a host sync.
 * true_rel_residual_l2 = ||b - A x||_2 / ||b||_2 (||b - A x||_2 when b = 0) of
 * the returned x, computed on the device at the end of every solve (PCG in
 * every precision, PBiCG, GAMG, batched) in FP64 from the FP64 coefficients:
 * for the mixed forms it is the proof that the FP64 system was solved.
 * Every reduction of the library is deterministic (fixed per-thread,
 * per-block and per-grid order; no atomics in any sum), so equal inputs give
 * bit-identical reports and solutions run to run: there is no separate
 * "deterministic" control. */
typedef struct {
    double initial_residual;
    double final_residual;
    double true_rel_residual_l2;
    int32_t n_iter;         /* PCG iterations (all inner iterations for MIXED) */
    int32_t n_outer;        /* refinement steps (MIXED), else 0               */
    int32_t converged;
    int32_t singular;
    int32_t status;         /* spuma_status of the device side                */
    int32_t n_levels;       /* DIC level count used                           */
} spuma_solver_perf;

/* ------------------------------------------------------------------------
 * Topology.  spuma_workspace_bytes() gives the size of the caller's device
 * workspace for a mesh; spuma_ldu_create() builds, on the device, everything
 * derived from the addressing (face-to-cell gather lists, the DIC level sets,
 * the level-ordered internal layout) into it.  Create is SYNCHRONOUS (it
 * reads the validation result and the level count back) and returns
 * SPUMA_ERR_NOT_UPPER_TRIANGULAR unless 0 <= l(f) < u(f) < n_cells and the
 * faces are sorted by (l, u) without duplicates.  The handle keeps pointers
 * into the workspace, which must stay allocated and untouched until
 * spuma_ldu_destroy().  The addressing arrays are copied; the caller may free
 * them after create returns.  flags: 0, or SPUMA_WORKSPACE_ASYMMETRIC for a
 * workspace that also holds what spuma_pbicg_solve needs (48F + 16N more
 * bytes); create detects the larger size by itself.
 * ---------------------------------------------------------------------- */
size_t spuma_workspace_bytes(int32_t n_cells, int32_t n_faces, int32_t flags);
spuma_status spuma_ldu_create(int32_t n_cells, int32_t n_faces, const int32_t* lower_addr,
                              const int32_t* upper_addr, void* workspace, size_t workspace_bytes,
                              spuma_stream_t stream, spuma_ldu_t* out);
/* Same, with the cell centres cell_c[N][3] (device, FP64; may be NULL): rows
 * of each DIC level are then stored in the Morton order of their centres
 * instead of ascending cell index.  Only the storage order changes; every
 * result is bit-identical, but the gathers of neighbouring values become
 * local on meshes whose numbering is not (e.g. randomly renumbered ones). */
spuma_status spuma_ldu_create_with_centres(int32_t n_cells, int32_t n_faces, const int32_t* lower_addr,
                                           const int32_t* upper_addr, const double* cell_c,
                                           void* workspace, size_t workspace_bytes,
                                           spuma_stream_t stream, spuma_ldu_t* out);
spuma_status spuma_ldu_destroy(spuma_ldu_t h);
/* Host-side facts of a handle: cell and face count, DIC level count. */
spuma_status spuma_ldu_info(spuma_ldu_t h, int32_t* n_cells, int32_t* n_faces, int32_t* n_levels);
/* Synchronises the stream and returns the device-side status of the last
 * operation on this handle (SPUMA_OK if none failed). */
spuma_status spuma_ldu_device_status(spuma_ldu_t h, spuma_stream_t stream);

/* ------------------------------------------------------------------------
 * Laplacian assembly, "Gauss linear corrected" (paper appendix, fvSchemes
 * listing; "P assembly" rows of the scaling tables, Sec. 4.4).  Implicit part
 * of A = -laplacian(gamma, p):
 *   a_f = (gamma_f |S_f|) / max(n_f . d_f, 0.05 |d_f|),  n_f = S_f/|S_f|,
 *   d_f = C[u(f)] - C[l(f)];  upper_f = -a_f;
 *   diag_i = sum of a_f over the internal faces of i (face order), then plus
 *   a_b = (gamma_b |S_b|)/max(n_b . (Cb_b - C_i), 0.05 |Cb_b - C_i|) for each
 *   Dirichlet boundary face b of cell i (type 1, value 0), in face order.
 *   Zero-gradient faces (type 0) add nothing.
 * Arithmetic order: |S| = sqrt((Sx Sx + Sy Sy) + Sz Sz), n.d =
 * ((Sx dx + Sy dy) + Sz dz)/|S|, a = (gamma |S|)/max(n.d, 0.05 |d|), no
 * fused multiply-add; the result is bit-identical to a sequential face loop.
 * Layout: face_sf[F][3], cell_c[N][3], face_gamma[F]; boundary arrays
 * bface_cell[B], bface_sf[B][3] (outward), bface_cf[B][3], bface_gamma[B],
 * bface_type[B] (int8).  Outputs upper[F], diag[N] (FP64, original order).
 * n_bfaces may be 0 (boundary pointers then may be NULL).
 * ---------------------------------------------------------------------- */
spuma_status spuma_assemble_laplacian(spuma_ldu_t h, const double* face_sf, const double* cell_c,
                                      const double* face_gamma, int32_t n_bfaces,
                                      const int32_t* bface_cell, const double* bface_sf,
                                      const double* bface_cf, const double* bface_gamma,
                                      const int8_t* bface_type, double* upper, double* diag,
                                      spuma_stream_t stream);
/* Reverse mode of the assembly above with respect to the diffusivities, the
 * geometry held fixed (an extension of the paper's method: the chain from
 * the solve's adjoint, spuma_pcg_adjoint, to gamma).  a_f is linear in
 * gamma_f with d a_f / d gamma_f = |S_f| / max(n_f . d_f, 0.05 |d_f|), so
 *   dldgamma_f  = ((dlddiag_{l(f)} + dlddiag_{u(f)}) - dldupper_f) * d a_f / d gamma_f,
 *   dldbgamma_b = dlddiag_{cell(b)} * d a_b / d gamma_b  (Dirichlet faces), 0 (zero gradient).
 * Same geometry arrays and layout as the assembly; dldupper[F], dlddiag[N]
 * in, dldgamma[F] and dldbgamma[B] out (FP64, original order; dldbgamma may
 * be NULL, and so may the boundary arrays when n_bfaces is 0).  One kernel
 * per face set, no atomics: each output element is written once. */
spuma_status spuma_assemble_laplacian_adjoint(spuma_ldu_t h, const double* face_sf, const double* cell_c,
                                              int32_t n_bfaces, const int32_t* bface_cell,
                                              const double* bface_sf, const double* bface_cf,
                                              const int8_t* bface_type, const double* dldupper,
                                              const double* dlddiag, double* dldgamma, double* dldbgamma,
                                              spuma_stream_t stream);

/* ------------------------------------------------------------------------
 * lduMatrix::Amul (paper Sec. 4.2, profiling table "SpMVM (Amul + Tmul)"):
 *   y_i = d_i x_i + sum_{f: u(f)=i} a_f x_{l(f)} + sum_{f: l(f)=i} a_f x_{u(f)}
 * with the terms of row i taken in face order (neighbour-side faces
 * ascending, then owner-side faces ascending), each a fused multiply-add:
 * bit-identical to the sequential face loop y_u += a_f x_l; y_l += a_f x_u.
 * No atomics: a face-to-cell gather.  precision SPUMA_F64: double arrays;
 * SPUMA_F32: float arrays.  Vectors in the caller's (original) cell order.
 * ---------------------------------------------------------------------- */
spuma_status spuma_amul(spuma_ldu_t h, int32_t precision, const void* diag, const void* upper,
                        const void* x, void* y, spuma_stream_t stream);

/* ------------------------------------------------------------------------
 * Prepared matrix.  spuma_matrix_prepare() copies diag/upper into the
 * handle's level-ordered internal layout (FP64 and FP32 copies) and, for
 * SPUMA_PRECOND_DIC, computes the DIC factor
 *   p_i = d_i - sum_{f: u(f)=i, ascending} (a_f a_f)/p_{l(f)},  rD_i = 1/p_i
 * (paper Sec. 4.3, coarse-level DIC), level by level, bit-identical to the
 * sequential face loop; for SPUMA_PRECOND_DIAGONAL rD_i = 1/d_i.
 * spuma_pcg_solve() calls it itself; it is exposed for the Amul benchmark
 * and the parity tests.
 * spuma_read_rD() copies rD (FP64, original order) to rD_out.
 * spuma_amul_prepared(): y = A x on the prepared matrix, vectors in the
 * handle's internal (level) order, the exact kernel phase that PCG runs.
 * spuma_permute(): dir 0 gathers original -> internal, 1 scatters back
 * (FP64 vectors).
 * spuma_precondition(): w = M^-1 r for the prepared preconditioner
 * (original order, FP64):  w_i = rD_i r_i;  forward sweep, faces ascending:
 * w_u -= (rD_u a_f) w_l;  backward sweep, faces descending:
 * w_l -= (rD_l a_f) w_u;  each -= a fused multiply-add of the rounded
 * product, bit-identical to the sequential sweeps.
 * ---------------------------------------------------------------------- */
spuma_status spuma_matrix_prepare(spuma_ldu_t h, const double* diag, const double* upper,
                                  int32_t precond, spuma_stream_t stream);
spuma_status spuma_read_rD(spuma_ldu_t h, double* rD_out, spuma_stream_t stream);
spuma_status spuma_amul_prepared(spuma_ldu_t h, int32_t precision, const void* x_internal,
                                 void* y_internal, spuma_stream_t stream);
spuma_status spuma_permute(spuma_ldu_t h, int32_t dir, const double* src, double* dst,
                           spuma_stream_t stream);
spuma_status spuma_precondition(spuma_ldu_t h, int32_t precond, const double* r, double* w,
                                spuma_stream_t stream);

/* ------------------------------------------------------------------------
 * PCG solve (paper appendix, fvSolution listing: PCG with DIC or diagonal
 * preconditioning; OpenFOAM's PCG recurrences, sumProd/sumMag reductions):
 *   q = A x; r = b - q; normFactor = sum(|q - s xbar| + |b - s xbar|) + 1e-20
 *   (s = row sums, xbar = mean x); res0 = sum|r| / normFactor; then, if
 *   min_iter > 0 or res0 is not converged, repeat
 *     w = M^-1 r; rho = w.r; p = w (first) | w + (rho/rho_old) p;
 *     q = A p; sigma = q.p (singular if |sigma|/normFactor < 1e-300);
 *     alpha = rho/sigma; x += alpha p; r -= alpha q; res = sum|r|/normFactor
 *   while (n_iter < max_iter and not converged) or n_iter < min_iter,
 *   converged: res < tolerance or (rel_tol > 0 and res < rel_tol res0).
 * x is the initial guess on entry and the solution on exit (original order).
 * precision SPUMA_MIXED / SPUMA_MIXED_RESTART: FP32 coefficients, Amul and
 * DIC sweeps inside FP64 refinement (FP64 residual, FP64 reductions, FP64
 * rD).  Reliable updates (MIXED): FP32 PCG on r; when sum|r32| fell below
 * inner_rel_tol times its value at the last update: x += xs, r = b - A x in
 * FP64, r32 = float(r), p kept; stop when the FP64 residual converges.
 * Restarted (MIXED_RESTART): r = b - A x (FP64); stop when sum|r|/normFactor
 * < tolerance or after max_outer steps; s = max|r|; inner FP32 PCG on
 * A d = r/s from d = 0 to inner_rel_tol; x += s d.
 * The whole solve is one persistent cooperative kernel (plus the prepare
 * kernels): no host round trip per iteration.  perf is a DEVICE pointer.
 * ---------------------------------------------------------------------- */
spuma_status spuma_pcg_solve(spuma_ldu_t h, const double* diag, const double* upper,
                             const double* b, double* x, const spuma_solver_controls* ctl,
                             spuma_solver_perf* perf, spuma_stream_t stream);

/* ------------------------------------------------------------------------
 * The same PCG solve without any device allocation (the paper has no
 * counterpart: this serves callers that cannot call cudaMalloc, such as a
 * solver plugin inside an application that owns the device allocator, or a
 * code path that must not pay cudaMalloc's implicit synchronisation).  The
 * mesh topology and all solver scratch live in one static device array of
 * spuma_static_workspace_bytes() bytes (32 MiB, enough for hex meshes of
 * about 65 thousand cells) that every GPU loading the library holds until the
 * process exits; a larger mesh is rejected with SPUMA_ERR_WORKSPACE_TOO_SMALL
 * before any device work.  The caller passes the addressing, the
 * coefficients, b, x (initial guess in, solution out) and perf, all device
 * pointers, as for spuma_ldu_create + spuma_pcg_solve, which this call
 * performs in one go (the topology build waits for the stream).  Every
 * call looks up the array's device address with the current device (the
 * first call on a device also loads the library's device code there: make
 * that first call before any stream capture).  All arguments are checked
 * before the array is touched.  Every call reuses the same array and each
 * call clears what it needs, but calls whose work overlaps on the GPU (other
 * streams, other host threads) race on it.
 * ---------------------------------------------------------------------- */
size_t spuma_static_workspace_bytes(void);
spuma_status spuma_pcg_solve_static(int32_t n_cells, int32_t n_faces, const int32_t* lower_addr,
                                    const int32_t* upper_addr, const double* diag, const double* upper,
                                    const double* b, double* x, const spuma_solver_controls* ctl,
                                    spuma_solver_perf* perf, spuma_stream_t stream);

/* ------------------------------------------------------------------------
 * The pressure-correction step around the solve (the paper's SIMPLE loop
 * with the schemes of its fvSchemes listing: gradSchemes Gauss linear,
 * interpolationSchemes linear, laplacianSchemes Gauss linear corrected,
 * snGradSchemes corrected; nNonOrthogonalCorrectors 0 in its fvSolution).
 * All quantities are integrated over the cell (no division by volume except
 * in the gradient); original order, FP64; the geometry arrays are those of
 * spuma_assemble_laplacian plus face_cf[F][3] (internal face centres) and
 * cell_v[N] (volumes); boundary faces: Dirichlet (type 1) carry p = 0,
 * zero-gradient (type 0) p_b = p_cell.  Every per-cell result is a gather in
 * ascending face order, then the cell's boundary faces in ascending order:
 * bit-identical to the sequential face loop.  These calls use the handle's
 * vector region as scratch (as the assembly does): do not overlap them with
 * a solve on the same handle.  spuma_fv_grad and spuma_pressure_rhs also
 * use the matrix region for a face-indexed scratch: a matrix prepared with
 * spuma_matrix_prepare() must be prepared again after them (a solve always
 * prepares its own).  The per-cell lists of boundary faces are built on the
 * first call with a given (bface_cell pointer, n_bfaces) and reused while
 * calls pass the same pair: a mesh's boundary topology is fixed (a boundary
 * with more than two faces per cell on average is listed on every call).
 *
 * spuma_fv_weights: w[F], the owner weight of the linear interpolation
 *   p_f = w p_l + (1 - w) p_u, w = |S.(C_u - C_f)| / (|S.(C_f - C_l)| + |S.(C_u - C_f)|).
 * spuma_fv_grad: grad[N][3] = (1/V_i) sum_f S_f p_f (outward S: +S_f for the
 *   owner, -S_f for the neighbour; boundary S_b p_b).
 * spuma_pressure_rhs: corr[F] = (gamma_f |S_f|) (k_f . (w grad_l + (1 - w) grad_u)),
 *   the explicit non-orthogonal correction of the corrected laplacian, with
 *   k_f = S_f/|S_f| - d_f / max(n.d, 0.05 |d|) and d_f = C_u - C_l; and
 *   b[N] = sum_f +-(corr_f - phi_f) (+ owner, - neighbour) - sum_b phi_b, so
 *   that laplacian(gamma, p) = div(phiHbyA) reads A p = b with the (upper,
 *   diag) of spuma_assemble_laplacian.  phi[F], bphi[B]: phiHbyA.
 * spuma_pressure_flux: phi_out_f = phi_f - (a_f (p_u - p_l) + corr_f), a_f =
 *   -upper_f; bphi_out_b = bphi_b + a_b p_cell on Dirichlet faces (a_b the
 *   assembly's boundary coefficient), bphi_b on zero-gradient ones.  With p
 *   from A p = b the result is divergence-free to the solver tolerance.
 * spuma_fv_div: div[N] = sum_f +-phi_f + sum_b bphi_b (integrated).
 * ---------------------------------------------------------------------- */
spuma_status spuma_fv_weights(spuma_ldu_t h, const double* face_sf, const double* face_cf, const double* cell_c,
                              double* w, spuma_stream_t stream);
spuma_status spuma_fv_grad(spuma_ldu_t h, const double* face_sf, const double* w, const double* cell_v,
                           int32_t n_bfaces, const int32_t* bface_cell, const double* bface_sf,
                           const int8_t* bface_type, const double* p, double* grad, spuma_stream_t stream);
spuma_status spuma_pressure_rhs(spuma_ldu_t h, const double* face_sf, const double* cell_c, const double* w,
                                const double* face_gamma, const double* grad, const double* phi,
                                int32_t n_bfaces, const int32_t* bface_cell, const double* bphi, double* corr,
                                double* b, spuma_stream_t stream);
spuma_status spuma_pressure_flux(spuma_ldu_t h, const double* upper, const double* corr, const double* p,
                                 const double* phi, int32_t n_bfaces, const int32_t* bface_cell,
                                 const double* bface_sf, const double* bface_cf, const double* bface_gamma,
                                 const int8_t* bface_type, const double* cell_c, const double* bphi,
                                 double* phi_out, double* bphi_out, spuma_stream_t stream);
spuma_status spuma_fv_div(spuma_ldu_t h, const double* phi, int32_t n_bfaces, const int32_t* bface_cell,
                          const double* bphi, double* div, spuma_stream_t stream);

/* ------------------------------------------------------------------------
 * PBiCG on an asymmetric LDU matrix (the paper's solver for U, k and omega:
 * "PBiCG, preconditioner aDILU" in its fvSolution listing; "SpMVM (Amul +
 * Tmul)" and "aDILUPreconditioner" in its profiling table, Sec. 4.2).
 * A_{u(f),l(f)} = lower_f, A_{l(f),u(f)} = upper_f (OpenFOAM lduMatrix).
 * OpenFOAM's bi-conjugate gradients: rA = b - A x, rT = b - A^T x; each
 * iteration wA = M^-1 rA, wT = M^-T rT, wArA = wA.rT, pA = wA + beta pA,
 * pT = wT + beta pT (beta = wArA/wArA_old), wA = A pA, wT = A^T pT,
 * alpha = wArA/(wA.pT), x += alpha pA, rA -= alpha wA, rT -= alpha wT;
 * residual, normFactor (row sums of A), singular test and stopping rule as
 * spuma_pcg_solve.  Preconditioners: NONE, DIAGONAL, or DILU (M = (D + L)
 * D^-1 (D + U), pivots d_u -= upper_f lower_f / d_l in face order, applied
 * with the level-scheduled sweeps of the DIC path, one level per grid
 * barrier; M^-T with lower and upper exchanged).  FP64 only (precision must
 * be SPUMA_F64).  One persistent cooperative launch; x in/out (initial
 * guess), perf as spuma_pcg_solve.  The workspace must have been sized with
 * SPUMA_WORKSPACE_ASYMMETRIC, else SPUMA_ERR_WORKSPACE_TOO_SMALL; a zero or
 * non-finite DILU pivot is reported as SPUMA_ERR_SINGULAR in perf.status.
 * Invalidates a spuma_matrix_prepare()'d symmetric matrix.
 * ---------------------------------------------------------------------- */
spuma_status spuma_pbicg_solve(spuma_ldu_t h, const double* diag, const double* lower, const double* upper,
                               const double* b, double* x, const spuma_solver_controls* ctl,
                               spuma_solver_perf* perf, spuma_stream_t stream);

/* ------------------------------------------------------------------------
 * GAMG for the pressure equation (the paper's production pressure solver:
 * "GAMG, smoother Richardson" in its fvSolution listing; Richardson (damped
 * Jacobi) on every level and a diagonal PCG at the coarsest one, with
 * OpenFOAM's coarsening unmodified, Sec. 4.3).
 * spuma_gamg_create: builds the level hierarchy on the HOST (synchronous;
 *   it copies the addressing and face_weight[F] (device, e.g. |S_f|) back):
 *   pairwise agglomeration by face weight, cells in ascending order (pair
 *   with the unassigned neighbour across the heaviest face, first in face
 *   order on ties; join the aggregate across the heaviest face when all
 *   neighbours are taken; no faces: stay alone); coarse faces between
 *   different aggregates, sorted by (min, max), weights summed; levels added
 *   while the coarse level has more than 10 cells and fewer than the level
 *   above.  The independent passes of the build run on the host's cores
 *   (the agglomeration itself is sequential); a host allocation or thread
 *   failure returns SPUMA_ERR_HOST.  spuma_gamg_workspace_bytes then gives
 *   the device workspace that spuma_gamg_bind takes (256-byte aligned;
 *   synchronous upload).
 * spuma_gamg_solve: one persistent cooperative launch: Galerkin coarse
 *   matrices P^T A P (P piecewise constant; sums in ascending fine order:
 *   upper_F = sum of the fine upper_f of F; diag_C = sum of the fine diag of
 *   C, then + 2 upper_f of each fine face inside C), then the iterations
 *   x += V(0, r), r = b - A x with PCG's normalised residual, normFactor and
 *   stopping rule (tolerance, rel_tol, max_iter, min_iter; precision F64).
 *   V(k, r): no pre-smoothing; r_{k+1} = sum over each aggregate; at the
 *   coarsest level diagonal PCG from 0 to 1e-8 relative; e_k = injection of
 *   e_{k+1}, scaled by (e.r)/(e.A e) when e.A e > 0; two damped-Jacobi sweeps
 *   e_i = fma(omega/d_i, r_i - (A e)_i, e_i), omega = 2/3.  x in/out (initial
 *   guess), original order; perf as spuma_pcg_solve (n_levels = GAMG levels).
 *   The hierarchy's handle h must outlive the GAMG object; its status and
 *   barrier words are shared with h's other calls (stream-ordered).  With
 *   two or more levels, level 0 runs in h's internal (DIC level) order: its
 *   coefficients are gathered into h's FP64 matrix region, so a matrix
 *   prepared on h before (spuma_matrix_prepare) must be prepared again before
 *   spuma_amul_prepared or spuma_precondition (spuma_precondition returns
 *   SPUMA_ERR_INVALID_ARG until then; spuma_pcg_solve prepares its own).
 * ---------------------------------------------------------------------- */
/* spuma_gamg_set_options: the smoother of later solves, SPUMA_GAMG_RICHARDSON
 *   (default; damped Jacobi as above) or SPUMA_GAMG_GAUSS_SEIDEL_2STAGE (the
 *   paper's second parallel smoother, after Berger-Vergiat et al.: each sweep
 *   q = r - A e, y = q/d, e_i += (q_i - sum over the row's lower entries in
 *   face order of a_f y_col)/d_i, the Gauss-Seidel lower solve replaced by one
 *   Jacobi step and one Jacobi-Richardson sweep; 1/d rounded once, each
 *   product rounded, one FMA per lower term), and the coarsest level's PCG
 *   preconditioner, SPUMA_PRECOND_DIAGONAL (default) or SPUMA_PRECOND_DIC
 *   (the profiling run's "coarsestSolver=DIC+PCG"; factor and sweeps in the
 *   sequential face order, by one thread: the coarsest level has about ten
 *   cells).  Host only; no device work. */
#define SPUMA_GAMG_RICHARDSON 0
#define SPUMA_GAMG_GAUSS_SEIDEL_2STAGE 1
typedef struct spuma_gamg* spuma_gamg_t;
spuma_status spuma_gamg_create(spuma_ldu_t h, const double* face_weight, spuma_stream_t stream, spuma_gamg_t* out);
size_t spuma_gamg_workspace_bytes(spuma_gamg_t g);
spuma_status spuma_gamg_bind(spuma_gamg_t g, void* workspace, size_t workspace_bytes, spuma_stream_t stream);
spuma_status spuma_gamg_info(spuma_gamg_t g, int32_t* n_levels, int32_t* level_cells, int32_t max_levels);
spuma_status spuma_gamg_solve(spuma_gamg_t g, const double* diag, const double* upper, const double* b, double* x,
                              const spuma_solver_controls* ctl, spuma_solver_perf* perf, spuma_stream_t stream);
spuma_status spuma_gamg_set_options(spuma_gamg_t g, int32_t smoother, int32_t coarsest_precond);
spuma_status spuma_gamg_destroy(spuma_gamg_t g);

/* ------------------------------------------------------------------------
 * Adjoint of x = A^-1 b for a loss L(x), given x and dldx = dL/dx:
 *   A lambda = dldx (A symmetric: A^T = A, same PCG, lambda from 0);
 *   dL/db = lambda;  dL/dupper_f = -(lambda_{l(f)} x_{u(f)} + lambda_{u(f)} x_{l(f)});
 *   dL/ddiag_i = -lambda_i x_i  (dlddiag may be NULL).
 * x is taken as given (recomputed by the caller's forward), no Krylov
 * history is kept.  Outputs in original order: dldb[N], dldupper[F].
 * ---------------------------------------------------------------------- */
spuma_status spuma_pcg_adjoint(spuma_ldu_t h, const double* diag, const double* upper,
                               const double* x, const double* dldx, double* dldb,
                               double* dldupper, double* dlddiag, const spuma_solver_controls* ctl,
                               spuma_solver_perf* perf, spuma_stream_t stream);

/* ------------------------------------------------------------------------
 * Batched solve: n_sys independent systems (each with its own handle and
 * workspace) in ONE persistent cooperative launch (an extension of the
 * paper's pressure solve to many small systems); each system converges on its own
 * (per-system device-side convergence) with the controls *ctl.  Arrays of
 * n_sys DEVICE pointers are passed as HOST arrays; perf[n_sys] is device
 * memory.  spuma_batch_create() records the pointers, picks the block size,
 * the weighting of the grid split between systems and the grid size with the
 * library's autotuner when flags has SPUMA_BATCH_AUTOTUNE (timed trial solves
 * on the stream from x = 0, the caller's x untouched; a staged search over
 * block sizes 64..1024, split weights cells^{1, 4/3, 5/3} and a full or
 * half-size grid; cached per problem signature in memory and, when
 * SPUMA_TUNE_CACHE names a file, in that JSON file), and captures the launch
 * (barrier resets + the kernel) in a CUDA graph that spuma_batch_run()
 * replays.  A failed capture is an error (SPUMA_ERR_CUDA, the reason in
 * spuma_last_error) unless flags has SPUMA_BATCH_ALLOW_DIRECT, which replays
 * by direct launches instead; SPUMA_BATCH_NO_GRAPH skips the capture.
 * spuma_batch_info() reports the chosen block size, grid, the tuned time (-1
 * when not tuned) and whether a graph was captured; spuma_batch_trials()
 * copies the candidates the tuner timed (up to max_trials) and returns their
 * count (0 after a cache hit or without tuning).
 * spuma_batch_solve() is the one-shot form (no graph, no tuning).
 * ---------------------------------------------------------------------- */
#define SPUMA_BATCH_AUTOTUNE 1
#define SPUMA_BATCH_ALLOW_DIRECT 2
#define SPUMA_BATCH_NO_GRAPH 4
spuma_status spuma_batch_create(int32_t n_sys, const spuma_ldu_t* hs, const double* const* diag,
                                const double* const* upper, const double* const* b,
                                double* const* x, const spuma_solver_controls* ctl,
                                spuma_solver_perf* perf, int32_t flags, spuma_stream_t stream,
                                spuma_batch_t* out);
spuma_status spuma_batch_run(spuma_batch_t bt, spuma_stream_t stream);
spuma_status spuma_batch_info(spuma_batch_t bt, int32_t* block_threads, int32_t* grid_blocks,
                              double* tuned_ms, int32_t* graph_captured);
int32_t spuma_batch_trials(spuma_batch_t bt, int32_t max_trials, int32_t* block_threads,
                           int32_t* split_policy, int32_t* grid_blocks, double* ms);
spuma_status spuma_batch_destroy(spuma_batch_t bt);
spuma_status spuma_batch_solve(int32_t n_sys, const spuma_ldu_t* hs, const double* const* diag,
                               const double* const* upper, const double* const* b,
                               double* const* x, const spuma_solver_controls* ctl,
                               spuma_solver_perf* perf, spuma_stream_t stream);

/* Host-only helpers of the batch autotuner (no device work).
 * spuma_batch_split: split grid blocks between n_sys systems in proportion to
 * weights[], at least one block each, largest-remainder rounding; writes
 * split_out[0..n_sys] (block ranges) and returns 1, or 0 when grid < n_sys.
 * spuma_tune_cache_lookup / _store: the tuner's cache, kept in memory and,
 * when path is not NULL or empty, in a JSON file whose lines read
 *   "signature": [block_threads, split_policy, grid_div, milliseconds],
 * (split_policy: 0, 1, 2 for weights cells^1, ^(4/3), ^(5/3); grid_div: the
 * co-resident grid divided by 1 or 2).  Lookup returns 1 on a hit; store
 * returns 1 on success.                                                    */
int32_t spuma_batch_split(int32_t n_sys, const double* weights, int32_t grid, int32_t* split_out);
int32_t spuma_tune_cache_lookup(const char* path, const char* signature, int32_t* block_threads,
                                int32_t* split_policy, int32_t* grid_div, double* ms);
int32_t spuma_tune_cache_store(const char* path, const char* signature, int32_t block_threads,
                               int32_t split_policy, int32_t grid_div, double ms);

/* ------------------------------------------------------------------------
 * Diagnostics.
 * spuma_status_string: static text of a status.  spuma_last_error: text of
 * the last host-side error of the calling thread.  spuma_launch_count: the
 * number of kernels this library has launched in the process (a counter on
 * the host, for benchmarks).  spuma_set_barrier_timeout_ns: time limit of
 * every device-side grid-barrier wait in later launches (default 2 s); a test
 * sets it to 0 to check that an expired wait returns
 * SPUMA_ERR_DEVICE_TIMEOUT instead of hanging.
 * ---------------------------------------------------------------------- */
/* spuma_read_phase_clocks: when the environment variable SPUMA_PHASE_CLOCKS
 * is set at launch, the solver's first block adds SM-clock cycles per phase
 * into a table in the workspace (slots 0..63 forward DIC level L, 64..127
 * backward level L, 128 search direction, 129 Amul + p.Ap, 130 diagonal
 * pass, 132 FP64 refinement residual, 134 x/r update pass, 140 PCG
 * iterations); this copies the first n entries (synchronous).  More
 * variables change how later solves run, never what they compute (read once
 * per process): SPUMA_SOLVE_BLOCKS_PER_SM caps the solver's blocks per SM,
 * SPUMA_TAIL_ROWS sets the row limit of the small last DIC levels that the
 * first block sweeps alone (0: none), SPUMA_SWEEP=0 strides a level's
 * rows over the blocks instead of giving each block one contiguous chunk of
 * every level, SPUMA_AMUL_CHUNKS=1 makes the PCG's Amul phase walk those
 * chunks too (on meshes whose levels are wide), and
 * SPUMA_GAMG_FUSE_SCALE_ROWS=n makes GAMG's coarse levels of at most n
 * cells apply the correction's scaling inside their first smoothing sweep
 * (0, the default: a pass of its own); SPUMA_GAMG_ORDER=inherited (read by
 * spuma_gamg_create) stores GAMG's middle levels in the order inherited
 * from the level above instead of breadth-first.  With SPUMA_PHASE_CLOCKS a GAMG
 * solve fills the same table per V-cycle: 0..49 restriction into level
 * k+1, 64..113 prolongation, scaling and smoothing of level k, 128 the
 * coarsest level, 129 the outer update and residual, 130 V-cycles.        */
spuma_status spuma_read_phase_clocks(spuma_ldu_t h, int64_t* out, int32_t n, spuma_stream_t stream);
const char* spuma_status_string(int32_t status);
const char* spuma_last_error(void);
uint64_t spuma_launch_count(void);
void spuma_set_barrier_timeout_ns(uint64_t ns);

#ifdef __cplusplus
}
#endif
#endif /* SPUMA_H */
