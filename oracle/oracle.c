/*
 * oracle.c -- plain, sequential CPU reference of the LDU pressure-solve path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The CUDA library
 * shares no code with it.
 *
 * Every loop runs in the order the method states it: faces ascending (or
 * descending for the backward DIC sweep), cells ascending.  Build with
 * -O2 -ffp-contract=off so that the compiler fuses nothing; where the method
 * is read as a fused multiply-add (the row sums of Amul and the DIC sweeps,
 * and the Krylov vector recurrences x += alpha p, r -= alpha q, p = w + beta p
 * of PCG, PBiCG and the mixed forms, as an FMA-contracting build of
 * OpenFOAM computes them) the code calls fma()/fmaf() explicitly.
 *
 * Matrix: OpenFOAM's lduMatrix ("LDUorderedCOO", paper Sec. 2.1): diag[N],
 * upper[F] (symmetric, lower == upper), lowerAddr l[F] (owner) and upperAddr
 * u[F] (neighbour) with l(f) < u(f), faces sorted by (l, u).
 * Sign convention: A = -(OpenFOAM laplacian) so that A is SPD (diag > 0,
 * upper < 0).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Laplacian assembly, "Gauss linear corrected" (paper appendix, fvSchemes   */
/* listing: laplacianSchemes default Gauss linear corrected, snGradSchemes   */
/* corrected).  Implicit part only; the explicit non-orthogonal correction   */
/* goes to the source and is absent because b is given.                      */
/*   a_f  = (gamma_f |S_f|) / max(n.d, 0.05 |d|),  n = S_f/|S_f|,            */
/*          d = C_u - C_l                                                    */
/*   upper_f = -a_f;  diag_i = sum of a_f over the faces of i in face order, */
/*   then + a_b of each Dirichlet boundary face of i (value 0) in face order */
/* Exact operation order (shared definition with the GPU kernels):           */
/*   |S| = sqrt((Sx*Sx + Sy*Sy) + Sz*Sz); n.d = ((Sx*dx + Sy*dy) + Sz*dz)/|S| */
/*   denom = fmax(n.d, 0.05*|d|); a = (gamma*|S|)/denom                       */
/* ------------------------------------------------------------------------ */
static double face_coeff(const double* s, const double* cp, const double* cn, double gamma)
{
    double sx = s[0], sy = s[1], sz = s[2];
    double dx = cn[0] - cp[0], dy = cn[1] - cp[1], dz = cn[2] - cp[2];
    double mags = sqrt((sx * sx + sy * sy) + sz * sz);
    double magd = sqrt((dx * dx + dy * dy) + dz * dz);
    double ndotd = ((sx * dx + sy * dy) + sz * dz) / mags;
    double denom = fmax(ndotd, 0.05 * magd);
    return (gamma * mags) / denom;
}

void oracle_assemble_laplacian(int32_t n_cells, int32_t n_faces, const int32_t* l, const int32_t* u,
                               const double* sf, const double* c, const double* gamma,
                               int32_t n_b, const int32_t* bcell, const double* bsf,
                               const double* bcf, const double* bgamma, const int8_t* btype,
                               double* upper, double* diag)
{
    for (int32_t i = 0; i < n_cells; i++) diag[i] = 0.0;
    for (int32_t f = 0; f < n_faces; f++) {
        double a = face_coeff(sf + 3 * (int64_t)f, c + 3 * (int64_t)l[f], c + 3 * (int64_t)u[f], gamma[f]);
        upper[f] = -a;
        diag[l[f]] += a;
        diag[u[f]] += a;
    }
    for (int32_t b = 0; b < n_b; b++) {
        if (btype[b] != 1) continue;              /* zero gradient adds nothing */
        int32_t i = bcell[b];
        diag[i] += face_coeff(bsf + 3 * (int64_t)b, c + 3 * (int64_t)i, bcf + 3 * (int64_t)b, bgamma[b]);
    }
}

/* ------------------------------------------------------------------------ */
/* Reverse mode of the assembly above with respect to the diffusivities,     */
/* the geometry held fixed.  a_f is linear in gamma_f:                       */
/*   d a_f / d gamma_f = |S_f| / max(n.d, 0.05 |d|)  (face_coeff at gamma 1) */
/* and a_f enters upper_f with sign -1 and diag_l, diag_u with sign +1, a_b  */
/* (Dirichlet) enters diag of its cell.  Given gu = dL/dupper, gd = dL/ddiag:*/
/*   dL/dgamma_f = ((gd_l + gd_u) - gu_f) * (d a_f / d gamma_f)             */
/*   dL/dbgamma_b = gd_cell * (d a_b / d gamma_b)  (Dirichlet), 0 otherwise  */
/* ------------------------------------------------------------------------ */
void oracle_assembly_adjoint(int32_t n_faces, const int32_t* l, const int32_t* u, const double* sf,
                             const double* c, int32_t n_b, const int32_t* bcell, const double* bsf,
                             const double* bcf, const int8_t* btype, const double* gu, const double* gd,
                             double* ggamma, double* gbgamma)
{
    for (int32_t f = 0; f < n_faces; f++) {
        double da = face_coeff(sf + 3 * (int64_t)f, c + 3 * (int64_t)l[f], c + 3 * (int64_t)u[f], 1.0);
        ggamma[f] = ((gd[l[f]] + gd[u[f]]) - gu[f]) * da;
    }
    for (int32_t b = 0; b < n_b; b++) {
        if (btype[b] != 1) {
            gbgamma[b] = 0.0;
            continue;
        }
        int32_t i = bcell[b];
        double da = face_coeff(bsf + 3 * (int64_t)b, c + 3 * (int64_t)i, bcf + 3 * (int64_t)b, 1.0);
        gbgamma[b] = gd[i] * da;
    }
}

/* ------------------------------------------------------------------------ */
/* lduMatrix::Amul (paper Sec. 4.2 profiling table, "SpMVM (Amul + Tmul)"):   */
/*   y_i = d_i x_i, then for each face f ascending:                          */
/*   y_u += a_f x_l ; y_l += a_f x_u   (each += one fused multiply-add)      */
/* ------------------------------------------------------------------------ */
void oracle_amul(int32_t n, int32_t nf, const int32_t* l, const int32_t* u,
                 const double* diag, const double* upper, const double* x, double* y)
{
    for (int32_t i = 0; i < n; i++) y[i] = diag[i] * x[i];
    for (int32_t f = 0; f < nf; f++) {
        y[u[f]] = fma(upper[f], x[l[f]], y[u[f]]);
        y[l[f]] = fma(upper[f], x[u[f]], y[l[f]]);
    }
}

void oracle_amul_f32(int32_t n, int32_t nf, const int32_t* l, const int32_t* u,
                     const float* diag, const float* upper, const float* x, float* y)
{
    for (int32_t i = 0; i < n; i++) y[i] = diag[i] * x[i];
    for (int32_t f = 0; f < nf; f++) {
        y[u[f]] = fmaf(upper[f], x[l[f]], y[u[f]]);
        y[l[f]] = fmaf(upper[f], x[u[f]], y[l[f]]);
    }
}

/* ------------------------------------------------------------------------ */
/* DIC factor (preconditioner named in the paper, Sec. 4.3, Table of         */
/* smoothers / coarse-level preconditioners): pivots                          */
/*   p_i = d_i; for f ascending: p_u -= (a_f a_f) / p_l;  rD_i = 1 / p_i      */
/* Returns -1, or the first cell whose pivot is not > 0 (then rD is partial). */
/* ------------------------------------------------------------------------ */
int32_t oracle_dic_factor(int32_t n, int32_t nf, const int32_t* l, const int32_t* u,
                          const double* diag, const double* upper, double* rD)
{
    for (int32_t i = 0; i < n; i++) rD[i] = diag[i];
    for (int32_t f = 0; f < nf; f++) rD[u[f]] -= (upper[f] * upper[f]) / rD[l[f]];
    int32_t bad = -1;
    for (int32_t i = 0; i < n; i++) {
        if (!(rD[i] > 0.0) && bad < 0) bad = i;
        rD[i] = 1.0 / rD[i];
    }
    return bad;
}

/* DIC apply:  w_i = rD_i r_i;
 *   forward,  f ascending:  w_u -= (rD_u a_f) w_l
 *   backward, f descending: w_l -= (rD_l a_f) w_u
 * each -= one fused multiply-add of the rounded product (rD a_f).          */
void oracle_dic_precondition(int32_t n, int32_t nf, const int32_t* l, const int32_t* u,
                             const double* upper, const double* rD, const double* r, double* w)
{
    for (int32_t i = 0; i < n; i++) w[i] = rD[i] * r[i];
    for (int32_t f = 0; f < nf; f++) {
        double c = rD[u[f]] * upper[f];
        w[u[f]] = fma(-c, w[l[f]], w[u[f]]);
    }
    for (int32_t f = nf - 1; f >= 0; f--) {
        double c = rD[l[f]] * upper[f];
        w[l[f]] = fma(-c, w[u[f]], w[l[f]]);
    }
}

/* Single-precision sweeps of the mixed form: rD comes from the FP64 factor;
 * the sweep coefficient is the FP64 product rD*a rounded to float, the
 * diagonal scale is rD rounded to float.                                    */
void oracle_dic_precondition_f32(int32_t n, int32_t nf, const int32_t* l, const int32_t* u,
                                 const double* upper64, const double* rD64, const float* r, float* w)
{
    for (int32_t i = 0; i < n; i++) w[i] = (float)rD64[i] * r[i];
    for (int32_t f = 0; f < nf; f++) {
        float c = (float)(rD64[u[f]] * upper64[f]);
        w[u[f]] = fmaf(-c, w[l[f]], w[u[f]]);
    }
    for (int32_t f = nf - 1; f >= 0; f--) {
        float c = (float)(rD64[l[f]] * upper64[f]);
        w[l[f]] = fmaf(-c, w[u[f]], w[l[f]]);
    }
}

/* Diagonal preconditioner (fvSolution listing, pcgDiag): rD_i = 1/d_i once,
 * then w_i = rD_i r_i.                                                      */
void oracle_diag_reciprocal(int32_t n, const double* diag, double* rD)
{
    for (int32_t i = 0; i < n; i++) rD[i] = 1.0 / diag[i];
}

/* ------------------------------------------------------------------------ */
/* PCG with OpenFOAM semantics (fvSolution listing: tolerance, relTol,        */
/* maxIter, minIter; solverPerformance report).                               */
/*   q = A x; r = b - q                                                       */
/*   normFactor = sum(|q - s xbar| + |b - s xbar|) + 1e-20, s = row sums,     */
/*                xbar = mean(x)                                              */
/*   res0 = sum|r| / normFactor                                               */
/*   if min_iter > 0 or not converged(res0):                                  */
/*     repeat: rho_old = rho; w = M^-1 r; rho = w.r;                          */
/*             p = w (first) else p = w + (rho/rho_old) p;                    */
/*             q = A p; sigma = q.p; if |sigma|/normFactor < 1e-300: singular */
/*             alpha = rho/sigma; x += alpha p; r -= alpha q;                 */
/*             res = sum|r|/normFactor; n_iter++                              */
/*     while (n_iter < max_iter and not converged(res)) or n_iter < min_iter  */
/*   converged(res): res < tol or (rel_tol > 0 and res < rel_tol res0)        */
/* precond: 0 none, 1 diagonal, 2 DIC.                                        */
/* perf[0] initial residual, perf[1] final residual, perf[2] n_iter,          */
/* perf[3] singular (0/1), perf[4] converged (0/1).                           */
/* Returns 0, or -2 when the DIC pivot check fails.                           */
/* ------------------------------------------------------------------------ */
static double sum_mag(int32_t n, const double* v)
{
    double s = 0.0;
    for (int32_t i = 0; i < n; i++) s += fabs(v[i]);
    return s;
}

static double sum_prod(int32_t n, const double* a, const double* b)
{
    double s = 0.0;
    for (int32_t i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

static int converged(double res, double res0, double tol, double rel_tol)
{
    return res < tol || (rel_tol > 0.0 && res < rel_tol * res0);
}

double oracle_norm_factor(int32_t n, int32_t nf, const int32_t* l, const int32_t* u,
                          const double* diag, const double* upper, const double* x,
                          const double* b, const double* q)
{
    double* s = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int32_t i = 0; i < n; i++) s[i] = diag[i];
    for (int32_t f = 0; f < nf; f++) { s[l[f]] += upper[f]; s[u[f]] += upper[f]; }
    double xbar = 0.0;
    for (int32_t i = 0; i < n; i++) xbar += x[i];
    xbar = n > 0 ? xbar / (double)n : 0.0;
    double nfac = 0.0;
    for (int32_t i = 0; i < n; i++) {
        double t = s[i] * xbar;
        nfac += fabs(q[i] - t) + fabs(b[i] - t);
    }
    free(s);
    return nfac + 1e-20;
}

int32_t oracle_pcg(int32_t n, int32_t nf, const int32_t* l, const int32_t* u,
                   const double* diag, const double* upper, const double* b, double* x,
                   int32_t precond, double tol, double rel_tol, int32_t max_iter,
                   int32_t min_iter, double* perf)
{
    size_t bytes = sizeof(double) * (size_t)(n > 0 ? n : 1);
    double* r = (double*)malloc(bytes);
    double* w = (double*)malloc(bytes);
    double* p = (double*)malloc(bytes);
    double* q = (double*)malloc(bytes);
    double* rD = (double*)malloc(bytes);
    int32_t status = 0;
    memset(perf, 0, 5 * sizeof(double));

    oracle_amul(n, nf, l, u, diag, upper, x, q);
    for (int32_t i = 0; i < n; i++) r[i] = b[i] - q[i];
    double nfac = oracle_norm_factor(n, nf, l, u, diag, upper, x, b, q);
    double res0 = sum_mag(n, r) / nfac;
    double res = res0;
    int32_t it = 0, singular = 0;

    if (precond == 2) {
        if (oracle_dic_factor(n, nf, l, u, diag, upper, rD) >= 0) { status = -2; goto done; }
    } else if (precond == 1) {
        oracle_diag_reciprocal(n, diag, rD);
    }

    if (min_iter > 0 || !converged(res0, res0, tol, rel_tol)) {
        double rho = 1.0, rho_old;
        do {
            rho_old = rho;
            if (precond == 2) oracle_dic_precondition(n, nf, l, u, upper, rD, r, w);
            else if (precond == 1) for (int32_t i = 0; i < n; i++) w[i] = rD[i] * r[i];
            else for (int32_t i = 0; i < n; i++) w[i] = r[i];
            rho = sum_prod(n, w, r);
            if (it == 0) {
                for (int32_t i = 0; i < n; i++) p[i] = w[i];
            } else {
                double beta = rho / rho_old;
                for (int32_t i = 0; i < n; i++) p[i] = fma(beta, p[i], w[i]);
            }
            oracle_amul(n, nf, l, u, diag, upper, p, q);
            double sigma = sum_prod(n, q, p);
            if (fabs(sigma) / nfac < 1e-300) { singular = 1; break; }
            double alpha = rho / sigma;
            for (int32_t i = 0; i < n; i++) {
                x[i] = fma(alpha, p[i], x[i]);
                r[i] = fma(-alpha, q[i], r[i]);
            }
            res = sum_mag(n, r) / nfac;
        } while ((++it < max_iter && !converged(res, res0, tol, rel_tol)) || it < min_iter);
    }
done:
    perf[0] = res0;
    perf[1] = res;
    perf[2] = (double)it;
    perf[3] = (double)singular;
    perf[4] = (double)converged(res, res0, tol, rel_tol);
    free(r); free(w); free(p); free(q); free(rD);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Mixed precision: FP32 inner PCG (FP32 storage of the coefficients and of  */
/* the vectors, FP32 Amul and DIC sweeps) inside FP64 iterative refinement.  */
/* FP64: the outer residual r = b - A x with the FP64 coefficients, the      */
/* reductions (dot products and norms accumulate in double), the DIC factor  */
/* rD, the scalars alpha and beta, and the correction x += s d.              */
/*   outer: r = b - A64 x; res = sum|r|/normFactor (normFactor as in PCG,     */
/*          from the initial x); stop when converged(res) with the outer     */
/*          count >= 1 or res reached; s = max|r|; inner solve of             */
/*          A32 d = float(r/s) from d = 0 to inner_rel_tol (relative to the   */
/*          inner initial residual) or max_iter; x += s d.                    */
/* perf: [0] initial res, [1] final res, [2] total inner iterations,          */
/*       [3] singular, [4] converged, [5] outer iterations                   */
/* ------------------------------------------------------------------------ */
static double sum_prod_f32(int32_t n, const float* a, const float* b)
{
    double s = 0.0;
    for (int32_t i = 0; i < n; i++) s += (double)a[i] * (double)b[i];
    return s;
}

static double sum_mag_f32(int32_t n, const float* v)
{
    double s = 0.0;
    for (int32_t i = 0; i < n; i++) s += fabs((double)v[i]);
    return s;
}

int32_t oracle_mixed_ir(int32_t n, int32_t nf, const int32_t* l, const int32_t* u,
                        const double* diag, const double* upper, const double* b, double* x,
                        int32_t precond, double tol, double inner_rel_tol, int32_t max_iter,
                        int32_t max_outer, double* perf)
{
    size_t b64 = sizeof(double) * (size_t)(n > 0 ? n : 1);
    size_t b32 = sizeof(float) * (size_t)(n > 0 ? n : 1);
    size_t bf32 = sizeof(float) * (size_t)(nf > 0 ? nf : 1);
    double* r = (double*)malloc(b64);
    double* q64 = (double*)malloc(b64);
    double* rD = (double*)malloc(b64);
    float* d32 = (float*)malloc(b32);
    float* u32 = (float*)malloc(bf32);
    float* ri = (float*)malloc(b32);
    float* di = (float*)malloc(b32);
    float* w = (float*)malloc(b32);
    float* p = (float*)malloc(b32);
    float* q = (float*)malloc(b32);
    float* rD32 = (float*)malloc(b32);
    int32_t status = 0, total_it = 0, outer = 0, singular = 0;
    memset(perf, 0, 6 * sizeof(double));

    for (int32_t i = 0; i < n; i++) d32[i] = (float)diag[i];
    for (int32_t f = 0; f < nf; f++) u32[f] = (float)upper[f];
    if (precond == 2) {
        if (oracle_dic_factor(n, nf, l, u, diag, upper, rD) >= 0) { status = -2; goto done; }
    } else if (precond == 1) {
        oracle_diag_reciprocal(n, diag, rD);
    }
    for (int32_t i = 0; i < n; i++) rD32[i] = (float)rD[i];

    oracle_amul(n, nf, l, u, diag, upper, x, q64);
    double nfac = oracle_norm_factor(n, nf, l, u, diag, upper, x, b, q64);
    double res0 = 0.0, res = 0.0;
    for (;;) {
        oracle_amul(n, nf, l, u, diag, upper, x, q64);
        for (int32_t i = 0; i < n; i++) r[i] = b[i] - q64[i];
        res = sum_mag(n, r) / nfac;
        if (outer == 0) res0 = res;
        if (res < tol || outer >= max_outer || singular) break;
        double s = 0.0;
        for (int32_t i = 0; i < n; i++) if (fabs(r[i]) > s) s = fabs(r[i]);
        if (s == 0.0) break;
        for (int32_t i = 0; i < n; i++) { ri[i] = (float)(r[i] / s); di[i] = 0.0f; }
        /* inner FP32 PCG from d = 0: q = A d = 0, normFactor = sum|ri| + 1e-20 */
        double infac = sum_mag_f32(n, ri) + 1e-20;
        double ires0 = sum_mag_f32(n, ri) / infac, ires = ires0;
        double rho = 1.0, rho_old;
        int32_t it = 0;
        do {
            rho_old = rho;
            if (precond == 2) oracle_dic_precondition_f32(n, nf, l, u, upper, rD, ri, w);
            else if (precond == 1) for (int32_t i = 0; i < n; i++) w[i] = rD32[i] * ri[i];
            else for (int32_t i = 0; i < n; i++) w[i] = ri[i];
            rho = sum_prod_f32(n, w, ri);
            if (it == 0) {
                for (int32_t i = 0; i < n; i++) p[i] = w[i];
            } else {
                float beta = (float)(rho / rho_old);
                for (int32_t i = 0; i < n; i++) p[i] = fmaf(beta, p[i], w[i]);
            }
            oracle_amul_f32(n, nf, l, u, d32, u32, p, q);
            double sigma = sum_prod_f32(n, q, p);
            if (fabs(sigma) / infac < 1e-300) { singular = 1; break; }
            float alpha = (float)(rho / sigma);
            for (int32_t i = 0; i < n; i++) {
                di[i] = fmaf(alpha, p[i], di[i]);
                ri[i] = fmaf(-alpha, q[i], ri[i]);
            }
            ires = sum_mag_f32(n, ri) / infac;
            it++;
        } while (it < max_iter && !(ires < inner_rel_tol * ires0));
        total_it += it;
        for (int32_t i = 0; i < n; i++) x[i] = fma(s, (double)di[i], x[i]);
        outer++;
    }
done:
    perf[0] = res0;
    perf[1] = res;
    perf[2] = (double)total_it;
    perf[3] = (double)singular;
    perf[4] = (double)(res < tol);
    perf[5] = (double)outer;
    free(r); free(q64); free(rD); free(d32); free(u32); free(ri); free(di);
    free(w); free(p); free(q); free(rD32);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of x = A^-1 b for a loss L(x): with g = dL/dx, A lambda = g        */
/* (A symmetric, so A^T = A; same PCG);                                       */
/*   dL/db = lambda;  dL/dupper_f = -(lambda_l x_u + lambda_u x_l);           */
/*   dL/ddiag_i = -lambda_i x_i.                                              */
/* lambda is solved from 0 to tol with the given preconditioner.              */
/* ------------------------------------------------------------------------ */
int32_t oracle_adjoint(int32_t n, int32_t nf, const int32_t* l, const int32_t* u,
                       const double* diag, const double* upper, const double* x,
                       const double* g, int32_t precond, double tol, int32_t max_iter,
                       double* lambda, double* dupper, double* ddiag, double* perf)
{
    for (int32_t i = 0; i < n; i++) lambda[i] = 0.0;
    int32_t st = oracle_pcg(n, nf, l, u, diag, upper, g, lambda, precond, tol, 0.0, max_iter, 0, perf);
    if (st != 0) return st;
    for (int32_t f = 0; f < nf; f++)
        dupper[f] = -(lambda[l[f]] * x[u[f]] + lambda[u[f]] * x[l[f]]);
    for (int32_t i = 0; i < n; i++) ddiag[i] = -(lambda[i] * x[i]);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Mixed precision with reliable updates (residual replacement): the FP32    */
/* PCG (FP32 coefficients, Amul, DIC sweeps and vectors; reductions in       */
/* double; alpha, beta in double rounded to float) accumulates its           */
/* correction xs in FP32; whenever its recursively updated residual has      */
/* dropped below delta times the residual of the last update, or it claims    */
/* convergence, or max_iter is reached, the FP64 solution takes x += xs, the  */
/* true residual r = b - A64 x is recomputed in FP64 and replaces the FP32    */
/* residual, and the search direction p is kept (no Krylov restart).         */
/* The solve stops when that FP64 residual is converged (or max_iter).       */
/* perf: [0] initial res, [1] final res (FP64), [2] iterations,              */
/* [3] singular, [4] converged, [5] reliable updates                          */
/* ------------------------------------------------------------------------ */
int32_t oracle_mixed_reliable(int32_t n, int32_t nf, const int32_t* l, const int32_t* u,
                              const double* diag, const double* upper, const double* b, double* x,
                              int32_t precond, double tol, double rel_tol, double delta,
                              int32_t max_iter, double* perf)
{
    size_t b64 = sizeof(double) * (size_t)(n > 0 ? n : 1);
    size_t b32 = sizeof(float) * (size_t)(n > 0 ? n : 1);
    size_t bf32 = sizeof(float) * (size_t)(nf > 0 ? nf : 1);
    double* r64 = (double*)malloc(b64);
    double* q64 = (double*)malloc(b64);
    double* rD = (double*)malloc(b64);
    float* d32 = (float*)malloc(b32);
    float* u32 = (float*)malloc(bf32);
    float* r = (float*)malloc(b32);
    float* xs = (float*)malloc(b32);
    float* w = (float*)malloc(b32);
    float* p = (float*)malloc(b32);
    float* q = (float*)malloc(b32);
    float* rD32 = (float*)malloc(b32);
    int32_t status = 0, it = 0, updates = 0, singular = 0;
    double res0 = 0.0, res = 0.0;
    memset(perf, 0, 6 * sizeof(double));

    for (int32_t i = 0; i < n; i++) d32[i] = (float)diag[i];
    for (int32_t f = 0; f < nf; f++) u32[f] = (float)upper[f];
    if (precond == 2) {
        if (oracle_dic_factor(n, nf, l, u, diag, upper, rD) >= 0) { status = -2; goto done; }
    } else if (precond == 1) {
        oracle_diag_reciprocal(n, diag, rD);
    }
    for (int32_t i = 0; i < n; i++) rD32[i] = (float)rD[i];

    oracle_amul(n, nf, l, u, diag, upper, x, q64);
    for (int32_t i = 0; i < n; i++) r64[i] = b[i] - q64[i];
    double nfac = oracle_norm_factor(n, nf, l, u, diag, upper, x, b, q64);
    res0 = sum_mag(n, r64) / nfac;
    res = res0;
    if (converged(res0, res0, tol, rel_tol)) goto done;
    for (int32_t i = 0; i < n; i++) { r[i] = (float)r64[i]; xs[i] = 0.0f; }
    double rupd = res0, rho = 1.0, rho_old;
    for (;;) {
        rho_old = rho;
        if (precond == 2) oracle_dic_precondition_f32(n, nf, l, u, upper, rD, r, w);
        else if (precond == 1) for (int32_t i = 0; i < n; i++) w[i] = rD32[i] * r[i];
        else for (int32_t i = 0; i < n; i++) w[i] = r[i];
        rho = sum_prod_f32(n, w, r);
        if (it == 0) {
            for (int32_t i = 0; i < n; i++) p[i] = w[i];
        } else {
            float beta = (float)(rho / rho_old);
            for (int32_t i = 0; i < n; i++) p[i] = fmaf(beta, p[i], w[i]);
        }
        oracle_amul_f32(n, nf, l, u, d32, u32, p, q);
        double sigma = sum_prod_f32(n, q, p);
        if (fabs(sigma) / nfac < 1e-300) { singular = 1; break; }
        float alpha = (float)(rho / sigma);
        for (int32_t i = 0; i < n; i++) {
            xs[i] = fmaf(alpha, p[i], xs[i]);
            r[i] = fmaf(-alpha, q[i], r[i]);
        }
        it++;
        double ress = sum_mag_f32(n, r) / nfac;
        if (ress < delta * rupd || converged(ress, res0, tol, rel_tol) || it >= max_iter) {
            for (int32_t i = 0; i < n; i++) { x[i] += (double)xs[i]; xs[i] = 0.0f; }
            oracle_amul(n, nf, l, u, diag, upper, x, q64);
            for (int32_t i = 0; i < n; i++) r64[i] = b[i] - q64[i];
            res = sum_mag(n, r64) / nfac;
            updates++;
            if (converged(res, res0, tol, rel_tol) || it >= max_iter) break;
            for (int32_t i = 0; i < n; i++) r[i] = (float)r64[i];
            rupd = res;
        }
    }
    if (singular) {   /* fold the pending correction in */
        for (int32_t i = 0; i < n; i++) x[i] += (double)xs[i];
        oracle_amul(n, nf, l, u, diag, upper, x, q64);
        for (int32_t i = 0; i < n; i++) r64[i] = b[i] - q64[i];
        res = sum_mag(n, r64) / nfac;
    }
done:
    perf[0] = res0;
    perf[1] = res;
    perf[2] = (double)it;
    perf[3] = (double)singular;
    perf[4] = (double)converged(res, res0, tol, rel_tol);
    perf[5] = (double)updates;
    free(r64); free(q64); free(rD); free(d32); free(u32); free(r); free(xs);
    free(w); free(p); free(q); free(rD32);
    return status;
}

/* ======================================================================== */
/* Pressure-correction step around the solve (the paper's SIMPLE loop with  */
/* the schemes of its fvSchemes listing: gradSchemes Gauss linear,          */
/* interpolationSchemes linear, laplacianSchemes Gauss linear corrected,    */
/* snGradSchemes corrected; fvSolution: nNonOrthogonalCorrectors 0).  All   */
/* integrated over the cell (no division by volume except the gradient).    */
/* Boundary: Dirichlet faces carry p = 0, zero-gradient faces p_b = p_cell. */
/* ======================================================================== */

/* Linear interpolation weight of the owner (l) value at face f:             */
/*   w_f = |S.(C_u - C_f)| / (|S.(C_f - C_l)| + |S.(C_u - C_f)|),            */
/*   p_f = w_f p_l + (1 - w_f) p_u.                                          */
void oracle_fv_weights(int32_t nf, const int32_t* l, const int32_t* u, const double* sf, const double* cf,
                       const double* c, double* w)
{
    for (int32_t f = 0; f < nf; f++) {
        const double* s = sf + 3 * (int64_t)f;
        const double* x = cf + 3 * (int64_t)f;
        const double* cl = c + 3 * (int64_t)l[f];
        const double* cu = c + 3 * (int64_t)u[f];
        double own = fabs((s[0] * (x[0] - cl[0]) + s[1] * (x[1] - cl[1])) + s[2] * (x[2] - cl[2]));
        double nei = fabs((s[0] * (cu[0] - x[0]) + s[1] * (cu[1] - x[1])) + s[2] * (cu[2] - x[2]));
        w[f] = nei / (own + nei);
    }
}

/* Gauss linear gradient: grad_i = (1/V_i) sum over the faces of i of       */
/* S_f p_f (S outward: +S_f for the owner, -S_f for the neighbour), faces   */
/* in ascending order, then the boundary faces of i in ascending order.     */
void oracle_fv_grad(int32_t n, int32_t nf, const int32_t* l, const int32_t* u, const double* sf,
                    const double* w, const double* v, int32_t n_b, const int32_t* bcell, const double* bsf,
                    const int8_t* btype, const double* p, double* grad)
{
    for (int64_t k = 0; k < 3 * (int64_t)n; k++) grad[k] = 0.0;
    for (int32_t f = 0; f < nf; f++) {
        const double pf = w[f] * p[l[f]] + (1.0 - w[f]) * p[u[f]];
        for (int d = 0; d < 3; d++) {
            const double t = sf[3 * (int64_t)f + d] * pf;
            grad[3 * (int64_t)l[f] + d] += t;
            grad[3 * (int64_t)u[f] + d] -= t;
        }
    }
    for (int32_t b = 0; b < n_b; b++) {
        const int32_t i = bcell[b];
        const double pb = btype[b] == 1 ? 0.0 : p[i];
        for (int d = 0; d < 3; d++) grad[3 * (int64_t)i + d] += bsf[3 * (int64_t)b + d] * pb;
    }
    for (int32_t i = 0; i < n; i++)
        for (int d = 0; d < 3; d++) grad[3 * (int64_t)i + d] /= v[i];
}

/* Explicit non-orthogonal correction flux of the corrected laplacian and   */
/* the pressure right-hand side.  Per internal face:                        */
/*   |S| = sqrt((Sx Sx + Sy Sy) + Sz Sz), d = C_u - C_l, |d| likewise,        */
/*   n.d = ((Sx dx + Sy dy) + Sz dz)/|S|, delta = 1/max(n.d, 0.05 |d|),       */
/*   k = S/|S| - d delta  (the correction vector),                           */
/*   (grad p)_f = w grad_l + (1 - w) grad_u  (componentwise),                */
/*   corr_f = (gamma_f |S|) ((k_x g_x + k_y g_y) + k_z g_z).                  */
/* With A = -laplacian (implicit part) the pressure equation                 */
/*   laplacian(gamma, p) = div(phiHbyA) reads A p = b with                   */
/*   b_i = sum_f +-(corr_f - phi_f) (+ owner, - neighbour, faces ascending)  */
/*         - sum of phi_b over the boundary faces of i (ascending).          */
void oracle_pressure_rhs(int32_t n, int32_t nf, const int32_t* l, const int32_t* u, const double* sf,
                         const double* c, const double* w, const double* gamma, const double* grad,
                         const double* phi, int32_t n_b, const int32_t* bcell, const double* bphi,
                         double* corr, double* b)
{
    for (int32_t i = 0; i < n; i++) b[i] = 0.0;
    for (int32_t f = 0; f < nf; f++) {
        const double* s = sf + 3 * (int64_t)f;
        const double* cl = c + 3 * (int64_t)l[f];
        const double* cu = c + 3 * (int64_t)u[f];
        const double* gl = grad + 3 * (int64_t)l[f];
        const double* gu = grad + 3 * (int64_t)u[f];
        double dx = cu[0] - cl[0], dy = cu[1] - cl[1], dz = cu[2] - cl[2];
        double mags = sqrt((s[0] * s[0] + s[1] * s[1]) + s[2] * s[2]);
        double magd = sqrt((dx * dx + dy * dy) + dz * dz);
        double ndotd = ((s[0] * dx + s[1] * dy) + s[2] * dz) / mags;
        double delta = 1.0 / fmax(ndotd, 0.05 * magd);
        double kx = s[0] / mags - dx * delta, ky = s[1] / mags - dy * delta, kz = s[2] / mags - dz * delta;
        double wf = w[f], wu = 1.0 - w[f];
        double gx = wf * gl[0] + wu * gu[0], gy = wf * gl[1] + wu * gu[1], gz = wf * gl[2] + wu * gu[2];
        corr[f] = (gamma[f] * mags) * ((kx * gx + ky * gy) + kz * gz);
        const double t = corr[f] - phi[f];
        b[l[f]] += t;
        b[u[f]] -= t;
    }
    for (int32_t k = 0; k < n_b; k++) b[bcell[k]] -= bphi[k];
}

/* Flux after the solve: phi_f = phiHbyA_f - (a_f (p_u - p_l) + corr_f),     */
/* a_f = -upper_f; boundary: Dirichlet phi_b = phiHbyA_b + a_b p_cell with   */
/* a_b the boundary coefficient of the assembly, zero-gradient phiHbyA_b.   */
void oracle_pressure_flux(int32_t nf, const int32_t* l, const int32_t* u, const double* upper,
                          const double* corr, const double* p, const double* phi, int32_t n_b,
                          const int32_t* bcell, const double* bsf, const double* bcf, const double* bgamma,
                          const int8_t* btype, const double* c, const double* bphi, double* phi_out,
                          double* bphi_out)
{
    for (int32_t f = 0; f < nf; f++) phi_out[f] = phi[f] - ((-upper[f]) * (p[u[f]] - p[l[f]]) + corr[f]);
    for (int32_t b = 0; b < n_b; b++) {
        if (btype[b] != 1) {
            bphi_out[b] = bphi[b];
            continue;
        }
        const int32_t i = bcell[b];
        const double ab = face_coeff(bsf + 3 * (int64_t)b, c + 3 * (int64_t)i, bcf + 3 * (int64_t)b, bgamma[b]);
        bphi_out[b] = bphi[b] + ab * p[i];
    }
}

/* Integrated divergence: div_i = sum_f +-phi_f (+ owner, - neighbour, faces */
/* ascending) + the boundary fluxes of i (ascending).                        */
void oracle_fv_div(int32_t n, int32_t nf, const int32_t* l, const int32_t* u, const double* phi, int32_t n_b,
                   const int32_t* bcell, const double* bphi, double* div)
{
    for (int32_t i = 0; i < n; i++) div[i] = 0.0;
    for (int32_t f = 0; f < nf; f++) {
        div[l[f]] += phi[f];
        div[u[f]] -= phi[f];
    }
    for (int32_t b = 0; b < n_b; b++) div[bcell[b]] += bphi[b];
}

/* ======================================================================== */
/* Asymmetric LDU matrices and PBiCG with DILU (the paper's momentum / k /  */
/* omega solver: "PBiCG, preconditioner aDILU" in its fvSolution listing;  */
/* "SpMVM (Amul + Tmul)" and "aDILUPreconditioner" in its profiling table,  */
/* Sec. 4.2).  lduMatrix with lower != upper: A_{u(f),l(f)} = lower_f,      */
/* A_{l(f),u(f)} = upper_f.                                                 */
/* ======================================================================== */

/* Amul:  y_i = d_i x_i; faces ascending: y_u += lower_f x_l; y_l += upper_f x_u */
/* Tmul (A^T x): the same with lower and upper exchanged.  Each += is one FMA.  */
void oracle_amul_asym(int32_t n, int32_t nf, const int32_t* l, const int32_t* u, const double* diag,
                      const double* lower, const double* upper, const double* x, double* y)
{
    for (int32_t i = 0; i < n; i++) y[i] = diag[i] * x[i];
    for (int32_t f = 0; f < nf; f++) {
        y[u[f]] = fma(lower[f], x[l[f]], y[u[f]]);
        y[l[f]] = fma(upper[f], x[u[f]], y[l[f]]);
    }
}

/* DILU factor: pivots p_i = d_i; faces ascending: p_u -= (upper_f lower_f) / p_l;
 * rD_i = 1/p_i.  It makes diag((D + L) D^-1 (D + U)) = diag(A) with D = diag(p).
 * Returns -1, or the first cell whose pivot is zero or not finite.            */
int32_t oracle_dilu_factor(int32_t n, int32_t nf, const int32_t* l, const int32_t* u, const double* diag,
                           const double* lower, const double* upper, double* rD)
{
    for (int32_t i = 0; i < n; i++) rD[i] = diag[i];
    for (int32_t f = 0; f < nf; f++) rD[u[f]] -= (upper[f] * lower[f]) / rD[l[f]];
    int32_t bad = -1;
    for (int32_t i = 0; i < n; i++) {
        if (!(rD[i] != 0.0 && isfinite(rD[i])) && bad < 0) bad = i;
        rD[i] = 1.0 / rD[i];
    }
    return bad;
}

/* DILU apply, w = M^-1 r with M = (D + L) D^-1 (D + U):
 *   w_i = rD_i r_i; forward f ascending: w_u -= (rD_u lower_f) w_l;
 *   backward f descending: w_l -= (rD_l upper_f) w_u.
 * transpose (w = M^-T r): lower and upper exchanged.  Each -= one FMA of the
 * rounded product.                                                          */
void oracle_dilu_precondition(int32_t n, int32_t nf, const int32_t* l, const int32_t* u, const double* lower,
                              const double* upper, const double* rD, const double* r, double* w)
{
    for (int32_t i = 0; i < n; i++) w[i] = rD[i] * r[i];
    for (int32_t f = 0; f < nf; f++) {
        double c = rD[u[f]] * lower[f];
        w[u[f]] = fma(-c, w[l[f]], w[u[f]]);
    }
    for (int32_t f = nf - 1; f >= 0; f--) {
        double c = rD[l[f]] * upper[f];
        w[l[f]] = fma(-c, w[u[f]], w[l[f]]);
    }
}

/* OpenFOAM PBiCG (bi-conjugate gradients on A x = b and A^T x~ = b, with
 * the same normalised L1 residual as PCG; normFactor from the row sums of A):
 *   rA = b - A x, rT = b - A^T x; res0 = sum|rA|/normFactor; then
 *   do { wArA_old = wArA; wA = M^-1 rA; wT = M^-T rT; wArA = sum wA rT;
 *        first: pA = wA, pT = wT; else beta = wArA/wArA_old,
 *        pA = wA + beta pA, pT = wT + beta pT;
 *        wA = A pA; wT = A^T pT; wApT = sum wA pT;
 *        singular if |wApT|/normFactor < 1e-300;
 *        alpha = wArA/wApT; x += alpha pA; rA -= alpha wA; rT -= alpha wT;
 *        res = sum|rA|/normFactor }
 *   while the PCG loop condition holds.
 * precond: 0 none, 1 diagonal, 3 DILU.  perf as oracle_pcg.                  */
int32_t oracle_pbicg(int32_t n, int32_t nf, const int32_t* l, const int32_t* u, const double* diag,
                     const double* lower, const double* upper, const double* b, double* x, int32_t precond,
                     double tol, double rel_tol, int32_t max_iter, int32_t min_iter, double* perf)
{
    size_t bytes = sizeof(double) * (size_t)(n > 0 ? n : 1);
    double *rA = malloc(bytes), *rT = malloc(bytes), *wA = malloc(bytes), *wT = malloc(bytes);
    double *pA = malloc(bytes), *pT = malloc(bytes), *rD = malloc(bytes), *s = malloc(bytes);
    int32_t status = 0;
    memset(perf, 0, 5 * sizeof(double));
    oracle_amul_asym(n, nf, l, u, diag, lower, upper, x, wA);
    oracle_amul_asym(n, nf, l, u, diag, upper, lower, x, wT);
    for (int32_t i = 0; i < n; i++) {
        rA[i] = b[i] - wA[i];
        rT[i] = b[i] - wT[i];
    }
    /* normFactor: s = row sums of A, xbar = mean(x) */
    for (int32_t i = 0; i < n; i++) s[i] = diag[i];
    for (int32_t f = 0; f < nf; f++) {
        s[u[f]] += lower[f];
        s[l[f]] += upper[f];
    }
    double xbar = 0.0;
    for (int32_t i = 0; i < n; i++) xbar += x[i];
    xbar = n > 0 ? xbar / (double)n : 0.0;
    double nfac = 0.0;
    for (int32_t i = 0; i < n; i++) {
        double t = s[i] * xbar;
        nfac += fabs(wA[i] - t) + fabs(b[i] - t);
    }
    nfac += 1e-20;
    double res0 = sum_mag(n, rA) / nfac, res = res0;
    int32_t it = 0, singular = 0;
    if (precond == 3) {
        if (oracle_dilu_factor(n, nf, l, u, diag, lower, upper, rD) >= 0) { status = -2; goto done; }
    } else if (precond == 1) {
        oracle_diag_reciprocal(n, diag, rD);
    }
    if (min_iter > 0 || !converged(res0, res0, tol, rel_tol)) {
        double wArA = 1.0, wArA_old;
        do {
            wArA_old = wArA;
            if (precond == 3) {
                oracle_dilu_precondition(n, nf, l, u, lower, upper, rD, rA, wA);
                oracle_dilu_precondition(n, nf, l, u, upper, lower, rD, rT, wT);
            } else if (precond == 1) {
                for (int32_t i = 0; i < n; i++) { wA[i] = rD[i] * rA[i]; wT[i] = rD[i] * rT[i]; }
            } else {
                for (int32_t i = 0; i < n; i++) { wA[i] = rA[i]; wT[i] = rT[i]; }
            }
            wArA = sum_prod(n, wA, rT);
            if (it == 0) {
                for (int32_t i = 0; i < n; i++) { pA[i] = wA[i]; pT[i] = wT[i]; }
            } else {
                double beta = wArA / wArA_old;
                for (int32_t i = 0; i < n; i++) {
                    pA[i] = fma(beta, pA[i], wA[i]);
                    pT[i] = fma(beta, pT[i], wT[i]);
                }
            }
            oracle_amul_asym(n, nf, l, u, diag, lower, upper, pA, wA);
            oracle_amul_asym(n, nf, l, u, diag, upper, lower, pT, wT);
            double wApT = sum_prod(n, wA, pT);
            if (fabs(wApT) / nfac < 1e-300) { singular = 1; break; }
            double alpha = wArA / wApT;
            for (int32_t i = 0; i < n; i++) {
                x[i] = fma(alpha, pA[i], x[i]);
                rA[i] = fma(-alpha, wA[i], rA[i]);
                rT[i] = fma(-alpha, wT[i], rT[i]);
            }
            res = sum_mag(n, rA) / nfac;
        } while ((++it < max_iter && !converged(res, res0, tol, rel_tol)) || it < min_iter);
    }
done:
    perf[0] = res0;
    perf[1] = res;
    perf[2] = (double)it;
    perf[3] = (double)singular;
    perf[4] = (double)converged(res, res0, tol, rel_tol);
    free(rA); free(rT); free(wA); free(wT); free(pA); free(pT); free(rD); free(s);
    return status;
}

/* One damped-Jacobi (Richardson) sweep of the GAMG smoother:               */
/*   q = A e (oracle_amul), then e_i = fma(wrd_i, r_i - q_i, e_i), wrd_i =   */
/*   omega rD_i.  q is scratch.                                              */
void oracle_jacobi_sweep(int32_t n, int32_t nf, const int32_t* l, const int32_t* u, const double* diag,
                         const double* upper, const double* wrd, const double* r, double* e, double* q)
{
    oracle_amul(n, nf, l, u, diag, upper, e, q);
    for (int32_t i = 0; i < n; i++) e[i] = fma(wrd[i], r[i] - q[i], e[i]);
}

/* One two-stage Gauss-Seidel sweep of the GAMG smoother (the paper's second
 * parallel smoother, Sec. 4.3, after Berger-Vergiat et al.): the Gauss-Seidel
 * step e += (D + L)^-1 (r - A e) with the lower-triangular solve replaced by
 * one Jacobi step and one Jacobi-Richardson sweep:
 *   q = r - A e (oracle_amul, then one subtraction per row);
 *   y_i = rD_i q_i  (rD = 1/d);
 *   s_u = q_u - sum_{f: u(f) = u} upper_f y_{l(f)}, f ascending, one FMA per term;
 *   e_i = e_i + rD_i s_i.
 * (D + L)^-1 ~ D^-1 - D^-1 L D^-1; L is A's strictly lower part (row u(f),
 * column l(f), coefficient upper_f).  q and y are scratch.                 */
void oracle_gs2_sweep(int32_t n, int32_t nf, const int32_t* l, const int32_t* u, const double* diag,
                      const double* upper, const double* rD, const double* r, double* e, double* q, double* y)
{
    oracle_amul(n, nf, l, u, diag, upper, e, q);
    for (int32_t i = 0; i < n; i++) q[i] = r[i] - q[i];
    for (int32_t i = 0; i < n; i++) y[i] = rD[i] * q[i];
    for (int32_t f = 0; f < nf; f++) q[u[f]] = fma(-upper[f], y[l[f]], q[u[f]]);
    for (int32_t i = 0; i < n; i++) e[i] = e[i] + rD[i] * q[i];
}

/* sum_i a_i b_i in ascending order (GAMG correction scaling). */
double oracle_dot(int32_t n, const double* a, const double* b) { return sum_prod(n, a, b); }
