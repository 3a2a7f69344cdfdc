// solve.cu -- the persistent PCG solver (FP64 and mixed FP32/FP64 iterative
// refinement), the level-scheduled DIC factor and sweeps, the prepared-matrix
// Amul, and their host entry points.
//
// One cooperative launch per solve.  Rows live in the handle's level order:
// level L (rows whose longest chain of lower neighbours has length L) is the
// contiguous range lvl[L]..lvl[L+1], and every row keeps its neighbour-side
// ("lower") and owner-side ("upper") entries in ascending face order, so each
// row sum is taken in exactly the order of the sequential face loop.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <map>

#include "solve.cuh"

namespace spuma {

enum Slot { SL_A = 0, SL_B = 1, SL_C = 2, SL_D = 3 };

__device__ __forceinline__ bool converged(double res, double res0, double tol, double rel_tol)
{
    return res < tol || (rel_tol > 0.0 && res < rel_tol * res0);
}

template <class T>
__device__ __forceinline__ Mat<T> mat_of(const SolveArgs& a);
template <>
__device__ __forceinline__ Mat<double> mat_of<double>(const SolveArgs& a)
{
    return Mat<double>{a.Lptr, a.Lcol, a.La64, a.Lc64, a.Uptr, a.Ucol, a.Ua64, a.Uc64, a.d64, a.rD64};
}
template <>
__device__ __forceinline__ Mat<float> mat_of<float>(const SolveArgs& a)
{
    return Mat<float>{a.Lptr, a.Lcol, a.La32, a.Lc32, a.Uptr, a.Ucol, a.Ua32, a.Uc32, a.d32, a.rD32};
}

// y_p = d_p x_p + lower entries (ascending face) + upper entries (ascending face)
template <class T>
__device__ __forceinline__ T amul_row(const Mat<T>& A, const T* __restrict__ x, int p)
{
    T y = mul_rn(A.d[p], x[p]);
    const int l0 = A.Lptr[p], l1 = A.Lptr[p + 1];
    for (int e = l0; e < l1; e++) y = fmadd(A.La[e], x[A.Lcol[e]], y);
    const int u0 = A.Uptr[p], u1 = A.Uptr[p + 1];
    for (int e = u0; e < u1; e++) y = fmadd(A.Ua[e], x[A.Ucol[e]], y);
    return y;
}

template <class T>
struct Vecs {
    T *x, *r, *w, *p, *q;
};

struct RowIter {
    int first, stride;
};

__device__ __forceinline__ RowIter rows_of(const Group& g)
{
    return RowIter{g.bid * (int)blockDim.x + (int)threadIdx.x, g.nblocks * (int)blockDim.x};
}

// ------------------------------------------------------------ phases --------
// Gather the LDU coefficients into the internal layout (+ FP32 copies).
__device__ bool phase_gather(const SolveArgs& a, const Group& g)
{
    RowIter it = rows_of(g);
    bool bad = false;
    for (int e = it.first; e < a.nf; e += it.stride) {
        double lv = a.upper_orig[a.Lface[e]];
        double uv = a.upper_orig[a.Uface[e]];
        a.La64[e] = lv;
        a.Ua64[e] = uv;
        a.La32[e] = (float)lv;
        a.Ua32[e] = (float)uv;
        bad |= !isfinite(lv);
    }
    for (int p = it.first; p < a.n; p += it.stride) {
        double dv = a.diag_orig[a.perm[p]];
        a.d64[p] = dv;
        a.d32[p] = (float)dv;
        bad |= !isfinite(dv);
    }
    if (bad) flag_error(a.status, SPUMA_ERR_NONFINITE, -1);
    return group_sync(g);
}

// DIC pivots level by level: p_i = d_i - sum_{lower entries} (a a)/p_col,
// then rD = 1/p and the sweep coefficients rD_row * a (+ FP32 copies).
// Diagonal: rD = 1/d.
__device__ bool phase_factor(const SolveArgs& a, const Group& g)
{
    RowIter it = rows_of(g);
    if (a.precond == SPUMA_PRECOND_DIC) {
        for (int L = 0; L < a.nlev; L++) {
            const int r0 = a.lvl[L], r1 = a.lvl[L + 1];
            for (int p = r0 + it.first; p < r1; p += it.stride) {
                double piv = a.d64[p];
                for (int e = a.Lptr[p]; e < a.Lptr[p + 1]; e++) {
                    double av = a.La64[e];
                    piv = __dsub_rn(piv, __ddiv_rn(__dmul_rn(av, av), a.rD64[a.Lcol[e]]));
                }
                a.rD64[p] = piv;
                if (!(piv > 0.0)) flag_error(a.status, SPUMA_ERR_NOT_SPD, a.perm[p]);
            }
            if (!group_sync(g)) return false;
        }
    }
    for (int p = it.first; p < a.n; p += it.stride) {
        double rd;
        if (a.precond == SPUMA_PRECOND_DIC)
            rd = __ddiv_rn(1.0, a.rD64[p]);
        else if (a.precond == SPUMA_PRECOND_DIAGONAL)
            rd = __ddiv_rn(1.0, a.d64[p]);
        else
            rd = 1.0;
        a.rD64[p] = rd;
        a.rD32[p] = (float)rd;
        if (a.precond == SPUMA_PRECOND_DIC) {
            for (int e = a.Lptr[p]; e < a.Lptr[p + 1]; e++) {
                double c = __dmul_rn(rd, a.La64[e]);
                a.Lc64[e] = c;
                a.Lc32[e] = (float)c;
            }
            for (int e = a.Uptr[p]; e < a.Uptr[p + 1]; e++) {
                double c = __dmul_rn(rd, a.Ua64[e]);
                a.Uc64[e] = c;
                a.Uc32[e] = (float)c;
            }
        }
    }
    return group_sync(g);
}

// DIC forward sweep over all levels, optionally fused with the pending
// x/r update of the previous PCG iteration (x += alpha p, r -= alpha q) and
// the sum|r| of the updated residual (slot A).
template <class T>
__device__ bool dic_forward(const SolveArgs& a, const Mat<T>& A, Vecs<T> v, bool pending, T alpha, const Group& g)
{
    RowIter it = rows_of(g);
    double acc = 0.0;
    for (int L = 0; L < a.nlev; L++) {
        const int r0 = a.lvl[L], r1 = a.lvl[L + 1];
        for (int p = r0 + it.first; p < r1; p += it.stride) {
            T rr = v.r[p];
            if (pending) {
                v.x[p] = fmadd(alpha, v.p[p], v.x[p]);
                rr = fmadd(-alpha, v.q[p], rr);
                v.r[p] = rr;
                acc += fabs((double)rr);
            }
            T ww = mul_rn(A.rD[p], rr);
            for (int e = A.Lptr[p]; e < A.Lptr[p + 1]; e++) ww = fmadd(-A.Lc[e], v.w[A.Lcol[e]], ww);
            v.w[p] = ww;
        }
        if (L == a.nlev - 1 && pending) {
            double t[1] = {acc};
            block_reduce_store<1>(t, a.partials, SL_A, g.bid);
        }
        if (!group_sync(g)) return false;
    }
    return true;
}

// DIC backward sweep (levels descending, upper entries descending face order),
// with rho = sum w r into slot B.
template <class T>
__device__ bool dic_backward(const SolveArgs& a, const Mat<T>& A, Vecs<T> v, bool want_rho, const Group& g)
{
    RowIter it = rows_of(g);
    double acc = 0.0;
    for (int L = a.nlev - 1; L >= 0; L--) {
        const int r0 = a.lvl[L], r1 = a.lvl[L + 1];
        for (int p = r0 + it.first; p < r1; p += it.stride) {
            T ww = v.w[p];
            for (int e = A.Uptr[p + 1] - 1; e >= A.Uptr[p]; e--) ww = fmadd(-A.Uc[e], v.w[A.Ucol[e]], ww);
            v.w[p] = ww;
            acc = fma((double)ww, (double)v.r[p], acc);
        }
        if (L == 0 && want_rho) {
            double t[1] = {acc};
            block_reduce_store<1>(t, a.partials, SL_B, g.bid);
        }
        if (!group_sync(g)) return false;
    }
    return true;
}

// PCG iterations on (A, v.r) from the current v.x (OpenFOAM recurrences).
// Returns the iteration count, or -1 when a device error stopped the group.
template <class T>
__device__ int pcg_loop(const SolveArgs& a, const Mat<T>& A, Vecs<T> v, double nfac, double res0, double tol,
                        double rel_tol, int max_iter, int min_iter, double* res_out, int* singular,
                        const Group& g)
{
    RowIter it = rows_of(g);
    double res = res0;
    *res_out = res;
    if (!(min_iter > 0 || !converged(res0, res0, tol, rel_tol))) return 0;
    int n_it = 0;
    double rho = 1.0, rho_old;
    T alpha = (T)0;
    bool pending = false;
    for (;;) {
        rho_old = rho;
        if (a.precond == SPUMA_PRECOND_DIC) {
            if (!dic_forward<T>(a, A, v, pending, alpha, g)) return -1;
            if (pending) {
                double t[1];
                grid_reduce_read<1>(t, a.partials, SL_A, g.nblocks);
                res = t[0] / nfac;
                n_it++;
                if (!((n_it < max_iter && !converged(res, res0, tol, rel_tol)) || n_it < min_iter)) break;
            }
            if (!dic_backward<T>(a, A, v, true, g)) return -1;
            double t[1];
            grid_reduce_read<1>(t, a.partials, SL_B, g.nblocks);
            rho = t[0];
        } else {
            double acc[2] = {0.0, 0.0};
            for (int p = it.first; p < a.n; p += it.stride) {
                T rr = v.r[p];
                if (pending) {
                    v.x[p] = fmadd(alpha, v.p[p], v.x[p]);
                    rr = fmadd(-alpha, v.q[p], rr);
                    v.r[p] = rr;
                    acc[0] += fabs((double)rr);
                }
                T ww = a.precond == SPUMA_PRECOND_DIAGONAL ? mul_rn(A.rD[p], rr) : rr;
                v.w[p] = ww;
                acc[1] = fma((double)ww, (double)rr, acc[1]);
            }
            block_reduce_store<2>(acc, a.partials, SL_A, g.bid);
            if (!group_sync(g)) return -1;
            double t[2];
            grid_reduce_read<2>(t, a.partials, SL_A, g.nblocks);
            if (pending) {
                res = t[0] / nfac;
                n_it++;
                if (!((n_it < max_iter && !converged(res, res0, tol, rel_tol)) || n_it < min_iter)) break;
            }
            rho = t[1];
        }
        // search direction
        const bool first = n_it == 0;
        const T beta = first ? (T)0 : (T)(rho / rho_old);
        for (int p = it.first; p < a.n; p += it.stride) v.p[p] = first ? v.w[p] : fmadd(beta, v.p[p], v.w[p]);
        if (!group_sync(g)) return -1;
        // q = A p, sigma = q.p
        double sacc[1] = {0.0};
        for (int p = it.first; p < a.n; p += it.stride) {
            T qq = amul_row<T>(A, v.p, p);
            v.q[p] = qq;
            sacc[0] = fma((double)qq, (double)v.p[p], sacc[0]);
        }
        block_reduce_store<1>(sacc, a.partials, SL_C, g.bid);
        if (!group_sync(g)) return -1;
        double sg[1];
        grid_reduce_read<1>(sg, a.partials, SL_C, g.nblocks);
        if (fabs(sg[0]) / nfac < 1e-300) {
            *singular = 1;
            break;
        }
        alpha = (T)(rho / sg[0]);
        pending = true;
    }
    *res_out = res;
    return n_it;
}

// x = x_orig (or 0), b = b_orig in internal order; q = A x; r = b - q;
// normFactor = sum(|q - s xbar| + |b - s xbar|) + 1e-20; returns res0 and nfac.
__device__ bool phase_init(const SolveArgs& a, const Group& g, double* nfac, double* res0)
{
    RowIter it = rows_of(g);
    const Mat<double> A = mat_of<double>(a);
    for (int p = it.first; p < a.n; p += it.stride) {
        const int i = a.perm[p];
        a.x[p] = a.zero_x0 ? 0.0 : a.x_orig[i];
        double bv = a.b_orig[i];
        a.b[p] = bv;
        if (!isfinite(bv)) flag_error(a.status, SPUMA_ERR_NONFINITE, i);
    }
    if (!group_sync(g)) return false;
    double acc[2] = {0.0, 0.0};
    for (int p = it.first; p < a.n; p += it.stride) {
        double qq = amul_row<double>(A, a.x, p);
        a.q[p] = qq;
        double rr = a.b[p] - qq;
        a.r[p] = rr;
        acc[0] += a.x[p];
        acc[1] += fabs(rr);
    }
    block_reduce_store<2>(acc, a.partials, SL_A, g.bid);
    if (!group_sync(g)) return false;
    double t[2];
    grid_reduce_read<2>(t, a.partials, SL_A, g.nblocks);
    const double xbar = a.n > 0 ? t[0] / (double)a.n : 0.0;
    const double sum_r = t[1];
    double acc2[1] = {0.0};
    for (int p = it.first; p < a.n; p += it.stride) {
        double s = a.d64[p];
        for (int e = a.Lptr[p]; e < a.Lptr[p + 1]; e++) s += a.La64[e];
        for (int e = a.Uptr[p]; e < a.Uptr[p + 1]; e++) s += a.Ua64[e];
        const double tt = s * xbar;
        acc2[0] += fabs(a.q[p] - tt) + fabs(a.b[p] - tt);
    }
    block_reduce_store<1>(acc2, a.partials, SL_B, g.bid);
    if (!group_sync(g)) return false;
    double t2[1];
    grid_reduce_read<1>(t2, a.partials, SL_B, g.nblocks);
    *nfac = t2[0] + 1e-20;
    *res0 = sum_r / *nfac;
    return true;
}

__device__ void phase_store_x(const SolveArgs& a, const Group& g)
{
    RowIter it = rows_of(g);
    for (int p = it.first; p < a.n; p += it.stride) a.x_orig[a.perm[p]] = a.x[p];
}

// Mixed precision: FP64 refinement around FP32 inner PCG.
__device__ bool solve_mixed(const SolveArgs& a, const Group& g, double nfac, spuma_solver_perf& pf)
{
    RowIter it = rows_of(g);
    const Mat<double> A64 = mat_of<double>(a);
    const Mat<float> A32 = mat_of<float>(a);
    Vecs<float> vi{a.xi, a.ri, a.wi, a.pi, a.qi};
    int outer = 0, total = 0, singular = 0;
    double res = 0.0, res0 = 0.0;
    for (;;) {
        double acc[1] = {0.0}, mx[1] = {0.0};
        for (int p = it.first; p < a.n; p += it.stride) {
            double rr = a.b[p] - amul_row<double>(A64, a.x, p);
            a.r[p] = rr;
            acc[0] += fabs(rr);
            mx[0] = fmax(mx[0], fabs(rr));
        }
        block_reduce_store<1>(acc, a.partials, SL_A, g.bid);
        block_max_store<1>(mx, a.partials, SL_B, g.bid);
        if (!group_sync(g)) return false;
        double t[1], m[1];
        grid_reduce_read<1>(t, a.partials, SL_A, g.nblocks);
        grid_reduce_read<1, true>(m, a.partials, SL_B, g.nblocks);
        res = t[0] / nfac;
        if (outer == 0) res0 = res;
        if (res < a.tol || outer >= a.max_outer || singular) break;
        const double s = m[0];
        if (s == 0.0) break;
        double iacc[1] = {0.0};
        for (int p = it.first; p < a.n; p += it.stride) {
            float rv = (float)(a.r[p] / s);
            vi.r[p] = rv;
            vi.x[p] = 0.0f;
            iacc[0] += fabs((double)rv);
        }
        block_reduce_store<1>(iacc, a.partials, SL_C, g.bid);
        if (!group_sync(g)) return false;
        double ti[1];
        grid_reduce_read<1>(ti, a.partials, SL_C, g.nblocks);
        const double infac = ti[0] + 1e-20;
        const double ires0 = ti[0] / infac;
        double ires;
        int n_in = pcg_loop<float>(a, A32, vi, infac, ires0, 0.0, a.inner_rel_tol, a.max_iter, 1, &ires, &singular, g);
        if (n_in < 0) return false;
        total += n_in;
        for (int p = it.first; p < a.n; p += it.stride) a.x[p] = fma(s, (double)vi.x[p], a.x[p]);
        if (!group_sync(g)) return false;
        outer++;
    }
    pf.initial_residual = res0;
    pf.final_residual = res;
    pf.n_iter = total;
    pf.n_outer = outer;
    pf.converged = res < a.tol;
    pf.singular = singular;
    return true;
}

__device__ void run_system(const SolveArgs& a, const Group& g)
{
    spuma_solver_perf pf;
    pf.initial_residual = 0.0;
    pf.final_residual = 0.0;
    pf.n_iter = 0;
    pf.n_outer = 0;
    pf.converged = 0;
    pf.singular = 0;
    pf.status = 0;
    pf.n_levels = a.nlev;
    bool ok = true;
    if (a.mode == MODE_PREPARE || a.mode == MODE_SOLVE) {
        ok = phase_gather(a, g);
        if (ok) ok = phase_factor(a, g);
    }
    if (ok && a.mode == MODE_PRECONDITION) {
        // w = M^-1 r for r = b_orig, written to x_orig (FP64)
        RowIter it = rows_of(g);
        for (int p = it.first; p < a.n; p += it.stride) a.r[p] = a.b_orig[a.perm[p]];
        ok = group_sync(g);
        Vecs<double> v{a.x, a.r, a.w, a.p, a.q};
        const Mat<double> A = mat_of<double>(a);
        if (ok) {
            if (a.precond == SPUMA_PRECOND_DIC) {
                ok = dic_forward<double>(a, A, v, false, 0.0, g);
                if (ok) ok = dic_backward<double>(a, A, v, false, g);
            } else {
                for (int p = it.first; p < a.n; p += it.stride)
                    a.w[p] = a.precond == SPUMA_PRECOND_DIAGONAL ? __dmul_rn(a.rD64[p], a.r[p]) : a.r[p];
                ok = group_sync(g);
            }
        }
        if (ok)
            for (int p = it.first; p < a.n; p += it.stride) a.x_orig[a.perm[p]] = a.w[p];
    }
    if (ok && a.mode == MODE_SOLVE) {
        double nfac = 1.0, res0 = 0.0;
        ok = phase_init(a, g, &nfac, &res0);
        if (ok) {
            if (a.precision == SPUMA_MIXED) {
                ok = solve_mixed(a, g, nfac, pf);
            } else {
                Vecs<double> v{a.x, a.r, a.w, a.p, a.q};
                double res;
                int sing = 0;
                int n_it = pcg_loop<double>(a, mat_of<double>(a), v, nfac, res0, a.tol, a.rel_tol, a.max_iter,
                                            a.min_iter, &res, &sing, g);
                ok = n_it >= 0;
                pf.initial_residual = res0;
                pf.final_residual = res;
                pf.n_iter = n_it < 0 ? 0 : n_it;
                pf.converged = converged(res, res0, a.tol, a.rel_tol);
                pf.singular = sing;
            }
        }
        if (ok) phase_store_x(a, g);
    }
    if (g.bid == 0 && threadIdx.x == 0 && a.perf) {
        __threadfence();
        pf.status = ld_volatile_int(a.status);
        if (pf.status != 0) pf.converged = 0;
        *a.perf = pf;
    }
}

__global__ void __launch_bounds__(512) k_solve(SolveArgs a, unsigned long long timeout_ns)
{
    Group g{a.bar, a.bar + 32, a.status, (int)gridDim.x, (int)blockIdx.x, timeout_ns};
    run_system(a, g);
}

__global__ void __launch_bounds__(512) k_solve_batch(BatchTable t, unsigned long long timeout_ns)
{
    __shared__ SolveArgs sa;
    int s = 0;
    while (s + 1 < t.n_sys && (int)blockIdx.x >= t.split[s + 1]) s++;
    if (threadIdx.x == 0) sa = *t.args[s];
    __syncthreads();
    Group g{sa.bar, sa.bar + 32, sa.status, t.split[s + 1] - t.split[s], (int)blockIdx.x - t.split[s], timeout_ns};
    run_system(sa, g);
}

// Stand-alone Amul on the prepared matrix (internal order).
template <class T>
__global__ void k_amul_prepared(int n, Mat<T> A, const T* __restrict__ x, T* __restrict__ y)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) y[p] = amul_row<T>(A, x, p);
}

__global__ void k_permute(int n, int dir, const int* __restrict__ perm, const double* __restrict__ src, double* dst)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        if (dir == 0)
            dst[p] = src[perm[p]];
        else
            dst[perm[p]] = src[p];
    }
}

__global__ void k_read_rD(int n, const int* __restrict__ perm, const double* __restrict__ rD, double* out)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) out[perm[p]] = rD[p];
}

// ------------------------------------------------------------ host side -----
SolveArgs make_args(spuma_ldu_t h)
{
    SolveArgs a{};
    const Layout& L = h->L;
    a.n = h->n;
    a.nf = h->nf;
    a.nlev = h->nlev;
    a.lvl = h->at<int>(L.lvl);
    a.perm = h->at<int>(L.perm);
    a.Lptr = h->at<int>(L.Lptr);
    a.Lcol = h->at<int>(L.Lcol);
    a.Lface = h->at<int>(L.Lface);
    a.Uptr = h->at<int>(L.Uptr);
    a.Ucol = h->at<int>(L.Ucol);
    a.Uface = h->at<int>(L.Uface);
    a.La64 = h->at<double>(L.La64);
    a.Ua64 = h->at<double>(L.Ua64);
    a.Lc64 = h->at<double>(L.Lc64);
    a.Uc64 = h->at<double>(L.Uc64);
    a.d64 = h->at<double>(L.d64);
    a.rD64 = h->at<double>(L.rD64);
    a.La32 = h->at<float>(L.La32);
    a.Ua32 = h->at<float>(L.Ua32);
    a.Lc32 = h->at<float>(L.Lc32);
    a.Uc32 = h->at<float>(L.Uc32);
    a.d32 = h->at<float>(L.d32);
    a.rD32 = h->at<float>(L.rD32);
    a.x = h->at<double>(L.x64);
    a.r = h->at<double>(L.r64);
    a.w = h->at<double>(L.w64);
    a.p = h->at<double>(L.p64);
    a.q = h->at<double>(L.q64);
    a.b = h->at<double>(L.b64);
    a.xi = h->at<float>(L.x32);
    a.ri = h->at<float>(L.r32);
    a.wi = h->at<float>(L.w32);
    a.pi = h->at<float>(L.p32);
    a.qi = h->at<float>(L.q32);
    a.partials = h->at<double>(L.partials);
    a.bar = h->at<unsigned>(L.bar);
    a.status = h->at<int>(L.status);
    return a;
}

static std::mutex g_occ_mu;
static std::map<int, int> g_occ;   // (kernel, block threads) -> co-resident blocks per SM

int solve_blocks_per_sm(int threads, bool batch)
{
    std::lock_guard<std::mutex> lk(g_occ_mu);
    const int key = threads * 2 + (batch ? 1 : 0);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) return it->second;
    int nb = 0;
    cudaError_t e = batch ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_solve_batch, threads, 0)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_solve, threads, 0);
    if (e != cudaSuccess) nb = 0;
    g_occ[key] = nb;
    return nb;
}

int default_threads(const spuma_solver_controls* ctl)
{
    int t = ctl && ctl->block_threads > 0 ? ctl->block_threads : 256;
    return t;
}

spuma_status launch_solve(spuma_ldu_t h, const SolveArgs& a, int threads, cudaStream_t s)
{
    if (threads < 32 || threads > 1024 || threads % 32) {
        set_error("block_threads must be a multiple of 32 in [32, 1024]");
        return SPUMA_ERR_INVALID_ARG;
    }
    int per_sm = solve_blocks_per_sm(threads, false);
    if (per_sm < 1) { set_error("solver kernel cannot be resident"); return SPUMA_ERR_CUDA; }
    int64_t want = ((int64_t)a.n + threads - 1) / threads;
    int64_t maxg = std::min<int64_t>((int64_t)per_sm * h->num_sms, kMaxBlocks);
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, maxg));
    SPUMA_CUDA(cudaMemsetAsync(h->at<char>(h->L.bar), 0, h->L.status + 256 - h->L.bar, s));
    unsigned long long tns = barrier_timeout_ns();
    void* args[] = {(void*)&a, (void*)&tns};
    SPUMA_CUDA(cudaLaunchCooperativeKernel((const void*)k_solve, grid, threads, args, 0, s));
    count_launch();
    return SPUMA_OK;
}

spuma_status launch_batch_kernel(const BatchTable& t, int grid, int threads, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    unsigned long long tns = barrier_timeout_ns();
    SPUMA_CUDA(cudaLaunchKernelEx(&cfg, k_solve_batch, t, tns));
    return SPUMA_OK;
}

void fill_controls(SolveArgs& a, const spuma_solver_controls* ctl)
{
    a.precond = ctl->precond;
    a.precision = ctl->precision;
    a.tol = ctl->tolerance;
    a.rel_tol = ctl->rel_tol;
    a.inner_rel_tol = ctl->inner_rel_tol;
    a.max_iter = ctl->max_iter;
    a.min_iter = ctl->min_iter;
    a.max_outer = ctl->max_outer;
}

bool ctl_ok(const spuma_solver_controls* c)
{
    if (!c) return false;
    if (c->precond < 0 || c->precond > 2) return false;
    if (c->precision != SPUMA_F64 && c->precision != SPUMA_MIXED) return false;
    if (!(c->tolerance >= 0.0) || !(c->rel_tol >= 0.0) || c->max_iter < 0 || c->min_iter < 0) return false;
    if (c->precision == SPUMA_MIXED && (!(c->inner_rel_tol > 0.0) || c->max_outer < 0)) return false;
    return true;
}

spuma_status pcg_solve_internal(spuma_ldu_t h, const double* diag, const double* upper, const double* b, double* x,
                                const spuma_solver_controls* ctl, spuma_solver_perf* perf, cudaStream_t s,
                                int zero_x0)
{
    if (!h || !ctl_ok(ctl) || (h->n > 0 && (!diag || !b || !x)) || (h->nf > 0 && !upper)) {
        set_error("spuma_pcg_solve: bad argument");
        return SPUMA_ERR_INVALID_ARG;
    }
    if (h->n == 0) {
        if (perf) {
            spuma_solver_perf z{};
            z.converged = 1;
            SPUMA_CUDA(cudaMemcpyAsync(perf, &z, sizeof(z), cudaMemcpyHostToDevice, s));
        }
        return SPUMA_OK;
    }
    SolveArgs a = make_args(h);
    fill_controls(a, ctl);
    a.mode = MODE_SOLVE;
    a.zero_x0 = zero_x0;
    a.diag_orig = diag;
    a.upper_orig = upper;
    a.b_orig = b;
    a.x_orig = x;
    a.perf = perf;
    spuma_status st = launch_solve(h, a, default_threads(ctl), s);
    if (st == SPUMA_OK) h->prepared_precond = ctl->precond;
    return st;
}

}  // namespace spuma

using namespace spuma;

extern "C" {

spuma_status spuma_matrix_prepare(spuma_ldu_t h, const double* diag, const double* upper, int32_t precond,
                                  spuma_stream_t stream)
{
    if (!h || (h->n > 0 && !diag) || (h->nf > 0 && !upper) || precond < 0 || precond > 2) {
        set_error("spuma_matrix_prepare: bad argument");
        return SPUMA_ERR_INVALID_ARG;
    }
    if (h->n == 0) return SPUMA_OK;
    SolveArgs a = make_args(h);
    a.mode = MODE_PREPARE;
    a.precond = precond;
    a.diag_orig = diag;
    a.upper_orig = upper;
    spuma_status st = launch_solve(h, a, 256, (cudaStream_t)stream);
    if (st == SPUMA_OK) h->prepared_precond = precond;
    return st;
}

spuma_status spuma_read_rD(spuma_ldu_t h, double* rD_out, spuma_stream_t stream)
{
    if (!h || (h->n > 0 && !rD_out)) { set_error("spuma_read_rD: bad argument"); return SPUMA_ERR_INVALID_ARG; }
    if (h->n == 0) return SPUMA_OK;
    int g = std::min((h->n + 255) / 256, h->num_sms * 16);
    k_read_rD<<<g, 256, 0, (cudaStream_t)stream>>>(h->n, h->at<int>(h->L.perm), h->at<double>(h->L.rD64), rD_out);
    count_launch();
    SPUMA_CUDA(cudaGetLastError());
    return SPUMA_OK;
}

spuma_status spuma_amul_prepared(spuma_ldu_t h, int32_t precision, const void* x, void* y, spuma_stream_t stream)
{
    if (!h || (h->n > 0 && (!x || !y)) || (precision != SPUMA_F64 && precision != SPUMA_F32)) {
        set_error("spuma_amul_prepared: bad argument");
        return SPUMA_ERR_INVALID_ARG;
    }
    if (h->n == 0) return SPUMA_OK;
    SolveArgs a = make_args(h);
    int g = std::min((h->n + 255) / 256, h->num_sms * 16);
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == SPUMA_F64) {
        Mat<double> A{a.Lptr, a.Lcol, a.La64, a.Lc64, a.Uptr, a.Ucol, a.Ua64, a.Uc64, a.d64, a.rD64};
        k_amul_prepared<double><<<g, 256, 0, s>>>(h->n, A, (const double*)x, (double*)y);
    } else {
        Mat<float> A{a.Lptr, a.Lcol, a.La32, a.Lc32, a.Uptr, a.Ucol, a.Ua32, a.Uc32, a.d32, a.rD32};
        k_amul_prepared<float><<<g, 256, 0, s>>>(h->n, A, (const float*)x, (float*)y);
    }
    count_launch();
    SPUMA_CUDA(cudaGetLastError());
    return SPUMA_OK;
}

spuma_status spuma_permute(spuma_ldu_t h, int32_t dir, const double* src, double* dst, spuma_stream_t stream)
{
    if (!h || (dir != 0 && dir != 1) || (h->n > 0 && (!src || !dst)) || src == dst) {
        set_error("spuma_permute: bad argument");
        return SPUMA_ERR_INVALID_ARG;
    }
    if (h->n == 0) return SPUMA_OK;
    int g = std::min((h->n + 255) / 256, h->num_sms * 16);
    k_permute<<<g, 256, 0, (cudaStream_t)stream>>>(h->n, dir, h->at<int>(h->L.perm), src, dst);
    count_launch();
    SPUMA_CUDA(cudaGetLastError());
    return SPUMA_OK;
}

spuma_status spuma_precondition(spuma_ldu_t h, int32_t precond, const double* r, double* w, spuma_stream_t stream)
{
    if (!h || (h->n > 0 && (!r || !w)) || precond < 0 || precond > 2) {
        set_error("spuma_precondition: bad argument");
        return SPUMA_ERR_INVALID_ARG;
    }
    if (precond != SPUMA_PRECOND_NONE && h->prepared_precond != precond) {
        set_error("spuma_precondition: call spuma_matrix_prepare with this preconditioner first");
        return SPUMA_ERR_INVALID_ARG;
    }
    if (h->n == 0) return SPUMA_OK;
    SolveArgs a = make_args(h);
    a.mode = MODE_PRECONDITION;
    a.precond = precond;
    a.b_orig = r;
    a.x_orig = w;
    return launch_solve(h, a, 256, (cudaStream_t)stream);
}

spuma_status spuma_pcg_solve(spuma_ldu_t h, const double* diag, const double* upper, const double* b, double* x,
                             const spuma_solver_controls* ctl, spuma_solver_perf* perf, spuma_stream_t stream)
{
    return pcg_solve_internal(h, diag, upper, b, x, ctl, perf, (cudaStream_t)stream, 0);
}

}  // extern "C"
