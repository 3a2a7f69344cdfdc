// gamg.cu -- GAMG for the pressure equation (the paper's production pressure
// solver: "GAMG, smoother Richardson", Richardson on every level and a
// diagonal-preconditioned PCG at the coarsest one, with OpenFOAM's coarsening
// unmodified; the paper's other options, Sec. 4.3 smoother table: the
// two-stage Gauss-Seidel smoother and DIC-PCG at the coarsest level).
//
// The hierarchy depends on the mesh only (faces and their area weights), so
// it is built once, on the host, when the solver object is created, as
// OpenFOAM caches its agglomeration: pairwise agglomeration by face weight,
// cells in ascending order; an unassigned cell pairs with its unassigned
// neighbour across the heaviest face (first in face order on ties); a cell
// whose neighbours are all taken joins the aggregate across its heaviest
// face; a cell without faces stays alone.  The coarse graph keeps the faces
// between different aggregates, (min, max) ordered and sorted, with summed
// weights; levels are added while the coarse level has more than 10 cells
// and fewer cells than the level above.
//
// Every solve runs in one persistent cooperative launch: the Galerkin
// coarse matrices (P^T A P with piecewise-constant P, sums in ascending fine
// order), then the outer iterations x += V(0, r), r = b - A x with PCG's
// normalised residual and stopping rule.  V(k, r): no pre-smoothing;
// restriction (sum over the aggregate); the coarsest level by diagonal PCG
// from 0 to 1e-8 relative; prolongation by injection, scaled by the A-norm
// optimal step (e.r)/(e.Ae); two damped-Jacobi sweeps e += (2/3 rD)(r - Ae)
// (or two two-stage Gauss-Seidel sweeps e += (D^-1 - D^-1 L D^-1)(r - A e)).
// Levels of at most two rows per thread of one block run on the first block
// alone with block-level barriers (the coarsest level's PCG on one warp when
// it has at most 32 cells); the others on the whole grid.  Storage: level 0
// in the mesh handle's internal (DIC level, Morton) order, the middle levels
// breadth-first, the coarsest as built; rows and aggregates are moved, never
// reordered inside, so every per-row sum follows the sequential definition's
// order; dot products are deterministic block/grid reductions.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <memory>
#include <stdexcept>
#include <system_error>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"

namespace spuma {

constexpr int kGamgMaxLevels = 50;
constexpr int kGamgCoarsest = 10;
constexpr double kGamgOmega = 2.0 / 3.0;
constexpr int kGamgPostSweeps = 2;
constexpr double kGamgCoarseRelTol = 1e-8;
enum GamgSlot { GS_A = 0, GS_B = 1, GS_C = 2, GS_D = 3 };   // reduction slots

// Device view of one level (rows in the level's storage order: see
// gamg_store_order; faces in the level's own numbering).
struct GamgLevel {
    int n, nf;
    const int *rptr, *rcol, *rfac;          // row CSR for A_k: entries in ascending face order
    const int* rlo;                         // lower entries of each row (leading its entries)
    const int* agg;                         // cell -> next-level cell (k < L-1)
    const int *cptr, *ccell;                // next-level cell -> its cells (ascending)
    const int *fptr, *fface;                // next-level face -> its faces (ascending)
    const int *iptr, *iface;                // next-level cell -> the faces inside it (ascending)
    const double *diag, *upper;             // A_k (level 0: the caller's arrays)
    double *cdiag, *cupper;                 // A_{k+1} written here (k < L-1)
    double *wrd;                            // omega / diag (Richardson) or 1 / diag (two-stage Gauss-Seidel)
    double *rval;                           // A_k's off-diagonal coefficients in row-CSR order (per solve)
    double *r, *e, *q, *y;                  // right-hand side, correction, scratch, first-stage vector
};

// Level 0 in the mesh handle's internal order (rows grouped by DIC level,
// Morton order inside a level): the solver's internal CSR (lower entries,
// then upper, each in face order) and, when the mesh has it, its fixed-width
// Amul layout, their coefficients gathered from the caller's arrays at the
// start of each solve; the aggregation lists at internal positions (built
// with the hierarchy).  Every row sum keeps its face order, so the results
// are those of the original-order level.  Used when the hierarchy has more
// than one level.
struct GamgLvl0 {
    int on, n, ell_w;
    const int *perm, *Lptr, *Lcol, *Lface, *Uptr, *Ucol, *Uface, *Ecol;
    double *La, *Ua, *d, *Ea;             // the handle's matrix region, filled per solve
    const int* ccell_int;                 // level 0's aggregate lists at internal positions
};

struct GamgArgs {
    GamgLvl0 z;
    int nlev, small_from;
    const GamgLevel* lv;                    // device array [nlev]
    const double* b_orig;
    double* x_orig;
    double *x, *b, *res;                    // level-0 solution, rhs, outer residual (= lv[0].r)
    double *pw, *pp, *pq, *px;              // coarsest-level PCG vectors
    double* crD;                            // coarsest-level DIC reciprocal pivots
    int smoother;                           // 0 Richardson, 1 two-stage Gauss-Seidel
    int coarsest_precond;                   // SPUMA_PRECOND_DIAGONAL or SPUMA_PRECOND_DIC
    double* partials;
    int* status;
    spuma_solver_perf* perf;
    int max_iter, min_iter;
    double tol, rel_tol;
    long long* clk;                         // optional per-phase SM-clock totals of block 0 (diagnostics)
    // coarse levels (k >= 1) of at most this many cells apply the correction's
    // scaling inside their first smoothing sweep, each gathered e_j multiplied
    // by the factor as it is read (the same rounded products as the scaled
    // copy), one barrier step fewer; others keep the separate pass.  A
    // measurement override (SPUMA_GAMG_FUSE_SCALE_ROWS), 0 by default.
    int fuse_rows;
};

// --------------------------------------------------------------- device ---
// Optional phase timing (SPUMA_PHASE_CLOCKS): block 0's thread 0 adds SM-clock
// deltas into clk[slot]: 0..49 restriction into level k+1 (slot k), 64..113
// prolongation, scaling and smoothing of level k (64 + k), 128 the coarsest
// level, 129 the outer update and residual, 130 V-cycles counted.
struct GamgClock {
    long long* acc;
    long long t;
    __device__ __forceinline__ GamgClock(long long* a, int bid)
    {
        acc = (a && bid == 0 && threadIdx.x == 0) ? a : nullptr;
        t = clock64();
    }
    __device__ __forceinline__ void lap(int slot)
    {
        if (acc) {
            const long long now = clock64();
            acc[slot] += now - t;
            t = now;
        }
    }
};
struct Exec {
    int first, stride;
    bool grid, active;
};

__device__ __forceinline__ Exec exec_for(const GamgArgs& a, int k, const Group& g)
{
    if (k >= a.small_from)
        return Exec{(int)threadIdx.x, (int)blockDim.x, false, g.bid == 0};
    return Exec{g.bid * (int)blockDim.x + (int)threadIdx.x, g.nblocks * (int)blockDim.x, true, true};
}

// Barrier after a step done with `x`: the grid barrier, or the first block's
// block barrier (the other blocks skip it).
__device__ __forceinline__ bool exec_sync(const Exec& x, const Group& g)
{
    if (x.grid) return group_sync(g);
    if (g.bid == 0) __syncthreads();
    return true;
}

// Sums of NV values over the executing threads, returned to them.
template <int NV>
__device__ __forceinline__ bool exec_sum(const Exec& x, double (&v)[NV], const GamgArgs& a, int slot,
                                         const Group& g)
{
    if (x.grid) {
        block_reduce_store<NV>(v, a.partials, slot, g.bid);
        if (!group_sync(g)) return false;
        grid_reduce_read<NV>(v, a.partials, slot, g.nblocks);
        return true;
    }
    if (g.bid != 0) return true;
    // the first block alone: the same sums through shared memory only
    __shared__ double red[NV][32];
    __shared__ double bc[NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double s = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        v[k] = s;
    }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; k++) red[k][warp] = v[k];
    __syncthreads();
    if (warp == 0)
#pragma unroll
        for (int k = 0; k < NV; k++) {
            double s = lane < nw ? red[k][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) bc[k] = s;
        }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = bc[k];
    __syncthreads();
    return true;
}

// (A_k x)_i: d_i x_i, then the row's entries in face order, one FMA each;
// entries loaded in groups of 8 (columns and coefficients, then the
// gathers), the FMAs in entry order.
// X(c) gives x_c (a plain load, or a gather through the aggregation map).
template <class X>
__device__ __forceinline__ double gamg_amul_row_g(const GamgLevel& L, const double* d, X x, int i)
{
    double y = __dmul_rn(d[i], x(i));
    const int e1 = L.rptr[i + 1];
    for (int e0 = L.rptr[i]; e0 < e1; e0 += 8) {
        int c[8];
        double v[8], xv[8];
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const bool ok = e0 + j < e1;
            c[j] = ok ? __ldg(L.rcol + e0 + j) : -1;
            v[j] = ok ? L.rval[e0 + j] : 0.0;
        }
#pragma unroll
        for (int j = 0; j < 8; j++) xv[j] = c[j] >= 0 ? x(c[j]) : 0.0;
#pragma unroll
        for (int j = 0; j < 8; j++)
            if (c[j] >= 0) y = __fma_rn(v[j], xv[j], y);
    }
    return y;
}
__device__ __forceinline__ double gamg_amul_row(const GamgLevel& L, const double* d, const double* x, int i)
{
    return gamg_amul_row_g(L, d, [x](int c) { return x[c]; }, i);
}

// (A_0 x)_p in internal order: d_p x_p, then the row's entries in face order
// (fixed-width layout, or lower then upper CSR entries), one FMA each; entry
// loads grouped, then the gathers, then the FMAs in order.
template <class X>
__device__ __forceinline__ double lvl0_amul_row(const GamgLvl0& z, X x, int p)
{
    double y = __dmul_rn(z.d[p], x(p));
    if (z.ell_w > 0) {
        for (int j0 = 0; j0 < z.ell_w; j0 += 6) {
            int c[6];
            double v[6], xv[6];
#pragma unroll
            for (int j = 0; j < 6; j++) {
                const bool ok = j0 + j < z.ell_w;
                const size_t e = (size_t)(j0 + j) * z.n + p;
                c[j] = ok ? __ldcs(z.Ecol + e) : -1;
                v[j] = ok ? __ldcs(z.Ea + e) : 0.0;
            }
#pragma unroll
            for (int j = 0; j < 6; j++) xv[j] = c[j] >= 0 ? x(c[j]) : 0.0;
#pragma unroll
            for (int j = 0; j < 6; j++)
                if (c[j] >= 0) y = __fma_rn(v[j], xv[j], y);
        }
        return y;
    }
    for (int e = z.Lptr[p]; e < z.Lptr[p + 1]; e++) y = __fma_rn(z.La[e], x(z.Lcol[e]), y);
    for (int e = z.Uptr[p]; e < z.Uptr[p + 1]; e++) y = __fma_rn(z.Ua[e], x(z.Ucol[e]), y);
    return y;
}

// A level's row operations, in internal order at level 0 when z.on.
__device__ __forceinline__ double level_amul_row(const GamgArgs& a, int k, const double* x, int i)
{
    auto xv = [x](int c) { return x[c]; };
    if (k == 0 && a.z.on) return lvl0_amul_row(a.z, xv, i);
    return gamg_amul_row_g(a.lv[k], a.lv[k].diag, xv, i);
}

// Rows first, first + stride, ... of level k: body(i, (A_k x)_i, x_i, U_i,
// V_i) (U, V: the pass's own per-row inputs; NULL reads 0).  Level 0 in
// internal order with a fixed-width layout of at most 6 entries is
// software-pipelined: the next row's columns are loaded before this row's
// gathers, and this row's coefficients, x, diagonal, U and V load beside its
// gathers, so a row costs about one memory round trip; its sum is the same
// FMA chain as lvl0_amul_row's.  Measured at 200^3 (face-area Richardson):
// level 0's passes 948 -> 785 us per V-cycle; the same for the outer residual
// pass, and the next row's extents one row ahead on the row-CSR levels, were
// slower and are not used.
template <class Body>
__device__ __forceinline__ void level_rows(const GamgArgs& a, int k, const double* x, const double* U,
                                           const double* V, int first, int stride, Body body)
{
    const int n = a.lv[k].n;
    if (k == 0 && a.z.on && a.z.ell_w > 0 && a.z.ell_w <= 6) {
        const GamgLvl0& z = a.z;
        auto cols = [&](int (&c)[6], int p) {
#pragma unroll
            for (int j = 0; j < 6; j++) c[j] = j < z.ell_w ? __ldcs(z.Ecol + (size_t)j * z.n + p) : -1;
        };
        int cur[6];
        if (first < n) cols(cur, first);
        for (int p = first; p < n; p += stride) {
            int nxt[6];
            const int pn = p + stride;
            if (pn < n) cols(nxt, pn);
            double g6[6];
#pragma unroll
            for (int j = 0; j < 6; j++) g6[j] = cur[j] >= 0 ? x[cur[j]] : 0.0;
            const double xp = x[p], d = __ldcs(z.d + p);
            const double u = U ? U[p] : 0.0, v = V ? V[p] : 0.0;
            double y = __dmul_rn(d, xp);
#pragma unroll
            for (int j = 0; j < 6; j++)
                if (cur[j] >= 0) y = __fma_rn(__ldcs(z.Ea + (size_t)j * z.n + p), g6[j], y);
            body(p, y, xp, u, v);
#pragma unroll
            for (int j = 0; j < 6; j++) cur[j] = nxt[j];
        }
        return;
    }
    for (int i = first; i < n; i += stride) {
        const double u = U ? U[i] : 0.0, v = V ? V[i] : 0.0;
        body(i, level_amul_row(a, k, x, i), x[i], u, v);
    }
}

// s - sum over the row's lower entries (face order) of a_f y_col, one FMA each
// (the two-stage Gauss-Seidel's second stage).
__device__ __forceinline__ double level_lower_sweep(const GamgArgs& a, int k, const double* y, int i, double s)
{
    if (k == 0 && a.z.on) {
        for (int e = a.z.Lptr[i]; e < a.z.Lptr[i + 1]; e++) s = __fma_rn(-a.z.La[e], y[a.z.Lcol[e]], s);
        return s;
    }
    const GamgLevel& L = a.lv[k];
    const int e0 = L.rptr[i], e1 = e0 + L.rlo[i];
    for (int e = e0; e < e1; e++) s = __fma_rn(-L.rval[e], y[L.rcol[e]], s);
    return s;
}

// Level 0's coefficients in internal order (per solve): the CSR entries, the
// diagonal and the fixed-width layout, from the caller's (original) arrays.
__device__ void lvl0_gather(const GamgArgs& a, int first, int stride)
{
    const GamgLvl0& z = a.z;
    const GamgLevel& L0 = a.lv[0];
    for (int e = first; e < L0.nf; e += stride) {
        z.La[e] = L0.upper[z.Lface[e]];
        z.Ua[e] = L0.upper[z.Uface[e]];
    }
    for (int p = first; p < z.n; p += stride) {
        z.d[p] = L0.diag[z.perm[p]];
        if (z.ell_w > 0) {
            const int l0 = z.Lptr[p], nl = z.Lptr[p + 1] - l0, u0 = z.Uptr[p], nt = nl + z.Uptr[p + 1] - u0;
            for (int j = 0; j < z.ell_w; j++)
                z.Ea[(size_t)j * z.n + p] =
                    j < nl ? L0.upper[z.Lface[l0 + j]] : (j < nt ? L0.upper[z.Uface[u0 + j - nl]] : 0.0);
        }
    }
}

// Galerkin coarse matrices level by level, then omega/diag on every level.
__device__ bool gamg_coarse_matrices(const GamgArgs& a, const Group& g)
{
    if (a.z.on) lvl0_gather(a, g.bid * (int)blockDim.x + (int)threadIdx.x, g.nblocks * (int)blockDim.x);
    for (int k = 0; k + 1 < a.nlev; k++) {
        const GamgLevel& F = a.lv[k];
        const Exec x = exec_for(a, k + 1, g);
        if (x.active) {
            const int nfc = a.lv[k + 1].nf, nc = a.lv[k + 1].n;
            for (int c = x.first; c < nfc; c += x.stride) {
                double s = 0.0;
                for (int j = F.fptr[c]; j < F.fptr[c + 1]; j++) s = __dadd_rn(s, F.upper[F.fface[j]]);
                F.cupper[c] = s;
            }
            for (int c = x.first; c < nc; c += x.stride) {
                double s = 0.0;
                for (int j = F.cptr[c]; j < F.cptr[c + 1]; j++) s = __dadd_rn(s, F.diag[F.ccell[j]]);
                for (int j = F.iptr[c]; j < F.iptr[c + 1]; j++) s = __dadd_rn(s, __dmul_rn(2.0, F.upper[F.iface[j]]));
                F.cdiag[c] = s;
            }
        }
        if (!exec_sync(x, g)) return false;
    }
    // the first block's levels become visible to every block here
    if (!group_sync(g)) return false;
    const int first = g.bid * (int)blockDim.x + (int)threadIdx.x, stride = g.nblocks * (int)blockDim.x;
    for (int k = 0; k < a.nlev; k++) {
        const GamgLevel& L = a.lv[k];
        const bool z0 = k == 0 && a.z.on;
        const double* dg = z0 ? a.z.d : L.diag;
        for (int i = first; i < L.n; i += stride)
            L.wrd[i] = a.smoother == 1 ? __ddiv_rn(1.0, dg[i]) : __dmul_rn(kGamgOmega, __ddiv_rn(1.0, dg[i]));
        if (!z0)
            for (int e = first; e < 2 * L.nf; e += stride) L.rval[e] = L.upper[L.rfac[e]];
    }
    if (!group_sync(g)) return false;
    // DIC factor of the coarsest matrix by one thread, rows ascending: p_i =
    // d_i - sum of (a a)/p_col over the row's lower entries in face order (the
    // sequential face loop's order), then rD = 1/p; a pivot <= 0 is an error
    if (a.coarsest_precond == SPUMA_PRECOND_DIC && g.bid == 0 && threadIdx.x == 0) {
        const GamgLevel& L = a.lv[a.nlev - 1];
        for (int i = 0; i < L.n; i++) {
            double piv = L.diag[i];
            for (int e = L.rptr[i]; e < L.rptr[i + 1]; e++) {
                const int c = L.rcol[e];
                if (c < i) piv = __dsub_rn(piv, __ddiv_rn(__dmul_rn(L.rval[e], L.rval[e]), a.crD[c]));
            }
            a.crD[i] = piv;
            if (!(piv > 0.0)) flag_error(a.status, SPUMA_ERR_NOT_SPD, i);
        }
        for (int i = 0; i < L.n; i++) a.crD[i] = __ddiv_rn(1.0, a.crD[i]);
    }
    return group_sync(g);
}

// w = M^-1 r for the coarsest level's DIC factor, by one thread: w_i = rD_i
// r_i; forward, rows ascending, lower entries in face order: w_i -= (rD_i a)
// w_col; backward, rows descending, upper entries in descending face order:
// w_i -= (rD_i a) w_col; each -= one FMA of the rounded product (the order of
// the sequential face loops).
__device__ void gamg_dic_seq(const GamgLevel& L, const double* rD, const double* r, double* w)
{
    for (int i = 0; i < L.n; i++) w[i] = __dmul_rn(rD[i], r[i]);
    for (int i = 0; i < L.n; i++) {
        double wi = w[i];
        for (int e = L.rptr[i]; e < L.rptr[i + 1]; e++) {
            const int c = L.rcol[e];
            if (c < i) wi = __fma_rn(-__dmul_rn(rD[i], L.rval[e]), w[c], wi);
        }
        w[i] = wi;
    }
    for (int i = L.n - 1; i >= 0; i--) {
        double wi = w[i];
        for (int e = L.rptr[i + 1] - 1; e >= L.rptr[i]; e--) {
            const int c = L.rcol[e];
            if (c > i) wi = __fma_rn(-__dmul_rn(rD[i], L.rval[e]), w[c], wi);
        }
        w[i] = wi;
    }
}

// Sum over the warp's lanes (a butterfly: every lane gets the same value,
// the same sum as the first block's reduction when only warp 0 holds values).
__device__ __forceinline__ double warp_sum(double s)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// The coarsest level's PCG on warp 0 of the first block, one row per lane
// (levels of at most 32 cells, the usual case): the same steps and sums as
// gamg_coarsest below, with warp barriers instead of block barriers.
__device__ void gamg_coarsest_warp(const GamgArgs& a, const GamgLevel& L)
{
    const int i = (int)threadIdx.x;
    const bool row = i < L.n;
    double* e = L.e;
    double* r = a.pw;
    double *w = a.pq, *p = a.pp, *q = a.px;
    double ri = row ? L.r[i] : 0.0;
    if (row) {
        e[i] = 0.0;
        r[i] = ri;
    }
    const double v0 = warp_sum(row ? fabs(ri) : 0.0);
    const double nfac = v0 + 1e-20;
    const double res0 = v0 / nfac;
    double res = res0, rho = 1.0, rho_old;
    const int max_it = 2 * L.n + 10;
    int it = 0;
    if (res0 > 0.0) {
        do {
            rho_old = rho;
            double wi = 0.0;
            if (a.coarsest_precond == SPUMA_PRECOND_DIC) {
                __syncwarp();
                if (i == 0) gamg_dic_seq(L, a.crD, r, w);
                __syncwarp();
                if (row) wi = w[i];
            } else if (row) {
                wi = __dmul_rn(__ddiv_rn(1.0, L.diag[i]), ri);
                w[i] = wi;
            }
            rho = warp_sum(row ? __fma_rn(wi, ri, 0.0) : 0.0);
            const double beta = it == 0 ? 0.0 : rho / rho_old;
            if (row) p[i] = it == 0 ? wi : __fma_rn(beta, p[i], wi);
            __syncwarp();
            double qi = 0.0;
            if (row) {
                qi = gamg_amul_row(L, L.diag, p, i);
                q[i] = qi;
            }
            const double s = warp_sum(row ? __fma_rn(qi, p[i], 0.0) : 0.0);
            if (fabs(s) / nfac < 1e-300) break;
            const double alpha = rho / s;
            if (row) {
                e[i] = __fma_rn(alpha, p[i], e[i]);
                ri = __fma_rn(-alpha, qi, ri);
                r[i] = ri;
            }
            res = warp_sum(row ? fabs(ri) : 0.0) / nfac;
            __syncwarp();
        } while (++it < max_it && !(res < kGamgCoarseRelTol * res0));
    }
}

// Coarsest level: PCG with the diagonal preconditioner from 0, relative
// tolerance kGamgCoarseRelTol, at most 2n + 10 iterations (PCG recurrences).
__device__ bool gamg_coarsest(const GamgArgs& a, const Group& g)
{
    const int k = a.nlev - 1;
    const GamgLevel& L = a.lv[k];
    const Exec x = exec_for(a, k, g);
    if (!x.active) return true;   // the coarsest level is the first block's alone
    if (!x.grid && L.n <= 32) {
        if (threadIdx.x < 32) gamg_coarsest_warp(a, L);
        return exec_sync(x, g);
    }
    double* e = L.e;
    double* r = a.pw;   // residual
    double *w = a.pq, *p = a.pp, *q = a.px;
    double v[1] = {0.0};
    if (x.active)
        for (int i = x.first; i < L.n; i += x.stride) {
            e[i] = 0.0;
            r[i] = L.r[i];
            v[0] += fabs(L.r[i]);
        }
    if (!exec_sum<1>(x, v, a, GS_A, g)) return false;
    const double nfac = v[0] + 1e-20;   // x = 0: sum|A x - 0| + sum|b - 0|
    const double res0 = v[0] / nfac;
    double res = res0, rho = 1.0, rho_old;
    const int max_it = 2 * L.n + 10;
    int it = 0;
    if (res0 > 0.0) {
        do {
            rho_old = rho;
            double t[1] = {0.0};
            if (a.coarsest_precond == SPUMA_PRECOND_DIC) {
                if (g.bid == 0 && threadIdx.x == 0) gamg_dic_seq(L, a.crD, r, w);
                if (!exec_sync(x, g)) return false;
                for (int i = x.first; i < L.n; i += x.stride) t[0] = __fma_rn(w[i], r[i], t[0]);
            } else {
                for (int i = x.first; i < L.n; i += x.stride) {
                    const double wi = __dmul_rn(__ddiv_rn(1.0, L.diag[i]), r[i]);
                    w[i] = wi;
                    t[0] = __fma_rn(wi, r[i], t[0]);
                }
            }
            if (!exec_sum<1>(x, t, a, GS_B, g)) return false;
            rho = t[0];
            const double beta = it == 0 ? 0.0 : rho / rho_old;
            if (x.active)
                for (int i = x.first; i < L.n; i += x.stride) p[i] = it == 0 ? w[i] : __fma_rn(beta, p[i], w[i]);
            if (!exec_sync(x, g)) return false;
            double s[1] = {0.0};
            if (x.active)
                for (int i = x.first; i < L.n; i += x.stride) {
                    const double qi = gamg_amul_row(L, L.diag, p, i);
                    q[i] = qi;
                    s[0] = __fma_rn(qi, p[i], s[0]);
                }
            if (!exec_sum<1>(x, s, a, GS_C, g)) return false;
            if (fabs(s[0]) / nfac < 1e-300) break;
            const double alpha = rho / s[0];
            double m[1] = {0.0};
            if (x.active)
                for (int i = x.first; i < L.n; i += x.stride) {
                    e[i] = __fma_rn(alpha, p[i], e[i]);
                    r[i] = __fma_rn(-alpha, q[i], r[i]);
                    m[0] += fabs(r[i]);
                }
            if (!exec_sum<1>(x, m, a, GS_D, g)) return false;
            res = m[0] / nfac;
        } while (++it < max_it && !(res < kGamgCoarseRelTol * res0));
    }
    return exec_sync(x, g);
}

// e_0 = V(0, r_0), with r_0 = a.res; the last smoothing sweep of level 0 also
// adds e_0 to x (the outer update, fused).
__device__ bool gamg_vcycle(const GamgArgs& a, const Group& g, GamgClock& ck)
{
    // restriction down to the coarsest level
    for (int k = 0; k + 1 < a.nlev; k++) {
        const GamgLevel& F = a.lv[k];
        const GamgLevel& C = a.lv[k + 1];
        const Exec x = exec_for(a, k + 1, g);
        const int* cc = k == 0 && a.z.on ? a.z.ccell_int : F.ccell;
        if (x.active)
            for (int c = x.first; c < C.n; c += x.stride) {
                double s = 0.0;
                for (int j = F.cptr[c]; j < F.cptr[c + 1]; j++) s = __dadd_rn(s, F.r[cc[j]]);
                C.r[c] = s;
            }
        if (!exec_sync(x, g)) return false;
        ck.lap(k);
    }
    if (!gamg_coarsest(a, g)) return false;
    ck.lap(128);
    // prolongation, scaling and smoothing back up
    for (int k = a.nlev - 2; k >= 0; k--) {
        const GamgLevel& L = a.lv[k];
        const GamgLevel& C = a.lv[k + 1];
        if (k + 1 == a.small_from && !group_sync(g)) return false;   // the first block's levels are done
        const Exec x = exec_for(a, k, g);
        if (x.active)
            for (int i = x.first; i < L.n; i += x.stride) L.e[i] = C.e[L.agg[i]];
        if (!exec_sync(x, g)) return false;
        double v[2] = {0.0, 0.0};
        if (x.active)
            level_rows(a, k, L.e, L.r, nullptr, x.first, x.stride, [&](int, double qi, double ei, double ri, double) {
                v[0] = __fma_rn(ei, ri, v[0]);
                v[1] = __fma_rn(ei, qi, v[1]);
            });
        if (!exec_sum<2>(x, v, a, GS_A, g)) return false;
        const bool fuse = k >= 1 && L.n <= a.fuse_rows;
        const double sc = v[1] > 0.0 ? v[0] / v[1] : 1.0;   // x 1.0 leaves every value as it is
        if (!fuse && v[1] > 0.0) {
            if (x.active)
                for (int i = x.first; i < L.n; i += x.stride) L.e[i] = __dmul_rn(L.e[i], sc);
            if (!exec_sync(x, g)) return false;
        }
        auto scaled_e = [&L, sc](int c) { return __dmul_rn(L.e[c], sc); };
        if (a.smoother == 1) {
            // two-stage Gauss-Seidel: q = r - A e, y = rD q; then e += rD (q - L y),
            // the row's lower entries in face order (one FMA each)
            for (int s = 0; s < kGamgPostSweeps; s++) {
                const bool sc0 = fuse && s == 0;   // e read scaled in this sweep
                if (x.active) {
                    if (sc0) {
                        for (int i = x.first; i < L.n; i += x.stride) {
                            const double qi = __dsub_rn(L.r[i], gamg_amul_row_g(L, L.diag, scaled_e, i));
                            L.q[i] = qi;
                            L.y[i] = __dmul_rn(L.wrd[i], qi);
                        }
                    } else {
                        level_rows(a, k, L.e, L.r, L.wrd, x.first, x.stride,
                                   [&](int i, double ae, double, double ri, double wi) {
                                       const double qi = __dsub_rn(ri, ae);
                                       L.q[i] = qi;
                                       L.y[i] = __dmul_rn(wi, qi);
                                   });
                    }
                }
                if (!exec_sync(x, g)) return false;
                const bool fold = k == 0 && s == kGamgPostSweeps - 1;   // x += e_0 here
                if (x.active)
                    for (int i = x.first; i < L.n; i += x.stride) {
                        const double si = level_lower_sweep(a, k, L.y, i, L.q[i]);
                        const double e0 = sc0 ? __dmul_rn(L.e[i], sc) : L.e[i];
                        const double ei = __dadd_rn(e0, __dmul_rn(L.wrd[i], si));
                        L.e[i] = ei;
                        if (fold) a.x[i] = __dadd_rn(a.x[i], ei);
                    }
                if (!exec_sync(x, g)) return false;
            }
        } else {
            // Jacobi sweeps alternate between e and q (an even count ends in e)
            static_assert(kGamgPostSweeps % 2 == 0, "sweeps alternate e -> q -> e");
            for (int s = 0; s < kGamgPostSweeps; s++) {
                const double* src = (s & 1) ? L.q : L.e;
                double* dst = (s & 1) ? L.e : L.q;
                const bool fold = k == 0 && s == kGamgPostSweeps - 1;   // x += e_0 here
                if (x.active) {
                    if (fuse && s == 0) {
                        for (int i = x.first; i < L.n; i += x.stride)
                            dst[i] = __fma_rn(L.wrd[i], __dsub_rn(L.r[i], gamg_amul_row_g(L, L.diag, scaled_e, i)),
                                              scaled_e(i));
                    } else {
                        level_rows(a, k, src, L.wrd, L.r, x.first, x.stride,
                                   [&](int i, double as, double si, double wi, double ri) {
                                       const double ei = __fma_rn(wi, __dsub_rn(ri, as), si);
                                       dst[i] = ei;
                                       if (fold) a.x[i] = __dadd_rn(a.x[i], ei);
                                   });
                    }
                }
                if (!exec_sync(x, g)) return false;
            }
        }
        ck.lap(64 + k);
    }
    if (a.nlev == 1 || a.small_from == 0) return group_sync(g);
    return true;
}

__global__ void __launch_bounds__(1024, 1) k_gamg(GamgArgs a, unsigned long long timeout_ns)
{
    Group g{reinterpret_cast<unsigned long long*>(a.status + DS_BARRIER), a.status, (int)gridDim.x, (int)blockIdx.x, timeout_ns};
    spuma_solver_perf pf{};
    pf.n_levels = a.nlev;
    const GamgLevel& L0 = a.lv[0];
    struct {
        int first, stride;
    } it{g.bid * (int)blockDim.x + (int)threadIdx.x, g.nblocks * (int)blockDim.x};
    bool ok = gamg_coarse_matrices(a, g);
    // x, b, r = b - A x, normFactor (row sums of A times mean(x)), res0
    double v[1] = {0.0};
    const bool z0 = a.z.on;   // level 0 (x, b, r) in internal order
    if (ok) {
        for (int i = it.first; i < L0.n; i += it.stride) {
            const int o = z0 ? a.z.perm[i] : i;
            a.x[i] = a.x_orig[o];
            a.b[i] = a.b_orig[o];
            v[0] += a.x_orig[i];
            if (!isfinite(a.b_orig[i])) flag_error(a.status, SPUMA_ERR_NONFINITE, i);
        }
        block_reduce_store<1>(v, a.partials, GS_A, g.bid);
        ok = group_sync(g);
    }
    double nfac = 1.0, res0 = 0.0, res = 0.0;
    if (ok) {
        double t[1];
        grid_reduce_read<1>(t, a.partials, GS_A, g.nblocks);
        const double xbar = L0.n > 0 ? t[0] / (double)L0.n : 0.0;
        double acc[2] = {0.0, 0.0};
        for (int i = it.first; i < L0.n; i += it.stride) {
            const double q = level_amul_row(a, 0, a.x, i);
            const double r = a.b[i] - q;
            a.res[i] = r;
            double s;
            if (z0) {
                s = a.z.d[i];
                for (int e = a.z.Lptr[i]; e < a.z.Lptr[i + 1]; e++) s += a.z.La[e];
                for (int e = a.z.Uptr[i]; e < a.z.Uptr[i + 1]; e++) s += a.z.Ua[e];
            } else {
                s = L0.diag[i];
                for (int e = L0.rptr[i]; e < L0.rptr[i + 1]; e++) s += L0.rval[e];
            }
            const double tt = s * xbar;
            acc[0] += fabs(r);
            acc[1] += fabs(q - tt) + fabs(a.b[i] - tt);
        }
        block_reduce_store<2>(acc, a.partials, GS_B, g.bid);
        ok = group_sync(g);
        if (ok) {
            grid_reduce_read<2>(acc, a.partials, GS_B, g.nblocks);
            nfac = acc[1] + 1e-20;
            res0 = acc[0] / nfac;
            res = res0;
        }
    }
    auto conv = [&](double rr) { return rr < a.tol || (a.rel_tol > 0.0 && rr < a.rel_tol * res0); };
    int n_it = 0;
    GamgClock ck(a.clk, g.bid);
    if (ok && (a.min_iter > 0 || !conv(res0))) {
        for (;;) {
            ok = gamg_vcycle(a, g, ck);
            if (!ok) break;
            double acc[1] = {0.0};
            if (a.nlev == 1) {   // otherwise the last smoothing sweep of level 0 added e_0 to x
                for (int i = it.first; i < L0.n; i += it.stride) a.x[i] = __dadd_rn(a.x[i], L0.e[i]);
                ok = group_sync(g);
                if (!ok) break;
            }
            for (int i = it.first; i < L0.n; i += it.stride) {
                const double r = a.b[i] - level_amul_row(a, 0, a.x, i);
                a.res[i] = r;
                acc[0] += fabs(r);
            }
            block_reduce_store<1>(acc, a.partials, GS_C, g.bid);
            ok = group_sync(g);
            if (!ok) break;
            grid_reduce_read<1>(acc, a.partials, GS_C, g.nblocks);
            res = acc[0] / nfac;
            n_it++;
            ck.lap(129);
            if (ck.acc) ck.acc[130] += 1;
            if (!((n_it < a.max_iter && !conv(res)) || n_it < a.min_iter)) break;
        }
    }
    // the report's true residual ||b - A x||_2 / ||b||_2 (||b - A x||_2 when b = 0)
    if (ok) {
        double acc[2] = {0.0, 0.0};
        for (int i = it.first; i < L0.n; i += it.stride) {
            const double r = __dsub_rn(a.b[i], level_amul_row(a, 0, a.x, i));
            acc[0] = __fma_rn(r, r, acc[0]);
            acc[1] = __fma_rn(a.b[i], a.b[i], acc[1]);
        }
        block_reduce_store<2>(acc, a.partials, GS_D, g.bid);
        ok = group_sync(g);
        if (ok) {
            grid_reduce_read<2>(acc, a.partials, GS_D, g.nblocks);
            pf.true_rel_residual_l2 =
                acc[1] > 0.0 ? __ddiv_rn(__dsqrt_rn(acc[0]), __dsqrt_rn(acc[1])) : __dsqrt_rn(acc[0]);
        }
    }
    if (ok)
        for (int i = it.first; i < L0.n; i += it.stride) a.x_orig[z0 ? a.z.perm[i] : i] = a.x[i];
    if (g.bid == 0 && threadIdx.x == 0 && a.perf) {
        pf.initial_residual = res0;
        pf.final_residual = res;
        pf.n_iter = n_it;
        pf.converged = conv(res);
        __threadfence();
        pf.status = ld_volatile_int(a.status);
        if (!ok && pf.status == 0) pf.status = SPUMA_ERR_DEVICE_TIMEOUT;
        if (pf.status != 0) pf.converged = 0;
        *a.perf = pf;
    }
}

// ----------------------------------------------------------------- host ---
struct GamgHostLevel {
    int n = 0, nf = 0;
    std::vector<int> l, u;                   // faces of this level (sorted by (l, u))
    std::vector<int> rptr, rcol, rfac;       // row CSR
    std::vector<int> rlo;                    // lower entries of each row (they come first)
    std::vector<int> agg, cptr, ccell, fptr, fface, iptr, iface;   // towards the next level
    std::vector<int> ccell_int;              // level 0: ccell at internal positions
};

static void gamg_rows(GamgHostLevel& L)
{
    L.rptr.assign(L.n + 1, 0);
    for (int f = 0; f < L.nf; f++) {
        L.rptr[L.l[f] + 1]++;
        L.rptr[L.u[f] + 1]++;
    }
    for (int i = 0; i < L.n; i++) L.rptr[i + 1] += L.rptr[i];
    std::vector<int> cur(L.rptr.begin(), L.rptr.end() - 1);
    L.rcol.resize(2 * (size_t)L.nf);
    L.rfac.resize(2 * (size_t)L.nf);
    for (int f = 0; f < L.nf; f++) {   // ascending f: each row's entries in face order
        int a = L.l[f], b = L.u[f];
        L.rcol[cur[a]] = b;
        L.rfac[cur[a]++] = f;
        L.rcol[cur[b]] = a;
        L.rfac[cur[b]++] = f;
    }
}

// f(begin, end) over [0, n) in contiguous pieces on the host's cores (loops
// whose iterations write disjoint entries).
template <class Fn>
static void par_for(size_t n, Fn f, size_t min_n = 65536)
{
    const unsigned hc = std::thread::hardware_concurrency();
    const size_t T = std::min<size_t>(16, hc > 0 ? hc : 1);
    if (n < min_n || T == 1) {
        f((size_t)0, n);
        return;
    }
    const size_t chunk = (n + T - 1) / T;
    std::vector<std::thread> th;
    th.reserve(T);
    for (size_t t = 0; t < T; t++) {
        const size_t a = t * chunk, b = std::min(n, a + chunk);
        if (a >= b) continue;
        try {
            th.emplace_back(f, a, b);
        } catch (const std::system_error&) {
            f(a, b);   // no thread to be had: this piece on the calling thread
        }
    }
    for (auto& x : th) x.join();
}

// Stable least-significant-digit radix sort of (key, val) by key below kmax,
// 11-bit digits, each pass split over the host's cores (per-piece digit
// counts, so the scatter keeps every piece's order and the pieces' order).
static void radix_sort_stable(std::vector<uint64_t>& key, std::vector<int>& val, uint64_t kmax)
{
    const size_t m = key.size();
    const unsigned hc = std::thread::hardware_concurrency();
    const size_t T = m < 65536 ? 1 : std::min<size_t>(16, hc > 0 ? hc : 1);
    const size_t chunk = (m + T - 1) / T;
    std::vector<uint64_t> key2(m);
    std::vector<int> val2(m);
    std::vector<size_t> cnt(T * 2048);
    for (int shift = 0; shift < 64 && (kmax >> shift) > 0; shift += 11) {
        std::fill(cnt.begin(), cnt.end(), 0);
        auto count = [&](size_t t) {
            const size_t a = t * chunk, b = std::min(m, a + chunk);
            size_t* c = cnt.data() + t * 2048;
            for (size_t j = a; j < b; j++) c[(key[j] >> shift) & 2047u]++;
        };
        auto scatter = [&](size_t t) {
            const size_t a = t * chunk, b = std::min(m, a + chunk);
            size_t* c = cnt.data() + t * 2048;
            for (size_t j = a; j < b; j++) {
                const size_t o = c[(key[j] >> shift) & 2047u]++;
                key2[o] = key[j];
                val2[o] = val[j];
            }
        };
        auto run = [&](auto fn) {
            std::vector<std::thread> th;
            th.reserve(T);
            for (size_t t = 1; t < T; t++) {
                try {
                    th.emplace_back(fn, t);
                } catch (const std::system_error&) {
                    fn(t);   // no thread to be had: this piece on the calling thread
                }
            }
            fn((size_t)0);
            for (auto& x : th) x.join();
        };
        run(count);
        size_t base = 0;   // digit-major, piece-minor exclusive prefix
        for (int d = 0; d < 2048; d++)
            for (size_t t = 0; t < T; t++) {
                const size_t c = cnt[t * 2048 + d];
                cnt[t * 2048 + d] = base;
                base += c;
            }
        run(scatter);
        key.swap(key2);
        val.swap(val2);
    }
}

// Storage order of the levels; the results do not change.  Level 0 is kept
// in the mesh handle's internal order (when there are coarse levels), the
// middle levels in breadth-first order over their own graph, seeded in the
// order of each aggregate's first member in the level above (bfs), or in
// that inherited order itself, and the coarsest level in its own order.  Rows, aggregates and their lists are
// moved, never reordered inside: a row keeps its entries in face order, an
// aggregate its cells in ascending original order, so every sum is taken
// in the same order.  Afterwards: rows (rptr, rcol, rfac, rlo) of levels >= 1
// in storage order with columns at storage positions; agg maps storage
// positions to the next level's; cptr/ccell and iptr/iface follow the next
// level's storage order, with ccell at storage positions (level 0: original
// cell numbers, which index the caller's diagonal, and ccell_int at internal
// positions); faces (fptr, fface, l, u) keep their numbering.  perm0:
// internal position -> original cell of level 0.
static void gamg_store_order(std::vector<GamgHostLevel>& lv, const std::vector<int>& perm0, bool bfs)
{
    const int L = (int)lv.size();
    std::vector<std::vector<int>> pos(L), inv(L);
    for (int k = 0; k < L; k++) {
        const int n = lv[k].n;
        pos[k].assign(n, -1);
        inv[k].assign(n, 0);
        if (k == L - 1) {
            for (int i = 0; i < n; i++) pos[k][i] = inv[k][i] = i;
        } else if (k == 0) {
            for (int p = 0; p < n; p++) {
                inv[0][p] = perm0[p];
                pos[0][perm0[p]] = p;
            }
        } else if (bfs) {
            // breadth-first from each unvisited cell in the inherited order:
            // a cell's neighbours land within about one BFS front of it
            std::vector<int> seed;
            seed.reserve(n);
            std::vector<char> seen(n, 0);
            for (int q = 0; q < lv[k - 1].n; q++) {
                const int c = lv[k - 1].agg[inv[k - 1][q]];
                if (!seen[c]) {
                    seen[c] = 1;
                    seed.push_back(c);
                }
            }
            const GamgHostLevel& H = lv[k];
            int next = 0;
            for (int c0 : seed) {
                if (pos[k][c0] >= 0) continue;
                int head = next;
                pos[k][c0] = next;
                inv[k][next++] = c0;
                while (head < next) {
                    const int c = inv[k][head++];
                    for (int e = H.rptr[c]; e < H.rptr[c + 1]; e++) {
                        const int d = H.rcol[e];
                        if (pos[k][d] < 0) {
                            pos[k][d] = next;
                            inv[k][next++] = d;
                        }
                    }
                }
            }
        } else {
            int next = 0;
            for (int q = 0; q < lv[k - 1].n; q++) {
                const int c = lv[k - 1].agg[inv[k - 1][q]];
                if (pos[k][c] < 0) {
                    pos[k][c] = next;
                    inv[k][next++] = c;
                }
            }
        }
    }
    for (int k = 0; k < L; k++) {
        GamgHostLevel& H = lv[k];
        // rows: lower entries (column below the row in the original order)
        // lead each row, faces being sorted by (lower, upper); level 0's rows
        // stay in original order
        std::vector<int> rptr(H.n + 1, 0), rcol(H.rcol.size()), rfac(H.rfac.size()), rlo(H.n, 0);
        const int* I = k == 0 ? nullptr : inv[k].data();
        const int* P = k == 0 ? nullptr : pos[k].data();
        for (int q = 0; q < H.n; q++) {
            const int c = I ? I[q] : q;
            rptr[q + 1] = rptr[q] + (H.rptr[c + 1] - H.rptr[c]);
        }
        par_for((size_t)H.n, [&](size_t q0, size_t q1) {
            for (size_t q = q0; q < q1; q++) {
                const int c = I ? I[q] : (int)q;
                int o = rptr[q], lo = 0;
                for (int e = H.rptr[c]; e < H.rptr[c + 1]; e++, o++) {
                    rcol[o] = P ? P[H.rcol[e]] : H.rcol[e];
                    rfac[o] = H.rfac[e];
                    if (H.rcol[e] < c) lo++;
                }
                rlo[q] = lo;
            }
        });
        H.rptr.swap(rptr);
        H.rcol.swap(rcol);
        H.rfac.swap(rfac);
        H.rlo.swap(rlo);
        if (k + 1 >= L) continue;
        const int nc = lv[k + 1].n;
        std::vector<int> agg(H.n), cptr(nc + 1, 0), ccell(H.ccell.size()), iptr(nc + 1, 0), iface(H.iface.size()),
            ccell_int(k == 0 ? H.ccell.size() : 0);
        par_for((size_t)H.n, [&](size_t q0, size_t q1) {
            for (size_t q = q0; q < q1; q++) agg[q] = pos[k + 1][H.agg[inv[k][q]]];
        });
        for (int qc = 0; qc < nc; qc++) {
            const int c = inv[k + 1][qc];
            cptr[qc + 1] = cptr[qc] + (H.cptr[c + 1] - H.cptr[c]);
            iptr[qc + 1] = iptr[qc] + (H.iptr[c + 1] - H.iptr[c]);
        }
        par_for((size_t)nc, [&](size_t q0, size_t q1) {
            for (size_t qc = q0; qc < q1; qc++) {
                const int c = inv[k + 1][qc];
                int o = cptr[qc];
                for (int j = H.cptr[c]; j < H.cptr[c + 1]; j++, o++) {
                    const int fine = H.ccell[j];
                    ccell[o] = k == 0 ? fine : pos[k][fine];
                    if (k == 0) ccell_int[o] = pos[0][fine];
                }
                o = iptr[qc];
                for (int j = H.iptr[c]; j < H.iptr[c + 1]; j++, o++) iface[o] = H.iface[j];
            }
        });
        H.agg.swap(agg);
        H.cptr.swap(cptr);
        H.ccell.swap(ccell);
        H.iptr.swap(iptr);
        H.iface.swap(iface);
        H.ccell_int.swap(ccell_int);
    }
}

// One pairwise level; returns the next level's cell count.
static int gamg_agglomerate(const GamgHostLevel& L, const std::vector<double>& w, std::vector<int>& agg)
{
    agg.assign(L.n, -1);
    int nc = 0;
    for (int i = 0; i < L.n; i++) {
        if (agg[i] != -1) continue;
        int best = -1;
        double bw = -INFINITY;
        for (int e = L.rptr[i]; e < L.rptr[i + 1]; e++) {
            const int j = L.rcol[e], f = L.rfac[e];
            if (agg[j] == -1 && w[f] > bw) {
                best = j;
                bw = w[f];
            }
        }
        if (best >= 0) {
            agg[i] = agg[best] = nc++;
            continue;
        }
        bw = -INFINITY;
        for (int e = L.rptr[i]; e < L.rptr[i + 1]; e++) {
            const int j = L.rcol[e], f = L.rfac[e];
            if (w[f] > bw) {
                best = j;
                bw = w[f];
            }
        }
        agg[i] = best >= 0 ? agg[best] : nc++;
    }
    return nc;
}

}  // namespace spuma

using namespace spuma;

struct spuma_gamg {
    spuma_ldu_t h = nullptr;
    std::vector<GamgHostLevel> lv;
    size_t bytes = 0;
    char* ws = nullptr;
    GamgLevel* dlv = nullptr;            // device descriptors
    std::vector<GamgLevel> hlv;          // host copy of the descriptors
    double *x = nullptr, *b = nullptr, *pw = nullptr, *pp = nullptr, *pq = nullptr, *px = nullptr;
    double* crD = nullptr;
    double* partials = nullptr;
    int* ccell_int = nullptr;              // level 0's aggregate lists at internal positions (two or more levels)
    int small_from = 0;
    int smoother = 0;                      // 0 Richardson, 1 two-stage Gauss-Seidel
    int coarsest_precond = SPUMA_PRECOND_DIAGONAL;
};

namespace {

size_t gamg_layout(spuma_gamg& G, bool assign)
{
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = (off + bytes + 255) & ~(size_t)255;
        return assign ? (void*)(G.ws + o) : nullptr;
    };
    const int L = (int)G.lv.size();
    G.dlv = (GamgLevel*)take(sizeof(GamgLevel) * L);
    G.hlv.assign(L, GamgLevel{});
    for (int k = 0; k < L; k++) {
        GamgHostLevel& H = G.lv[k];
        GamgLevel& D = G.hlv[k];
        D.n = H.n;
        D.nf = H.nf;
        D.rptr = (int*)take(4 * H.rptr.size());
        D.rcol = (int*)take(4 * H.rcol.size() + 4);
        D.rfac = (int*)take(4 * H.rfac.size() + 4);
        D.rlo = (int*)take(4 * H.rlo.size() + 4);
        if (k + 1 < L) {
            D.agg = (int*)take(4 * H.agg.size() + 4);
            D.cptr = (int*)take(4 * H.cptr.size());
            D.ccell = (int*)take(4 * H.ccell.size() + 4);
            D.fptr = (int*)take(4 * H.fptr.size());
            D.fface = (int*)take(4 * H.fface.size() + 4);
            D.iptr = (int*)take(4 * H.iptr.size());
            D.iface = (int*)take(4 * H.iface.size() + 4);
        }
        if (k > 0) {
            D.diag = (double*)take(8 * (size_t)H.n + 8);
            D.upper = (double*)take(8 * (size_t)H.nf + 8);
        }
        D.wrd = (double*)take(8 * (size_t)H.n + 8);
        D.rval = (double*)take(16 * (size_t)H.nf + 8);
        D.r = (double*)take(8 * (size_t)H.n + 8);
        D.e = (double*)take(8 * (size_t)H.n + 8);
        D.q = (double*)take(8 * (size_t)H.n + 8);
        D.y = (double*)take(8 * (size_t)H.n + 8);
    }
    for (int k = 0; k + 1 < L; k++) {
        G.hlv[k].cdiag = const_cast<double*>(G.hlv[k + 1].diag);
        G.hlv[k].cupper = const_cast<double*>(G.hlv[k + 1].upper);
    }
    const size_t n0 = G.lv[0].n, nc = G.lv.back().n;
    G.x = (double*)take(8 * n0 + 8);
    G.b = (double*)take(8 * n0 + 8);
    G.pw = (double*)take(8 * nc + 8);
    G.pp = (double*)take(8 * nc + 8);
    G.pq = (double*)take(8 * nc + 8);
    G.px = (double*)take(8 * nc + 8);
    G.crD = (double*)take(8 * nc + 8);
    G.partials = (double*)take(8 * (size_t)kMaxBlocks * kSlots);
    G.ccell_int = L >= 2 ? (int*)take(4 * n0 + 4) : nullptr;
    return off;
}

}  // namespace

extern "C" {

static spuma_status gamg_create(spuma_ldu_t h, const double* face_weight, spuma_stream_t stream, spuma_gamg_t* out)
{
    if (!out) { set_error("out is NULL"); return SPUMA_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!h || (h->nf > 0 && !face_weight)) {
        set_error("spuma_gamg_create: bad argument");
        return SPUMA_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::unique_ptr<spuma_gamg> G(new spuma_gamg());
    G->h = h;
    GamgHostLevel L0;
    L0.n = h->n;
    L0.nf = h->nf;
    L0.l.resize(h->nf);
    L0.u.resize(h->nf);
    std::vector<double> w(h->nf);
    // the mesh handle's per-cell face lists (original order): neighbour-side
    // faces ascending with their lower cells, owner-side faces as a range
    std::vector<int> own_start(h->n + 1), lo_start(h->n + 1), lo_face(h->nf), lo_col(h->nf);
    cudaError_t e = cudaSuccess;
    if (h->nf > 0) {
        auto get = [&](void* dst, size_t off, size_t bytes) {
            if (e == cudaSuccess) e = cudaMemcpyAsync(dst, h->at<char>(off), bytes, cudaMemcpyDeviceToHost, s);
        };
        get(L0.l.data(), h->L.laddr, 4 * (size_t)h->nf);
        get(L0.u.data(), h->L.uaddr, 4 * (size_t)h->nf);
        get(own_start.data(), h->L.own_start, 4 * ((size_t)h->n + 1));
        get(lo_start.data(), h->L.lo_start, 4 * ((size_t)h->n + 1));
        get(lo_face.data(), h->L.lo_face, 4 * (size_t)h->nf);
        get(lo_col.data(), h->L.lo_col, 4 * (size_t)h->nf);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(w.data(), face_weight, 8 * (size_t)h->nf, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        return cuda_fail(e, "spuma_gamg_create: copy of the addressing");
    }
    // host-time breakdown of the build (SPUMA_GAMG_TIMING: printed to stderr)
    double t_rows = 0, t_agg = 0, t_faces = 0, t_lists = 0, t_order = 0;
    auto now = [] { return std::chrono::steady_clock::now(); };
    auto secs = [](std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
        return std::chrono::duration<double>(b - a).count();
    };
    auto tp = now();
    G->lv.push_back(std::move(L0));
    if (h->nf > 0) {
        // level 0's rows from those lists: the same entries, in face order, as
        // gamg_rows builds (lower entries first, faces being sorted by owner)
        GamgHostLevel& H = G->lv[0];
        H.rptr.assign(H.n + 1, 0);
        for (int i = 0; i < H.n; i++)
            H.rptr[i + 1] = H.rptr[i] + (lo_start[i + 1] - lo_start[i]) + (own_start[i + 1] - own_start[i]);
        H.rcol.resize(2 * (size_t)H.nf);
        H.rfac.resize(2 * (size_t)H.nf);
        par_for((size_t)H.n, [&](size_t i0, size_t i1) {
            for (size_t i = i0; i < i1; i++) {
                int o = H.rptr[i];
                for (int k = lo_start[i]; k < lo_start[i + 1]; k++, o++) {
                    H.rcol[o] = lo_col[k];
                    H.rfac[o] = lo_face[k];
                }
                for (int f = own_start[i]; f < own_start[i + 1]; f++, o++) {
                    H.rcol[o] = H.u[f];
                    H.rfac[o] = f;
                }
            }
        });
    } else {
        gamg_rows(G->lv[0]);
    }
    t_rows += secs(tp, now());
    while ((int)G->lv.size() < kGamgMaxLevels && G->lv.back().n > kGamgCoarsest) {
        GamgHostLevel& F = G->lv.back();
        tp = now();
        const int nc = gamg_agglomerate(F, w, F.agg);
        t_agg += secs(tp, now());
        if (nc >= F.n) break;
        tp = now();
        // coarse faces: (min, max) aggregate pairs, sorted, fine faces in
        // ascending order within each pair: a stable least-significant-digit
        // radix sort (11-bit digits) of the keys min * nc + max, taken in face
        // order (each pass streams through 2048 buckets: no random access over
        // the whole array, unlike a counting sort on the cell numbers)
        std::vector<uint64_t> key;
        std::vector<int> ord;
        {
            // the faces between different aggregates, in face order: counted
            // per piece of the face range, then written at the pieces' offsets
            const size_t P = 64, piece = ((size_t)F.nf + P - 1) / P;
            std::vector<size_t> off(P + 1, 0);
            par_for(P, [&](size_t p0, size_t p1) {
                for (size_t p = p0; p < p1; p++) {
                    size_t c = 0;
                    for (size_t f = p * piece; f < std::min((size_t)F.nf, (p + 1) * piece); f++)
                        c += F.agg[F.l[f]] != F.agg[F.u[f]];
                    off[p + 1] = c;
                }
            }, F.nf >= 65536 ? 1 : P + 1);
            for (size_t p = 0; p < P; p++) off[p + 1] += off[p];
            key.resize(off[P]);
            ord.resize(off[P]);
            par_for(P, [&](size_t p0, size_t p1) {
                for (size_t p = p0; p < p1; p++) {
                    size_t o = off[p];
                    for (size_t f = p * piece; f < std::min((size_t)F.nf, (p + 1) * piece); f++) {
                        const int a = F.agg[F.l[f]], b = F.agg[F.u[f]];
                        if (a != b) {
                            key[o] = (uint64_t)std::min(a, b) * (uint64_t)nc + (uint64_t)std::max(a, b);
                            ord[o++] = (int)f;
                        }
                    }
                }
            }, F.nf >= 65536 ? 1 : P + 1);
        }
        const size_t m = ord.size();
        radix_sort_stable(key, ord, (uint64_t)nc * (uint64_t)nc);
        // (key, ord) sorted by (min, max), ties in face order
        // runs of equal keys are the coarse faces; each one's weight is the
        // sum of its fine faces' weights in face order (runs in parallel)
        GamgHostLevel C;
        C.n = nc;
        F.fptr.clear();
        for (size_t j = 0; j < m; j++)
            if (j == 0 || key[j] != key[j - 1]) F.fptr.push_back((int)j);
        F.fptr.push_back((int)m);
        const size_t ncf = F.fptr.size() - 1;
        C.l.resize(ncf);
        C.u.resize(ncf);
        std::vector<double> wc(ncf);
        par_for(ncf, [&](size_t g0, size_t g1) {
            for (size_t g = g0; g < g1; g++) {
                const uint64_t kk = key[F.fptr[g]];
                C.l[g] = (int)(kk / (uint64_t)nc);
                C.u[g] = (int)(kk % (uint64_t)nc);
                double sum = 0.0;
                for (int j = F.fptr[g]; j < F.fptr[g + 1]; j++) sum += w[ord[j]];
                wc[g] = sum;
            }
        });
        F.fface.swap(ord);
        C.nf = (int)C.l.size();
        t_faces += secs(tp, now());
        tp = now();
        // next-level cell -> cells, -> faces inside it (ascending)
        F.cptr.assign(nc + 1, 0);
        for (int i = 0; i < F.n; i++) F.cptr[F.agg[i] + 1]++;
        for (int c = 0; c < nc; c++) F.cptr[c + 1] += F.cptr[c];
        F.ccell.resize(F.n);
        std::vector<int> cur(F.cptr.begin(), F.cptr.end() - 1);
        for (int i = 0; i < F.n; i++) F.ccell[cur[F.agg[i]]++] = i;
        F.iptr.assign(nc + 1, 0);
        for (int f = 0; f < F.nf; f++)
            if (F.agg[F.l[f]] == F.agg[F.u[f]]) F.iptr[F.agg[F.l[f]] + 1]++;
        for (int c = 0; c < nc; c++) F.iptr[c + 1] += F.iptr[c];
        F.iface.resize(F.iptr[nc]);
        cur.assign(F.iptr.begin(), F.iptr.end() - 1);
        for (int f = 0; f < F.nf; f++)
            if (F.agg[F.l[f]] == F.agg[F.u[f]]) F.iface[cur[F.agg[F.l[f]]]++] = f;
        t_lists += secs(tp, now());
        tp = now();
        gamg_rows(C);
        t_rows += secs(tp, now());
        G->lv.push_back(std::move(C));
        w.swap(wc);
    }
    std::vector<int> perm0;
    if (G->lv.size() >= 2) {
        perm0.resize(h->n);
        e = cudaMemcpyAsync(perm0.data(), h->at<int>(h->L.perm), 4 * (size_t)h->n, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
                return cuda_fail(e, "spuma_gamg_create: copy of the cell order");
        }
    }
    // storage order of the middle levels: breadth-first (default) or
    // inherited from the level above (SPUMA_GAMG_ORDER=inherited, a
    // measurement override)
    const char* ord = getenv("SPUMA_GAMG_ORDER");
    tp = now();
    gamg_store_order(G->lv, perm0, !(ord && std::string(ord) == "inherited"));
    t_order += secs(tp, now());
    if (getenv("SPUMA_GAMG_TIMING"))
        fprintf(stderr, "spuma_gamg_create host seconds: rows %.3f agglomerate %.3f coarse faces %.3f lists %.3f "
                "storage order %.3f\n", t_rows, t_agg, t_faces, t_lists, t_order);
    G->bytes = gamg_layout(*G, false);
    G->small_from = (int)G->lv.size();
    for (int k = 0; k < (int)G->lv.size(); k++)
        if (G->lv[k].n <= 2048) {
            G->small_from = k;
            break;
        }
    *out = G.release();
    return SPUMA_OK;
}

// No C++ exception crosses the C interface: a host allocation or thread
// that fails while the hierarchy is built returns SPUMA_ERR_HOST.
spuma_status spuma_gamg_create(spuma_ldu_t h, const double* face_weight, spuma_stream_t stream, spuma_gamg_t* out)
{
    return host_guard("spuma_gamg_create", [&] { return gamg_create(h, face_weight, stream, out); });
}

size_t spuma_gamg_workspace_bytes(spuma_gamg_t g) { return g ? g->bytes : 0; }

spuma_status spuma_gamg_bind(spuma_gamg_t g, void* workspace, size_t workspace_bytes, spuma_stream_t stream)
{
    if (!g || !workspace || ((uintptr_t)workspace & 255u) != 0) {
        set_error("spuma_gamg_bind: bad argument (workspace must be 256-byte aligned)");
        return SPUMA_ERR_INVALID_ARG;
    }
    if (workspace_bytes < g->bytes) {
        set_error("spuma_gamg_bind: workspace needs " + std::to_string(g->bytes) + " bytes");
        return SPUMA_ERR_WORKSPACE_TOO_SMALL;
    }
    g->ws = (char*)workspace;
    gamg_layout(*g, true);
    cudaStream_t s = (cudaStream_t)stream;
    auto up = [&](const void* dst, const std::vector<int>& v) {
        return v.empty() ? cudaSuccess
                         : cudaMemcpyAsync((void*)dst, v.data(), 4 * v.size(), cudaMemcpyHostToDevice, s);
    };
    for (size_t k = 0; k < g->lv.size(); k++) {
        const GamgHostLevel& H = g->lv[k];
        const GamgLevel& D = g->hlv[k];
        SPUMA_CUDA(up(D.rptr, H.rptr));
        SPUMA_CUDA(up(D.rcol, H.rcol));
        SPUMA_CUDA(up(D.rfac, H.rfac));
        SPUMA_CUDA(up(D.rlo, H.rlo));
        if (k + 1 < g->lv.size()) {
            SPUMA_CUDA(up(D.agg, H.agg));
            SPUMA_CUDA(up(D.cptr, H.cptr));
            SPUMA_CUDA(up(D.ccell, H.ccell));
            SPUMA_CUDA(up(D.fptr, H.fptr));
            SPUMA_CUDA(up(D.fface, H.fface));
            SPUMA_CUDA(up(D.iptr, H.iptr));
            SPUMA_CUDA(up(D.iface, H.iface));
        }
    }
    if (g->ccell_int) SPUMA_CUDA(up(g->ccell_int, g->lv[0].ccell_int));
    SPUMA_CUDA(cudaStreamSynchronize(s));
    return SPUMA_OK;
}

spuma_status spuma_gamg_info(spuma_gamg_t g, int32_t* n_levels, int32_t* level_cells, int32_t max_levels)
{
    if (!g) { set_error("spuma_gamg_info: handle is NULL"); return SPUMA_ERR_INVALID_ARG; }
    if (n_levels) *n_levels = (int32_t)g->lv.size();
    if (level_cells)
        for (int k = 0; k < (int)g->lv.size() && k < max_levels; k++) level_cells[k] = g->lv[k].n;
    return SPUMA_OK;
}

spuma_status spuma_gamg_solve(spuma_gamg_t g, const double* diag, const double* upper, const double* b, double* x,
                              const spuma_solver_controls* ctl, spuma_solver_perf* perf, spuma_stream_t stream)
{
    if (!g || !g->ws || !ctl || !(ctl->tolerance >= 0.0) || !(ctl->rel_tol >= 0.0) || ctl->max_iter < 0 ||
        ctl->min_iter < 0 || ctl->precision != SPUMA_F64 || (g->h->n > 0 && (!diag || !b || !x)) ||
        (g->h->nf > 0 && !upper)) {
        set_error("spuma_gamg_solve: bad argument (bound solver, precision F64)");
        return SPUMA_ERR_INVALID_ARG;
    }
    spuma_ldu_t h = g->h;
    cudaStream_t s = (cudaStream_t)stream;
    if (h->n == 0) {
        if (perf) {
            spuma_solver_perf z{};
            z.converged = 1;
            SPUMA_CUDA(cudaMemcpyAsync(perf, &z, sizeof(z), cudaMemcpyHostToDevice, s));
        }
        return SPUMA_OK;
    }
    g->hlv[0].diag = diag;
    g->hlv[0].upper = upper;
    SPUMA_CUDA(cudaMemcpyAsync(g->dlv, g->hlv.data(), sizeof(GamgLevel) * g->hlv.size(), cudaMemcpyHostToDevice, s));
    GamgArgs a{};
    a.nlev = (int)g->lv.size();
    a.small_from = g->small_from;
    a.lv = g->dlv;
    a.b_orig = b;
    a.x_orig = x;
    a.x = g->x;
    a.b = g->b;
    a.res = g->hlv[0].r;
    a.pw = g->pw;
    a.pp = g->pp;
    a.pq = g->pq;
    a.px = g->px;
    a.crD = g->crD;
    a.smoother = g->smoother;
    a.coarsest_precond = g->coarsest_precond;
    a.partials = g->partials;
    if (g->ccell_int) {
        // level 0 in internal order; its coefficients overwrite the handle's
        // matrix region, so the next PCG solve prepares its matrix again
        GamgLvl0& z = a.z;
        z.on = 1;
        z.n = h->n;
        z.ell_w = h->ell_w;
        z.perm = h->at<int>(h->L.perm);
        z.Lptr = h->at<int>(h->L.Lptr);
        z.Lcol = h->at<int>(h->L.Lcol);
        z.Lface = h->at<int>(h->L.Lface);
        z.Uptr = h->at<int>(h->L.Uptr);
        z.Ucol = h->at<int>(h->L.Ucol);
        z.Uface = h->at<int>(h->L.Uface);
        z.Ecol = h->at<int>(h->L.Ecol);
        z.La = h->at<double>(h->L.La64);
        z.Ua = h->at<double>(h->L.Ua64);
        z.d = h->at<double>(h->L.d64);
        z.Ea = h->at<double>(h->L.Ea64);
        z.ccell_int = g->ccell_int;
        h->prepared_precond = -1;
    }
    a.status = h->at<int>(h->L.status);
    {
        // measured at 200^3 with 262144: the levels it covers 1-8 % slower
        static const int fuse_env = getenv("SPUMA_GAMG_FUSE_SCALE_ROWS") ? atoi(getenv("SPUMA_GAMG_FUSE_SCALE_ROWS")) : 0;
        a.fuse_rows = fuse_env;
    }
    a.clk = nullptr;
    if (getenv("SPUMA_PHASE_CLOCKS")) {
        a.clk = h->at<long long>(h->L.clk);
        SPUMA_CUDA(cudaMemsetAsync(a.clk, 0, 8 * 256, s));
    }
    a.perf = perf;
    a.max_iter = ctl->max_iter;
    a.min_iter = ctl->min_iter;
    a.tol = ctl->tolerance;
    a.rel_tol = ctl->rel_tol;
    int per_sm = 0;
    SPUMA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gamg, 1024, 0));
    if (per_sm < 1) { set_error("GAMG kernel cannot be resident"); return SPUMA_ERR_CUDA; }
    const int64_t want = ((int64_t)h->n + 1023) / 1024;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, std::min<int64_t>((int64_t)per_sm * h->num_sms,
                                                                                          kMaxBlocks)));
    SPUMA_CUDA(cudaMemsetAsync(h->at<char>(h->L.bar), 0, h->L.status + 256 - h->L.bar, s));
    unsigned long long tns = barrier_timeout_ns();
    void* args[] = {(void*)&a, (void*)&tns};
    SPUMA_CUDA(cudaLaunchCooperativeKernel((const void*)k_gamg, grid, 1024, args, 0, s));
    count_launch();
    return SPUMA_OK;
}

spuma_status spuma_gamg_set_options(spuma_gamg_t g, int32_t smoother, int32_t coarsest_precond)
{
    if (!g || (smoother != SPUMA_GAMG_RICHARDSON && smoother != SPUMA_GAMG_GAUSS_SEIDEL_2STAGE) ||
        (coarsest_precond != SPUMA_PRECOND_DIAGONAL && coarsest_precond != SPUMA_PRECOND_DIC)) {
        set_error("spuma_gamg_set_options: bad argument (smoother 0 or 1, coarsest preconditioner DIAGONAL or DIC)");
        return SPUMA_ERR_INVALID_ARG;
    }
    g->smoother = smoother;
    g->coarsest_precond = coarsest_precond;
    return SPUMA_OK;
}

spuma_status spuma_gamg_destroy(spuma_gamg_t g)
{
    delete g;
    return SPUMA_OK;
}

}  // extern "C"
