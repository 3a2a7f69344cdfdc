// solve.cu -- the persistent PCG solver (FP64, and mixed FP32/FP64 by reliable
// updates or restarted refinement), the level-scheduled DIC factor and sweeps,
// the prepared-matrix Amul, and their host entry points.
//
// One cooperative launch per solve.  Rows live in the handle's level order:
// level L (rows whose longest chain of lower neighbours has length L) is the
// contiguous range lvl[L]..lvl[L+1], and every row keeps its neighbour-side
// ("lower") and owner-side ("upper") entries in ascending face order, so each
// row sum is taken in exactly the order of the sequential face loop.
//
// One PCG iteration with DIC (grid barriers after each step, and after each
// DIC level inside the sweeps):
//   update pass       x += alpha p, r -= alpha q, sum|r|       -> converged?
//   forward sweep     w = (P + L)^-1 r, level by level
//   backward sweep    w = (P + U)^-1 P w, rho = w.r            -> beta
//   search direction  p = w + beta p
//   Amul              q = A p, sigma = q.p                     -> alpha
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>

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
    return Mat<double>{a.Lptr, a.Lcol, a.La64, a.Lc64, a.Uptr, a.Ucol, a.Ua64, a.Uc64, a.d64, a.rD64,
                       a.Ecol, a.Ea64, a.ell_w, a.n};
}
template <>
__device__ __forceinline__ Mat<float> mat_of<float>(const SolveArgs& a)
{
    return Mat<float>{a.Lptr, a.Lcol, a.La32, a.Lc32, a.Uptr, a.Ucol, a.Ua32, a.Uc32, a.d32, a.rD32,
                      a.Ecol, a.Ea32, a.ell_w, a.n};
}

// Cache priorities.  The matrix streams (entries, row extents, diagonal,
// rD) are read once per pass: they are loaded evict-first (__ldcs), so that
// the vectors other rows gather stay in L2; a stand-alone Amul stores its
// result evict-first too.  Inside the solver, FP32 gathers (x in the Amul, w
// in the sweeps) are loaded evict-last on top of that, and the solver hands
// those lines back (evict-normal) before it returns; FP64 vectors, twice the
// size, keep the default priority, since pinning them evicts them from each
// other.  Measured at 200^3: stand-alone Amul FP64 168 -> 130 us, FP32
// 101 -> 91 us; mixed solve 352 -> 333 ms with evict-first streams, 330 ms
// with the FP32 gathers evict-last (FP64 gathers evict-last: Amul 130 -> 146 us).
template <class T, bool KEEP>
__device__ __forceinline__ unsigned long long keep_policy()
{
    unsigned long long p = 0;
    if constexpr (KEEP && sizeof(T) == 4)
        asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
template <bool KEEP>
__device__ __forceinline__ float gather(const float* v, int c, unsigned long long pol)
{
    if constexpr (KEEP) {
        float r;
        asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(r) : "l"(v + c), "l"(pol) : "memory");
        return r;
    } else {
        return v[c];
    }
}
template <bool KEEP>
__device__ __forceinline__ double gather(const double* v, int c, unsigned long long)
{
    return v[c];
}

// Back to evict-normal: every 128-byte line of [base, base + bytes), spread
// over the group's threads (a hint; the regions are 256-byte aligned).
__device__ __forceinline__ void release_lines(const void* base, size_t bytes, int first, int stride)
{
    const char* b = static_cast<const char*>(base);
    for (size_t off = (size_t)first * 128; off < bytes; off += (size_t)stride * 128)
        asm volatile("applypriority.global.L2::evict_normal [%0], 128;" : : "l"(b + off) : "memory");
}

// Shapes of the row chains: a row's entries are taken in groups whose column
// and coefficient loads are issued together, then the gathers, then the FMAs
// in entry order (two memory round trips per group, not per entry).  FP64 rows
// run one per thread, FP32 rows two per thread in lockstep.  Groups of 6 in
// the DIC sweeps (a hex-mesh row has at most 6 entries on either side) and in
// the Amul, which takes a row's lower and upper entries as one list (a whole
// hex-mesh row in one group).  Chosen by measurement on the 200^3 workload.
template <class T>
struct ChainShape {
    static constexpr int R = sizeof(T) == 4 ? 2 : 1;
    static constexpr int G = 6;
};
// Software-pipelined fixed-width Amul: R rows per round, whole rows of up to
// G entries.  Where it is used was decided by measurement at 200^3: inside
// the persistent solver for FP64 (219 -> 200 us per Amul; FP32 keeps its two
// rows per thread in lockstep, 112 against 131 us pipelined), and in the
// stand-alone prepared Amul for FP32 (107 -> 101 us; FP64 168 against 176 us).
template <class T>
struct PipeShape {
    static constexpr int R = 1;
    static constexpr int G = 6;
    static constexpr bool in_solver = sizeof(T) == 8;
    static constexpr bool stand_alone = sizeof(T) == 4;
};
template <class T>
struct AmulShape {
    static constexpr int R = sizeof(T) == 4 ? 2 : 1;
    static constexpr int G = 6;
};

// R rows' chains in lockstep; each row takes its entries [e0, e1) in its own
// order (DESC: from e1-1 down to e0).
template <class T, int R, int G, bool DESC, bool NEG>
__device__ __forceinline__ void rows_chain(T (&acc)[R], const int (&e0)[R], const int (&e1)[R], const int* col,
                                           const T* coef, const T* vec)
{
    const unsigned long long pol = keep_policy<T, true>();
    for (int off = 0;; off += G) {
        bool more = false;
#pragma unroll
        for (int k = 0; k < R; k++) more |= e0[k] + off < e1[k];
        if (!more) break;
        int c[R][G];
        T cf[R][G], v[R][G];
#pragma unroll
        for (int k = 0; k < R; k++)
#pragma unroll
            for (int j = 0; j < G; j++) {
                const int ej = DESC ? e1[k] - 1 - off - j : e0[k] + off + j;
                const bool ok = DESC ? ej >= e0[k] : ej < e1[k];
                c[k][j] = ok ? __ldcs(col + ej) : -1;
                cf[k][j] = ok ? __ldcs(coef + ej) : T(0);
            }
#pragma unroll
        for (int k = 0; k < R; k++)
#pragma unroll
            for (int j = 0; j < G; j++) v[k][j] = c[k][j] >= 0 ? gather<true>(vec, c[k][j], pol) : T(0);
#pragma unroll
        for (int k = 0; k < R; k++)
#pragma unroll
            for (int j = 0; j < G; j++)
                if (c[k][j] >= 0) acc[k] = fmadd(NEG ? -cf[k][j] : cf[k][j], v[k][j], acc[k]);
    }
}

// y = A x for R rows: d_p x_p, then the row's lower entries (ascending face)
// and upper entries (ascending face) taken as one list of nL + nU entries.
// KEEP: gathers of x evict-last (inside the solver, FP32).
template <class T, int R, int G, bool KEEP = true>
__device__ __forceinline__ void amul_rows(const Mat<T>& A, const T* x, const int (&p)[R], int n, T (&y)[R],
                                          T (&xp)[R])
{
    if (A.ell_w > 0) {
        // fixed-width layout: no row extents to load, entries coalesced
        const unsigned long long pol = keep_policy<T, KEEP>();
#pragma unroll
        for (int k = 0; k < R; k++) {
            const bool ok = p[k] < n;
            xp[k] = ok ? x[p[k]] : T(0);
            y[k] = ok ? mul_rn(__ldcs(A.d + p[k]), xp[k]) : T(0);
        }
        for (int j0 = 0; j0 < A.ell_w; j0 += G) {
            int c[R][G];
            T cf[R][G], vv[R][G];
#pragma unroll
            for (int k = 0; k < R; k++)
#pragma unroll
                for (int j = 0; j < G; j++) {
                    const bool ok = p[k] < n && j0 + j < A.ell_w;
                    const size_t e = (size_t)(j0 + j) * A.ell_stride + p[k];
                    c[k][j] = ok ? __ldcs(A.Ecol + e) : -1;
                    cf[k][j] = ok ? __ldcs(A.Ea + e) : T(0);
                }
#pragma unroll
            for (int k = 0; k < R; k++)
#pragma unroll
                for (int j = 0; j < G; j++) vv[k][j] = c[k][j] >= 0 ? gather<KEEP>(x, c[k][j], pol) : T(0);
#pragma unroll
            for (int k = 0; k < R; k++)
#pragma unroll
                for (int j = 0; j < G; j++)
                    if (c[k][j] >= 0) y[k] = fmadd(cf[k][j], vv[k][j], y[k]);
        }
        return;
    }
    const unsigned long long pol = keep_policy<T, KEEP>();
    int l0[R], nl[R], u0[R], nt[R];
#pragma unroll
    for (int k = 0; k < R; k++) {
        const bool ok = p[k] < n;
        l0[k] = ok ? __ldcs(A.Lptr + p[k]) : 0;
        nl[k] = ok ? __ldcs(A.Lptr + p[k] + 1) - l0[k] : 0;
        u0[k] = ok ? __ldcs(A.Uptr + p[k]) : 0;
        nt[k] = ok ? nl[k] + __ldcs(A.Uptr + p[k] + 1) - u0[k] : 0;
        xp[k] = ok ? x[p[k]] : T(0);
        y[k] = ok ? mul_rn(__ldcs(A.d + p[k]), xp[k]) : T(0);
    }
    for (int off = 0;; off += G) {
        bool more = false;
#pragma unroll
        for (int k = 0; k < R; k++) more |= off < nt[k];
        if (!more) break;
        int c[R][G];
        T cf[R][G], vv[R][G];
#pragma unroll
        for (int k = 0; k < R; k++)
#pragma unroll
            for (int j = 0; j < G; j++) {
                const int kk = off + j;
                const bool low = kk < nl[k];
                const int e = low ? l0[k] + kk : u0[k] + (kk - nl[k]);
                const bool ok = kk < nt[k];
                c[k][j] = ok ? __ldcs((low ? A.Lcol : A.Ucol) + e) : -1;
                cf[k][j] = ok ? __ldcs((low ? A.La : A.Ua) + e) : T(0);
            }
#pragma unroll
        for (int k = 0; k < R; k++)
#pragma unroll
            for (int j = 0; j < G; j++) vv[k][j] = c[k][j] >= 0 ? gather<KEEP>(x, c[k][j], pol) : T(0);
#pragma unroll
        for (int k = 0; k < R; k++)
#pragma unroll
            for (int j = 0; j < G; j++)
                if (c[k][j] >= 0) y[k] = fmadd(cf[k][j], vv[k][j], y[k]);
    }
}

// Fixed-width Amul rows, software-pipelined: the loads of a round (entries,
// x_p, d_p: none depends on an earlier result) are issued before the
// previous round's gathers, so each round costs about one memory round trip
// instead of two.  For rows of at most G entries (a whole row per round).
template <class T, int R, int G>
struct EllRound {
    int c[R][G];
    T a[R][G];
    T xp[R], d[R];
};

template <class T, int R, int G>
__device__ __forceinline__ void ell_load(EllRound<T, R, G>& e, const Mat<T>& A, const T* x, int pb, int stride, int n)
{
#pragma unroll
    for (int k = 0; k < R; k++) {
        const int p = pb + k * stride;
        const bool ok = p < n;
        e.xp[k] = ok ? x[p] : T(0);
        e.d[k] = ok ? __ldcs(A.d + p) : T(0);
#pragma unroll
        for (int j = 0; j < G; j++) {
            const bool okj = ok && j < A.ell_w;
            const size_t idx = (size_t)j * A.ell_stride + p;
            e.c[k][j] = okj ? __ldcs(A.Ecol + idx) : -1;
            e.a[k][j] = okj ? __ldcs(A.Ea + idx) : T(0);
        }
    }
}

template <class T, int R, int G>
__device__ __forceinline__ void ell_finish(const EllRound<T, R, G>& e, const Mat<T>& A, const T* x, T (&y)[R])
{
    T vv[R][G];
#pragma unroll
    for (int k = 0; k < R; k++)
#pragma unroll
        for (int j = 0; j < G; j++) vv[k][j] = e.c[k][j] >= 0 ? gather<false>(x, e.c[k][j], 0) : T(0);
#pragma unroll
    for (int k = 0; k < R; k++) {
        y[k] = mul_rn(e.d[k], e.xp[k]);
#pragma unroll
        for (int j = 0; j < G; j++)
            if (e.c[k][j] >= 0) y[k] = fmadd(e.a[k][j], vv[k][j], y[k]);
    }
}

// q = A x over rows first + j stride (j = 0, 1, ...) below n; the sink gets
// (row, q_row, x_row) of every row.
template <class T, int R, int G, class Sink>
__device__ __forceinline__ void ell_amul_pipelined(const Mat<T>& A, const T* x, int first, int stride, int n,
                                                   Sink sink)
{
    EllRound<T, R, G> cur, nxt;
    ell_load<T, R, G>(cur, A, x, first, stride, n);
    for (int pb = first; pb < n; pb += R * stride) {
        const int pn = pb + R * stride;
        if (pn < n) ell_load<T, R, G>(nxt, A, x, pn, stride, n);
        T y[R];
        ell_finish<T, R, G>(cur, A, x, y);
#pragma unroll
        for (int k = 0; k < R; k++)
            if (pb + k * stride < n) sink(pb + k * stride, y[k], cur.xp[k]);
        cur = nxt;
    }
}

template <class T>
__device__ __forceinline__ T amul_row(const Mat<T>& A, const T* x, int p)
{
    int pp[1] = {p};
    T y[1], xp[1];
    amul_rows<T, 1, AmulShape<T>::G>(A, x, pp, p + 1, y, xp);
    return y[0];
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

// Optional phase timing: group block 0, thread 0 adds SM-clock deltas between
// consecutive marks into phase_clk[slot] (slots: 0..63 forward level, 64..127
// backward level, 128 search direction, 129 Amul + sigma, 130 diagonal pass,
// 132 FP64 refinement residual, 134 update pass, 140 iterations).
enum ClkSlot { CK_FWD = 0, CK_BWD = 64, CK_PUPD = 128, CK_AMUL = 129, CK_DIAG = 130, CK_RESID = 132,
               CK_UPD = 134, CK_ITERS = 140 };

__device__ __forceinline__ long long sm_clock()
{
    long long t;
    asm volatile("mov.u64 %0, %%clock64;" : "=l"(t));
    return t;
}

struct PhaseClock {
    long long* acc;
    long long t;
    __device__ __forceinline__ PhaseClock(long long* a, int bid)
    {
        acc = (a && bid == 0 && threadIdx.x == 0) ? a : nullptr;
        t = sm_clock();
    }
    __device__ __forceinline__ void lap(int slot)
    {
        if (acc) {
            const long long now = sm_clock();
            acc[slot] += now - t;
            t = now;
        }
    }
    __device__ __forceinline__ void count(int slot)
    {
        if (acc) acc[slot] += 1;
    }
};

// Per-thread reduction accumulators.  FP64: fused multiply-add into a double.
// FP32 data: the exact product (a*b, fma(a, b, -a*b)) is added to a
// double-float (hi, lo) pair by Knuth's two-sum, so the sum keeps ~48 bits
// without converting every element to double; the pair is converted once.
template <class T>
struct Acc;
template <>
struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void prod(double a, double b) { s = __fma_rn(a, b, s); }
    __device__ __forceinline__ void add(double a) { s = __dadd_rn(s, a); }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct Acc<float> {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add2(float p, float e)
    {
        const float sum = __fadd_rn(hi, p);
        const float bb = __fsub_rn(sum, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(sum, bb)), __fsub_rn(p, bb));
        hi = sum;
        lo = __fadd_rn(lo, __fadd_rn(err, e));
    }
    __device__ __forceinline__ void prod(float a, float b)
    {
        const float p = __fmul_rn(a, b);
        add2(p, __fmaf_rn(a, b, -p));
    }
    __device__ __forceinline__ void add(float a) { add2(a, 0.0f); }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// 16-byte vector of the working precision (float4 / double2): the streaming
// passes move 16 bytes per load so that enough bytes are in flight per SM.
template <class T>
struct V16;
template <>
struct V16<float> {
    using type = float4;
    static constexpr int n = 4;
};
template <>
struct V16<double> {
    using type = double2;
    static constexpr int n = 2;
};
__device__ __forceinline__ float4 vfma(float a, float4 x, float4 y)
{
    return make_float4(__fmaf_rn(a, x.x, y.x), __fmaf_rn(a, x.y, y.y), __fmaf_rn(a, x.z, y.z), __fmaf_rn(a, x.w, y.w));
}
__device__ __forceinline__ double2 vfma(double a, double2 x, double2 y)
{
    return make_double2(__fma_rn(a, x.x, y.x), __fma_rn(a, x.y, y.y));
}
template <class A>
__device__ __forceinline__ void vadd_abs(A& acc, float4 r)
{
    acc.add(fabsf(r.x));
    acc.add(fabsf(r.y));
    acc.add(fabsf(r.z));
    acc.add(fabsf(r.w));
}
template <class A>
__device__ __forceinline__ void vadd_abs(A& acc, double2 r)
{
    acc.add(fabs(r.x));
    acc.add(fabs(r.y));
}
// ------------------------------------------------------------ phases --------
__device__ __forceinline__ void gather_symmetric(const SolveArgs& a, const RowIter& it, bool& bad);

// Gather the LDU coefficients into the internal layout (+ FP32 copies).
template <bool ASYM>
__device__ bool phase_gather(const SolveArgs& a, const Group& g)
{
    RowIter it = rows_of(g);
    bool bad = false;
    if constexpr (ASYM) {
        // asymmetric: row u's lower entry of face f holds lower_f (A) and
        // upper_f (A^T), row l's upper entry upper_f (A) and lower_f (A^T)
        for (int e = it.first; e < a.nf; e += it.stride) {
            const int fl = a.Lface[e], fu = a.Uface[e];
            const double lo = a.lower_orig[fl], lt = a.upper_orig[fl];
            const double up = a.upper_orig[fu], ut = a.lower_orig[fu];
            a.La64[e] = lo;
            a.LaT64[e] = lt;
            a.Ua64[e] = up;
            a.UaT64[e] = ut;
            bad |= !isfinite(lo) || !isfinite(lt);
        }
        for (int p = it.first; p < a.n; p += it.stride) {
            const double dv = a.diag_orig[a.perm[p]];
            a.d64[p] = dv;
            bad |= !isfinite(dv);
            if (a.ell_w > 0) {
                // fixed-width layout: A (lower_f in row u, upper_f in row l) and A^T
                const int l0 = a.Lptr[p], nl = a.Lptr[p + 1] - l0, u0 = a.Uptr[p], nt = nl + a.Uptr[p + 1] - u0;
                for (int j = 0; j < a.ell_w; j++) {
                    double v = 0.0, vt = 0.0;
                    if (j < nl) {
                        const int f = a.Lface[l0 + j];
                        v = a.lower_orig[f];
                        vt = a.upper_orig[f];
                    } else if (j < nt) {
                        const int f = a.Uface[u0 + j - nl];
                        v = a.upper_orig[f];
                        vt = a.lower_orig[f];
                    }
                    a.Ea64[(size_t)j * a.n + p] = v;
                    a.EaT64[(size_t)j * a.n + p] = vt;
                }
            }
        }
    } else {
        gather_symmetric(a, it, bad);
    }
    if (bad) flag_error(a.status, SPUMA_ERR_NONFINITE, -1);
    return group_sync(g);
}

// Symmetric gather: a_f into the internal CSR (+ FP32 copies), the diagonal,
// and the fixed-width Amul layout's coefficients.
__device__ __forceinline__ void gather_symmetric(const SolveArgs& a, const RowIter& it, bool& bad)
{
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
        if (a.ell_w > 0) {
            const int l0 = a.Lptr[p], nl = a.Lptr[p + 1] - l0, u0 = a.Uptr[p], nt = nl + a.Uptr[p + 1] - u0;
            for (int j = 0; j < a.ell_w; j++) {
                const double v = j < nl ? a.upper_orig[a.Lface[l0 + j]]
                                        : (j < nt ? a.upper_orig[a.Uface[u0 + j - nl]] : 0.0);
                a.Ea64[(size_t)j * a.n + p] = v;
                a.Ea32[(size_t)j * a.n + p] = (float)v;
            }
        }
    }
}

// DIC pivots level by level: p_i = d_i - sum_{lower entries} (a a)/p_col,
// then rD = 1/p and the sweep coefficients rD_row * a (+ FP32 copies).
// Diagonal: rD = 1/d.
template <bool ASYM>
__device__ bool phase_factor(const SolveArgs& a, const Group& g)
{
    RowIter it = rows_of(g);
    if (ASYM && a.precond == SPUMA_PRECOND_DILU) {
        // DILU pivots, level by level: p_u -= (upper_f lower_f) / p_l in face order
        for (int L = 0; L < a.nlev; L++) {
            const int r0 = a.lvl[L], r1 = a.lvl[L + 1];
            for (int p = r0 + it.first; p < r1; p += it.stride) {
                double piv = a.d64[p];
                for (int e = a.Lptr[p]; e < a.Lptr[p + 1]; e++)
                    piv = __dsub_rn(piv, __ddiv_rn(__dmul_rn(a.LaT64[e], a.La64[e]), a.rD64[a.Lcol[e]]));
                a.rD64[p] = piv;
                if (!(piv != 0.0 && isfinite(piv))) flag_error(a.status, SPUMA_ERR_SINGULAR, a.perm[p]);
            }
            if (!group_sync(g)) return false;
        }
        for (int p = it.first; p < a.n; p += it.stride) {
            const double rd = __ddiv_rn(1.0, a.rD64[p]);
            a.rD64[p] = rd;
            for (int e = a.Lptr[p]; e < a.Lptr[p + 1]; e++) {
                a.Lc64[e] = __dmul_rn(rd, a.La64[e]);
                a.LcT64[e] = __dmul_rn(rd, a.LaT64[e]);
            }
            for (int e = a.Uptr[p]; e < a.Uptr[p + 1]; e++) {
                a.Uc64[e] = __dmul_rn(rd, a.Ua64[e]);
                a.UcT64[e] = __dmul_rn(rd, a.UaT64[e]);
            }
        }
        return group_sync(g);
    }
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
        if (a.precond == SPUMA_PRECOND_DIC) {
            rd = __ddiv_rn(1.0, a.rD64[p]);
        } else if (a.precond == SPUMA_PRECOND_DIAGONAL) {
            rd = __ddiv_rn(1.0, a.d64[p]);
        } else {
            rd = 1.0;
        }
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

// ------------------------------------------------------ DIC sweeps ---------
// What the sweeps' reduction takes: rho = w.r (PCG), rho = w.dotv with a
// vector of the caller's (PBiCG: wA.rT), or nothing (PBiCG's M^-T apply).
// A template argument, so that the PCG kernels keep their own code.
enum RhoWith { RHO_R = 0, RHO_VEC = 1, RHO_NONE = 2 };

// Forward rows of one level: w = rD r - sum (rD a) w_lower (ascending face
// order); with `rho` (top level: no upper neighbours, so w is final here)
// also rho += w r (or w dotv).
template <class T, int RW>
__device__ __forceinline__ void fwd_rows(const Mat<T>& A, Vecs<T> v, int r0, int r1, int first, int stride, bool rho,
                                         const T* dotv, Acc<T>& arho)
{
    constexpr int R = ChainShape<T>::R, G = ChainShape<T>::G;
    for (int pb = r0 + first; pb < r1; pb += R * stride) {
        int p[R], e0[R], e1[R];
        bool ok[R];
        T ww[R], rr[R];
#pragma unroll
        for (int k = 0; k < R; k++) {
            p[k] = pb + k * stride;
            ok[k] = p[k] < r1;
            e0[k] = ok[k] ? __ldcs(A.Lptr + p[k]) : 0;
            e1[k] = ok[k] ? __ldcs(A.Lptr + p[k] + 1) : 0;
            rr[k] = ok[k] ? v.r[p[k]] : T(0);
            ww[k] = ok[k] ? mul_rn(__ldcs(A.rD + p[k]), rr[k]) : T(0);
        }
        rows_chain<T, R, G, false, true>(ww, e0, e1, A.Lcol, A.Lc, v.w);
#pragma unroll
        for (int k = 0; k < R; k++)
            if (ok[k]) {
                v.w[p[k]] = ww[k];
                if (RW != RHO_NONE && rho) arho.prod(ww[k], RW == RHO_R ? rr[k] : dotv[p[k]]);
            }
    }
}

// Backward rows of one level: w -= sum (rD a) w_upper (descending face
// order); rho += w r (or w dotv).
template <class T, int RW>
__device__ __forceinline__ void bwd_rows(const Mat<T>& A, Vecs<T> v, int r0, int r1, int first, int stride,
                                         const T* dotv, Acc<T>& arho)
{
    constexpr int R = ChainShape<T>::R, G = ChainShape<T>::G;
    // row extents one round ahead: the next round's are loaded while this
    // round's entries and gathers are in flight (measured: backward sweep
    // 135 -> 128 us per FP32 iteration at 200^3; no gain in the forward one)
    int e0n[R], e1n[R];
#pragma unroll
    for (int k = 0; k < R; k++) {
        const int pn = r0 + first + k * stride;
        e0n[k] = pn < r1 ? __ldcs(A.Uptr + pn) : 0;
        e1n[k] = pn < r1 ? __ldcs(A.Uptr + pn + 1) : 0;
    }
    for (int pb = r0 + first; pb < r1; pb += R * stride) {
        int p[R], e0[R], e1[R];
        bool ok[R];
        T ww[R];
#pragma unroll
        for (int k = 0; k < R; k++) {
            p[k] = pb + k * stride;
            ok[k] = p[k] < r1;
            e0[k] = ok[k] ? e0n[k] : 0;
            e1[k] = ok[k] ? e1n[k] : 0;
            const int pn = pb + (R + k) * stride;
            e0n[k] = pn < r1 ? __ldcs(A.Uptr + pn) : 0;
            e1n[k] = pn < r1 ? __ldcs(A.Uptr + pn + 1) : 0;
        }
#pragma unroll
        for (int k = 0; k < R; k++) ww[k] = ok[k] ? v.w[p[k]] : T(0);
        rows_chain<T, R, G, true, true>(ww, e0, e1, A.Ucol, A.Uc, v.w);
#pragma unroll
        for (int k = 0; k < R; k++)
            if (ok[k]) {
                v.w[p[k]] = ww[k];
                if (RW != RHO_NONE) arho.prod(ww[k], RW == RHO_R ? v.r[p[k]] : dotv[p[k]]);
            }
    }
}

// The block's contiguous chunk [c0, c1) of level L (sweep mapping 1):
// the same 1/nblocks share of every level's Morton order, so a block's chunks
// of consecutive levels cover nearly the same region of the mesh.
__device__ __forceinline__ void level_chunk(const int* lvl, int L, int nblocks, int bid, int& c0, int& c1)
{
    const int r0 = lvl[L], r1 = lvl[L + 1];
    const int chunk = (r1 - r0 + nblocks - 1) / nblocks;
    c0 = (int)min((long long)r0 + (long long)bid * chunk, (long long)r1);
    c1 = min(c0 + chunk, r1);
}

// w = M^-1 r with the DIC (or DILU) factor held in A's sweep coefficients,
// and the block partials of rho (RhoWith) in `slot` before the last grid
// barrier.  Forward sweep over levels 0 .. nlev-1, backward over nlev-2 .. 0
// (the top level has no upper neighbours: its backward step would leave w
// as it is, so its rho terms are taken in the forward step), one grid
// barrier per level.  The small last levels (level >= tail_from) run on the
// group's first block alone, forward then backward, with block-level
// barriers and one grid barrier after them.
// Row mapping (a.sweep): 1 (default), each block sweeps one contiguous chunk
// of every level (the same 1/nblocks share of each level's Morton order);
// 0, a level's rows strided over the group in blockDim-row pieces.  Measured
// at 200^3: mixed solve 328.8 against 333.5 ms, FP64 582.5 against 599.7 ms.
template <class T, int RW = RHO_R>
__device__ bool dic_apply(const SolveArgs& a, const Mat<T>& A, Vecs<T> v, const Group& g, PhaseClock& pc,
                          const T* dotv = nullptr, int slot = SL_B)
{
    const RowIter it = rows_of(g);
    const int nlev = a.nlev, tail = min(a.tail_from, nlev);
    const int tid = (int)threadIdx.x, bs = (int)blockDim.x;
    Acc<T> arho;
    auto end_step = [&](bool last) {
        if (RW != RHO_NONE && last) {
            double t[1] = {arho.value()};
            block_reduce_store<1>(t, a.partials, slot, g.bid);
        }
        return group_sync(g);
    };
    if (nlev == 0) return end_step(true);
    const bool chunks = a.sweep != 0;
    auto rows = [&](int L, int& c0, int& c1, int& first, int& stride) {
        if (chunks) {
            level_chunk(a.lvl, L, g.nblocks, g.bid, c0, c1);
            first = tid;
            stride = bs;
        } else {
            c0 = a.lvl[L];
            c1 = a.lvl[L + 1];
            first = it.first;
            stride = it.stride;
        }
    };
    for (int L = 0; L < tail; L++) {
        int c0, c1, first, stride;
        rows(L, c0, c1, first, stride);
        fwd_rows<T, RW>(A, v, c0, c1, first, stride, L == nlev - 1, dotv, arho);
        if (!end_step(nlev == 1)) return false;
        pc.lap(CK_FWD + min(L, 63));
    }
    if (tail < nlev) {
        if (g.bid == 0) {
            for (int L = tail; L < nlev; L++) {
                fwd_rows<T, RW>(A, v, a.lvl[L], a.lvl[L + 1], tid, bs, L == nlev - 1, dotv, arho);
                __syncthreads();
            }
            for (int L = nlev - 2; L >= tail; L--) {
                bwd_rows<T, RW>(A, v, a.lvl[L], a.lvl[L + 1], tid, bs, dotv, arho);
                __syncthreads();
            }
        }
        if (!end_step(tail == 0)) return false;
        pc.lap(CK_FWD + min(tail, 63));
    }
    for (int L = min(tail, nlev - 1) - 1; L >= 0; L--) {
        int c0, c1, first, stride;
        rows(L, c0, c1, first, stride);
        bwd_rows<T, RW>(A, v, c0, c1, first, stride, dotv, arho);
        if (!end_step(L == 0)) return false;
        pc.lap(CK_BWD + min(L, 63));
    }
    return true;
}

// ----------------------------------------------------- streaming passes ---
// Diagonal / no preconditioning in one pass, fused with the pending x/r
// update; returns sum|r| (of the updated r) and rho = w.r through t[0], t[1].
template <class T>
__device__ bool diag_pass(const SolveArgs& a, const Mat<T>& A, Vecs<T> v, bool pending, T alpha, const Group& g,
                          double (&t)[2])
{
    RowIter it = rows_of(g);
    Acc<T> ares, arho;
    for (int p = it.first; p < a.n; p += it.stride) {
        T rr = v.r[p];
        if (pending) {
            v.x[p] = fmadd(alpha, v.p[p], v.x[p]);
            rr = fmadd(-alpha, v.q[p], rr);
            v.r[p] = rr;
            ares.add(fabs(rr));
        }
        T ww = a.precond == SPUMA_PRECOND_DIAGONAL ? mul_rn(A.rD[p], rr) : rr;
        v.w[p] = ww;
        arho.prod(ww, rr);
    }
    double acc[2] = {ares.value(), arho.value()};
    block_reduce_store<2>(acc, a.partials, SL_A, g.bid);
    if (!group_sync(g)) return false;
    grid_reduce_read<2>(t, a.partials, SL_A, g.nblocks);
    return true;
}

// p = w (first) or w + beta p; 16-byte loads, scalar tail
template <class T>
__device__ bool search_direction(const SolveArgs& a, Vecs<T> v, bool first, T beta, const Group& g)
{
    using VT = typename V16<T>::type;
    constexpr int W = V16<T>::n;
    RowIter it = rows_of(g);
    const int nv = a.n / W;
    VT* pv = reinterpret_cast<VT*>(v.p);
    const VT* wv = reinterpret_cast<const VT*>(v.w);
    for (int i = it.first; i < nv; i += it.stride) {
        const VT ww = wv[i];
        pv[i] = first ? ww : vfma(beta, pv[i], ww);
    }
    for (int p = nv * W + it.first; p < a.n; p += it.stride) v.p[p] = first ? v.w[p] : fmadd(beta, v.p[p], v.w[p]);
    return group_sync(g);
}

// q = A p and sigma = q.p
template <class T>
__device__ bool amul_sigma(const SolveArgs& a, const Mat<T>& A, Vecs<T> v, const Group& g, double* sigma)
{
    constexpr int R = AmulShape<T>::R, G = AmulShape<T>::G;
    Acc<T> asig;
    RowIter it = rows_of(g);
    // rows [r0, r1) from `first` with `stride`
    auto range = [&](int r0, int r1, int first, int stride) {
        if (PipeShape<T>::in_solver && A.ell_w > 0 && A.ell_w <= PipeShape<T>::G) {
            ell_amul_pipelined<T, PipeShape<T>::R, PipeShape<T>::G>(A, v.p, r0 + first, stride, r1,
                                                                    [&](int p, T y, T xp) {
                                                                        v.q[p] = y;
                                                                        asig.prod(y, xp);
                                                                    });
            return;
        }
        for (int pb = r0 + first; pb < r1; pb += R * stride) {
            int p[R];
            T y[R], pp[R];
#pragma unroll
            for (int k = 0; k < R; k++) p[k] = pb + k * stride;
            amul_rows<T, R, G>(A, v.p, p, r1, y, pp);
#pragma unroll
            for (int k = 0; k < R; k++)
                if (p[k] < r1) {
                    v.q[p[k]] = y[k];
                    asig.prod(y[k], pp[k]);
                }
        }
    };
    // with amul_chunks each block takes its contiguous chunk of every level,
    // as in the sweeps: the rows a block takes cover one region of the mesh in
    // all levels, so the repeated gathers of a value stay in its SM's L1;
    // otherwise one segment, all rows strided over the group
    const int nseg = a.amul_chunks ? a.nlev : 1;
    for (int L = 0; L < nseg; L++) {
        int c0 = 0, c1 = a.n, first = it.first, stride = it.stride;
        if (a.amul_chunks) {
            level_chunk(a.lvl, L, g.nblocks, g.bid, c0, c1);
            first = (int)threadIdx.x;
            stride = (int)blockDim.x;
        }
        range(c0, c1, first, stride);
    }
    double sacc[1] = {asig.value()};
    block_reduce_store<1>(sacc, a.partials, SL_C, g.bid);
    if (!group_sync(g)) return false;
    double sg[1];
    grid_reduce_read<1>(sg, a.partials, SL_C, g.nblocks);
    *sigma = sg[0];
    return true;
}

// x += alpha p, r -= alpha q and sum|r| as a pass of its own, ahead of the
// forward sweep (16-byte loads, scalar tail).
template <class T>
__device__ bool update_pass(const SolveArgs& a, Vecs<T> v, T alpha, const Group& g, double* ressum)
{
    using VT = typename V16<T>::type;
    constexpr int W = V16<T>::n;
    RowIter it = rows_of(g);
    Acc<T> acc;
    const int nv = a.n / W;
    VT* xv = reinterpret_cast<VT*>(v.x);
    VT* rv = reinterpret_cast<VT*>(v.r);
    const VT* pv = reinterpret_cast<const VT*>(v.p);
    const VT* qv = reinterpret_cast<const VT*>(v.q);
    for (int i = it.first; i < nv; i += it.stride) {
        const VT rr = vfma(-alpha, qv[i], rv[i]);
        __stcs(xv + i, vfma(alpha, pv[i], __ldcs(xv + i)));
        rv[i] = rr;
        vadd_abs(acc, rr);
    }
    for (int p = nv * W + it.first; p < a.n; p += it.stride) {
        v.x[p] = fmadd(alpha, v.p[p], v.x[p]);
        const T r1 = fmadd(-alpha, v.q[p], v.r[p]);
        v.r[p] = r1;
        acc.add(fabs(r1));
    }
    double t[1] = {acc.value()};
    block_reduce_store<1>(t, a.partials, SL_D, g.bid);
    if (!group_sync(g)) return false;
    grid_reduce_read<1>(t, a.partials, SL_D, g.nblocks);
    *ressum = t[0];
    return true;
}

// w = M^-1 r and rho = w.r, after the pending update (x += alpha p,
// r -= alpha q, a pass of its own for DIC, fused into the diagonal pass
// otherwise), whose sum|r| is handed to `after_update`: it stops the loop
// (1), lets it go on (0) or replaces r and asks for w to be computed from the
// new r (2).
// Returns 0 (w and rho ready), 2 (stop) or -1 (device error).
template <class T, class AfterUpdate>
__device__ int precondition(const SolveArgs& a, const Mat<T>& A, Vecs<T> v, bool pending, T alpha, const Group& g,
                            PhaseClock& pc, double* rho, AfterUpdate after_update)
{
    if (a.precond == SPUMA_PRECOND_DIC) {
        if (pending) {
            double ressum;
            if (!update_pass<T>(a, v, alpha, g, &ressum)) return -1;
            pc.lap(CK_UPD);
            const int act = after_update(ressum);
            if (act < 0) return -1;
            if (act == 1) return 2;
        }
        if (!dic_apply<T>(a, A, v, g, pc)) return -1;
        double t[1];
        grid_reduce_read<1>(t, a.partials, SL_B, g.nblocks);
        *rho = t[0];
        return 0;
    }
    double t[2];
    if (!diag_pass<T>(a, A, v, pending, alpha, g, t)) return -1;
    pc.lap(CK_DIAG);
    const int act = pending ? after_update(t[0]) : 0;
    if (act < 0) return -1;
    if (act == 1) return 2;
    if (act == 2 && !diag_pass<T>(a, A, v, false, T(0), g, t)) return -1;
    *rho = t[1];
    return 0;
}

// PCG iterations on (A, v.r) from the current v.x (OpenFOAM recurrences).
// Returns the iteration count, or -1 when a device error stopped the group.
template <class T>
__device__ int pcg_loop(const SolveArgs& a, const Mat<T>& A, Vecs<T> v, double nfac, double res0, double tol,
                        double rel_tol, int max_iter, int min_iter, double* res_out, int* singular,
                        const Group& g)
{
    PhaseClock pc(a.phase_clk, g.bid);
    double res = res0;
    *res_out = res;
    if (!(min_iter > 0 || !converged(res0, res0, tol, rel_tol))) return 0;
    int n_it = 0;
    double rho = 1.0, rho_old;
    T alpha = (T)0;
    bool pending = false;
    for (;;) {
        rho_old = rho;
        const int st = precondition<T>(a, A, v, pending, alpha, g, pc, &rho, [&](double ressum) {
            res = ressum / nfac;
            n_it++;
            return ((n_it < max_iter && !converged(res, res0, tol, rel_tol)) || n_it < min_iter) ? 0 : 1;
        });
        if (st < 0) return -1;
        if (st == 2) break;
        const bool first = !pending;
        if (!search_direction<T>(a, v, first, first ? (T)0 : (T)(rho / rho_old), g)) return -1;
        pc.lap(CK_PUPD);
        double sigma;
        if (!amul_sigma<T>(a, A, v, g, &sigma)) return -1;
        pc.lap(CK_AMUL);
        pc.count(CK_ITERS);
        if (fabs(sigma) / nfac < 1e-300) {
            *singular = 1;
            break;
        }
        alpha = (T)(rho / sigma);
        pending = true;
    }
    *res_out = res;
    return n_it;
}

// FP64 refinement step of the mixed forms: x += xs (FP32 correction, reset to
// 0) when fold, then r = b - A64 x with sum|r| and max|r|, and r32 = float(r).
__device__ bool refine_residual(const SolveArgs& a, const Group& g, bool fold, double* ressum, double* rmax)
{
    RowIter it = rows_of(g);
    const Mat<double> A64 = mat_of<double>(a);
    if (fold) {
        for (int p = it.first; p < a.n; p += it.stride) {
            a.x[p] = __dadd_rn(a.x[p], (double)a.xi[p]);
            a.xi[p] = 0.0f;
        }
        if (!group_sync(g)) return false;
    }
    double acc[1] = {0.0}, mx[1] = {0.0};
    for (int p = it.first; p < a.n; p += it.stride) {
        const double rr = a.b[p] - amul_row<double>(A64, a.x, p);
        a.r[p] = rr;
        a.ri[p] = (float)rr;
        acc[0] += fabs(rr);
        mx[0] = fmax(mx[0], fabs(rr));
    }
    block_reduce_store<1>(acc, a.partials, SL_D, g.bid);
    block_max_store<1>(mx, a.partials, SL_D + 1, g.bid);
    if (!group_sync(g)) return false;
    double t[1], m[1];
    grid_reduce_read<1>(t, a.partials, SL_D, g.nblocks);
    grid_reduce_read<1, true>(m, a.partials, SL_D + 1, g.nblocks);
    *ressum = t[0];
    *rmax = m[0];
    return true;
}

// Mixed precision with reliable updates: FP32 PCG whose correction and
// residual are replaced by FP64 ones (x += xs; r = b - A64 x) whenever the
// FP32 residual has dropped by inner_rel_tol since the last replacement, the
// FP32 residual claims convergence, or max_iter is reached; the search
// direction is kept, so the Krylov space is never restarted.
__device__ bool solve_mixed_reliable(const SolveArgs& a, const Group& g, double nfac, double res0,
                                     spuma_solver_perf& pf)
{
    RowIter it = rows_of(g);
    const Mat<float> A32 = mat_of<float>(a);
    Vecs<float> v{a.xi, a.ri, a.wi, a.pi, a.qi};
    PhaseClock pc(a.phase_clk, g.bid);
    const double delta = a.inner_rel_tol;
    double res = res0, rupd = res0, rho = 1.0, rho_old;
    int n_it = 0, updates = 0, singular = 0;
    float alpha = 0.0f;
    bool pending = false, ok = true;
    if (!converged(res0, res0, a.tol, a.rel_tol)) {
        for (int p = it.first; p < a.n; p += it.stride) {
            v.r[p] = (float)a.r[p];
            v.x[p] = 0.0f;
        }
        if (!group_sync(g)) return false;
        for (;;) {
            rho_old = rho;
            const int st = precondition<float>(a, A32, v, pending, alpha, g, pc, &rho, [&](double ressum) {
                n_it++;
                const double ress = ressum / nfac;
                if (!(ress < delta * rupd || converged(ress, res0, a.tol, a.rel_tol) || n_it >= a.max_iter)) return 0;
                double rs, rm;
                if (!refine_residual(a, g, true, &rs, &rm)) return -1;
                pc.lap(CK_RESID);
                updates++;
                res = rs / nfac;
                if (converged(res, res0, a.tol, a.rel_tol) || n_it >= a.max_iter) return 1;
                rupd = res;
                return 2;
            });
            if (st < 0) return false;
            if (st == 2) break;
            const bool first = !pending;
            if (!search_direction<float>(a, v, first, first ? 0.0f : (float)(rho / rho_old), g)) return false;
            pc.lap(CK_PUPD);
            double sigma;
            if (!amul_sigma<float>(a, A32, v, g, &sigma)) return false;
            pc.lap(CK_AMUL);
            pc.count(CK_ITERS);
            if (fabs(sigma) / nfac < 1e-300) {
                singular = 1;
                double rs, rm;
                ok = refine_residual(a, g, true, &rs, &rm);
                res = rs / nfac;
                break;
            }
            alpha = (float)(rho / sigma);
            pending = true;
        }
    }
    // the FP32 w and p were gathered evict-last: hand their lines back
    release_lines(a.wi, 4 * (size_t)a.n, it.first, it.stride);
    release_lines(a.pi, 4 * (size_t)a.n, it.first, it.stride);
    pf.initial_residual = res0;
    pf.final_residual = res;
    pf.n_iter = n_it;
    pf.n_outer = updates;
    pf.converged = converged(res, res0, a.tol, a.rel_tol);
    pf.singular = singular;
    return ok;
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

// The report's true residual ||b - A x||_2 / ||b||_2 (||b - A x||_2 when b = 0)
// in FP64 from the FP64 coefficients of A, for every solve kind: each r_p in
// the Amul's face order, the sums of squares as fused multiply-adds per
// thread, then the deterministic block and grid reductions.  b_int: b in
// internal order, or NULL to read the caller's b through perm (PBiCG reuses
// the internal b as its transposed residual).
__device__ bool true_residual(const SolveArgs& a, const Mat<double>& A, const double* b_int, const Group& g,
                              double* out)
{
    RowIter it = rows_of(g);
    double acc[2] = {0.0, 0.0};
    for (int p = it.first; p < a.n; p += it.stride) {
        const double bv = b_int ? b_int[p] : a.b_orig[a.perm[p]];
        const double rr = __dsub_rn(bv, amul_row<double>(A, a.x, p));
        acc[0] = __fma_rn(rr, rr, acc[0]);
        acc[1] = __fma_rn(bv, bv, acc[1]);
    }
    block_reduce_store<2>(acc, a.partials, SL_A, g.bid);
    if (!group_sync(g)) return false;
    double t[2];
    grid_reduce_read<2>(t, a.partials, SL_A, g.nblocks);
    *out = t[1] > 0.0 ? __ddiv_rn(__dsqrt_rn(t[0]), __dsqrt_rn(t[1])) : __dsqrt_rn(t[0]);
    return true;
}

__device__ void phase_store_x(const SolveArgs& a, const Group& g)
{
    RowIter it = rows_of(g);
    for (int p = it.first; p < a.n; p += it.stride) a.x_orig[a.perm[p]] = a.x[p];
}

// Mixed precision, restarted form: FP64 refinement around FP32 inner PCG
// solves of A d = r / max|r| from d = 0 to inner_rel_tol.
__device__ bool solve_mixed_restart(const SolveArgs& a, const Group& g, double nfac, spuma_solver_perf& pf)
{
    RowIter it = rows_of(g);
    const Mat<float> A32 = mat_of<float>(a);
    Vecs<float> vi{a.xi, a.ri, a.wi, a.pi, a.qi};
    int outer = 0, total = 0, singular = 0;
    double res = 0.0, res0 = 0.0;
    for (;;) {
        double rs, rm;
        if (!refine_residual(a, g, false, &rs, &rm)) return false;
        res = rs / nfac;
        if (outer == 0) res0 = res;
        if (res < a.tol || outer >= a.max_outer || singular) break;
        const double s = rm;
        if (s == 0.0) break;
        Acc<float> ain;
        for (int p = it.first; p < a.n; p += it.stride) {
            float rv = (float)(a.r[p] / s);
            vi.r[p] = rv;
            vi.x[p] = 0.0f;
            ain.add(fabsf(rv));
        }
        double iacc[1] = {ain.value()};
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
    release_lines(a.wi, 4 * (size_t)a.n, it.first, it.stride);
    release_lines(a.pi, 4 * (size_t)a.n, it.first, it.stride);
    pf.initial_residual = res0;
    pf.final_residual = res;
    pf.n_iter = total;
    pf.n_outer = outer;
    pf.converged = res < a.tol;
    pf.singular = singular;
    return true;
}

// Kinds of persistent launch, one kernel each so that every kernel holds only
// its own path (register allocation is per kernel).
// -------------------------------------------------------------- PBiCG ---
// OpenFOAM PBiCG on an asymmetric matrix (the paper's momentum solver: PBiCG
// with DILU), FP64, after phase_init (x, rA = b - A x, normFactor from the
// row sums of A).  Vectors: x, rA = r, wA = w, pA = p, wT = q, rT = b (the
// right-hand side is not needed past rT = b - A^T x), pT.  A^T shares A's
// structure: its lower entries of row u hold upper_f and its upper entries of
// row l lower_f; the transposed DILU sweeps use rD times those.
__device__ bool solve_pbicg(const SolveArgs& a, const Group& g, double nfac, double res0, spuma_solver_perf& pf)
{
    RowIter it = rows_of(g);
    const Mat<double> A = mat_of<double>(a);
    Mat<double> AT = A;
    AT.La = a.LaT64;
    AT.Ua = a.UaT64;
    AT.Lc = a.LcT64;
    AT.Uc = a.UcT64;
    AT.Ea = a.EaT64;
    double *x = a.x, *rA = a.r, *wA = a.w, *pA = a.p, *wT = a.q, *rT = a.b, *pT = a.pT;
    PhaseClock pc(a.phase_clk, g.bid);
    for (int p = it.first; p < a.n; p += it.stride) rT[p] = a.b[p] - amul_row<double>(AT, x, p);
    if (!group_sync(g)) return false;
    double res = res0;
    int n_it = 0, singular = 0;
    if (a.min_iter > 0 || !converged(res0, res0, a.tol, a.rel_tol)) {
        double wArA = 1.0, wArA_old, alpha = 0.0;
        bool pending = false;
        for (;;) {
            if (pending) {
                double acc[1] = {0.0};
                for (int p = it.first; p < a.n; p += it.stride) {
                    x[p] = fmadd(alpha, pA[p], x[p]);
                    rA[p] = fmadd(-alpha, wA[p], rA[p]);
                    rT[p] = fmadd(-alpha, wT[p], rT[p]);
                    acc[0] += fabs(rA[p]);
                }
                block_reduce_store<1>(acc, a.partials, SL_D, g.bid);
                if (!group_sync(g)) return false;
                grid_reduce_read<1>(acc, a.partials, SL_D, g.nblocks);
                res = acc[0] / nfac;
                n_it++;
                pc.lap(CK_UPD);
                if (!((n_it < a.max_iter && !converged(res, res0, a.tol, a.rel_tol)) || n_it < a.min_iter)) break;
            }
            wArA_old = wArA;
            if (a.precond == SPUMA_PRECOND_DILU) {
                if (!dic_apply<double, RHO_VEC>(a, A, Vecs<double>{x, rA, wA, pA, wT}, g, pc, rT, SL_B)) return false;
                if (!dic_apply<double, RHO_NONE>(a, AT, Vecs<double>{x, rT, wT, pT, wA}, g, pc)) return false;
            } else {
                double acc[1] = {0.0};
                for (int p = it.first; p < a.n; p += it.stride) {
                    const double wa = __dmul_rn(a.rD64[p], rA[p]);
                    wA[p] = wa;
                    wT[p] = __dmul_rn(a.rD64[p], rT[p]);
                    acc[0] = fmadd(wa, rT[p], acc[0]);
                }
                block_reduce_store<1>(acc, a.partials, SL_B, g.bid);
                if (!group_sync(g)) return false;
                pc.lap(CK_DIAG);
            }
            double t[1];
            grid_reduce_read<1>(t, a.partials, SL_B, g.nblocks);
            wArA = t[0];
            const bool first = !pending;
            const double beta = first ? 0.0 : wArA / wArA_old;
            for (int p = it.first; p < a.n; p += it.stride) {
                pA[p] = first ? wA[p] : fmadd(beta, pA[p], wA[p]);
                pT[p] = first ? wT[p] : fmadd(beta, pT[p], wT[p]);
            }
            if (!group_sync(g)) return false;
            pc.lap(CK_PUPD);
            double acc[1] = {0.0};
            for (int p = it.first; p < a.n; p += it.stride) {
                const double y = amul_row<double>(A, pA, p);
                wA[p] = y;
                wT[p] = amul_row<double>(AT, pT, p);
                acc[0] = fmadd(y, pT[p], acc[0]);
            }
            block_reduce_store<1>(acc, a.partials, SL_C, g.bid);
            if (!group_sync(g)) return false;
            grid_reduce_read<1>(acc, a.partials, SL_C, g.nblocks);
            pc.lap(CK_AMUL);
            pc.count(CK_ITERS);
            const double wApT = acc[0];
            if (fabs(wApT) / nfac < 1e-300) {
                singular = 1;
                break;
            }
            alpha = wArA / wApT;
            pending = true;
        }
    }
    pf.initial_residual = res0;
    pf.final_residual = res;
    pf.n_iter = n_it;
    pf.converged = converged(res, res0, a.tol, a.rel_tol);
    pf.singular = singular;
    return true;
}

enum SolveKind { KIND_SETUP = 0, KIND_F64 = 1, KIND_MIXED = 2, KIND_MIXED_RESTART = 3, KIND_PBICG = 4 };

// TRUE_INLINE: the report's true residual is computed inside the launch
// (batched launches); the single-system solver leaves it to the two small
// kernels that follow it on the stream (k_true_residual_*), so that its own
// register allocation is not burdened by one more Amul.
template <int KIND, bool TRUE_INLINE>
__device__ void run_system(const SolveArgs& a, const Group& g)
{
    spuma_solver_perf pf;
    pf.initial_residual = 0.0;
    pf.final_residual = 0.0;
    pf.true_rel_residual_l2 = 0.0;
    pf.n_iter = 0;
    pf.n_outer = 0;
    pf.converged = 0;
    pf.singular = 0;
    pf.status = 0;
    pf.n_levels = a.nlev;
    bool ok = true;
    if (a.mode == MODE_PREPARE || a.mode == MODE_SOLVE) {
        ok = phase_gather<KIND == KIND_PBICG>(a, g);
        if (ok) ok = phase_factor<KIND == KIND_PBICG>(a, g);
    }
    if (KIND == KIND_SETUP && ok && a.mode == MODE_PRECONDITION) {
        // w = M^-1 r for r = b_orig, written to x_orig (FP64)
        RowIter it = rows_of(g);
        for (int p = it.first; p < a.n; p += it.stride) a.r[p] = a.b_orig[a.perm[p]];
        ok = group_sync(g);
        Vecs<double> v{a.x, a.r, a.w, a.p, a.q};
        const Mat<double> A = mat_of<double>(a);
        if (ok) {
            if (a.precond == SPUMA_PRECOND_DIC) {
                PhaseClock pc(nullptr, g.bid);
                ok = dic_apply<double>(a, A, v, g, pc);
            } else {
                for (int p = it.first; p < a.n; p += it.stride)
                    a.w[p] = a.precond == SPUMA_PRECOND_DIAGONAL ? __dmul_rn(a.rD64[p], a.r[p]) : a.r[p];
                ok = group_sync(g);
            }
        }
        if (ok)
            for (int p = it.first; p < a.n; p += it.stride) a.x_orig[a.perm[p]] = a.w[p];
    }
    if constexpr (KIND != KIND_SETUP) {
        if (ok && a.mode == MODE_SOLVE) {
            double nfac = 1.0, res0 = 0.0;
            ok = phase_init(a, g, &nfac, &res0);
            if (ok) {
                if constexpr (KIND == KIND_PBICG) {
                    ok = solve_pbicg(a, g, nfac, res0, pf);
                } else if constexpr (KIND == KIND_MIXED) {
                    ok = solve_mixed_reliable(a, g, nfac, res0, pf);
                } else if constexpr (KIND == KIND_MIXED_RESTART) {
                    ok = solve_mixed_restart(a, g, nfac, pf);
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
            if constexpr (TRUE_INLINE) {
                if (ok) {
                    Mat<double> A64 = mat_of<double>(a);
                    if (KIND == KIND_PBICG) A64.ell_w = 0;   // asymmetric: the internal CSR holds A
                    ok = true_residual(a, A64, KIND == KIND_PBICG ? nullptr : a.b, g, &pf.true_rel_residual_l2);
                }
            }
            if (ok && !a.no_store) phase_store_x(a, g);
        }
    }
    if (g.bid == 0 && threadIdx.x == 0 && a.perf) {
        __threadfence();
        pf.status = ld_volatile_int(a.status);
        // a group that stopped always has a status; keep the report honest if not
        if (!ok && pf.status == 0) pf.status = SPUMA_ERR_DEVICE_TIMEOUT;
        if (pf.status != 0) pf.converged = 0;
        *a.perf = pf;
    }
}

template <int KIND>
__global__ void __launch_bounds__(1024, 1) k_solve(SolveArgs a, unsigned long long timeout_ns)
{
    Group g{reinterpret_cast<unsigned long long*>(a.status + DS_BARRIER), a.status, (int)gridDim.x, (int)blockIdx.x, timeout_ns};
    run_system<KIND, false>(a, g);
}

// The single-system solver's true residual, after it on the stream: per-block
// sums of r_p^2 and b_p^2 (r = b - A64 x in the Amul's face order, one FMA per
// term, each thread's rows in order) into the partials, then one warp adds
// the block partials in block order and writes ||r||_2/||b||_2 (||r||_2 when
// b = 0) into the report.  Deterministic, like every reduction here.
__global__ void __launch_bounds__(256) k_true_residual_part(SolveArgs a, int asym)
{
    Mat<double> A64 = mat_of<double>(a);
    if (asym) A64.ell_w = 0;
    double acc[2] = {0.0, 0.0};
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < a.n; p += gridDim.x * blockDim.x) {
        const double bv = asym ? a.b_orig[a.perm[p]] : a.b[p];
        const double rr = __dsub_rn(bv, amul_row<double>(A64, a.x, p));
        acc[0] = __fma_rn(rr, rr, acc[0]);
        acc[1] = __fma_rn(bv, bv, acc[1]);
    }
    block_reduce_store<2>(acc, a.partials, SL_A, blockIdx.x);
}

__global__ void k_true_residual_final(SolveArgs a, int nblocks)
{
    double t[2];
    grid_reduce_read<2>(t, a.partials, SL_A, nblocks);
    if (threadIdx.x == 0 && a.perf)
        a.perf->true_rel_residual_l2 = t[1] > 0.0 ? __ddiv_rn(__dsqrt_rn(t[0]), __dsqrt_rn(t[1])) : __dsqrt_rn(t[0]);
}

// The batched launch, one instance per solve kind and largest block size
// (the register budget follows from it: 128 per thread up to 512 threads, 64
// at 1024).
template <int KIND, int MAXT>
__global__ void __launch_bounds__(MAXT, MAXT <= 256 ? 2 : 1) k_solve_batch(BatchTable t, unsigned long long timeout_ns)
{
    __shared__ SolveArgs sa;
    int s = 0;
    while (s + 1 < t.n_sys && (int)blockIdx.x >= t.split[s + 1]) s++;
    if (threadIdx.x == 0) sa = *t.args[s];
    __syncthreads();
    Group g{reinterpret_cast<unsigned long long*>(sa.status + DS_BARRIER), sa.status, t.split[s + 1] - t.split[s],
            (int)blockIdx.x - t.split[s], timeout_ns};
    run_system<KIND, true>(sa, g);
}

// Stand-alone Amul on the prepared matrix (internal order): the PCG's Amul
// phase as a kernel of its own.
template <class T>
__global__ void __launch_bounds__(256) k_amul_prepared(int n, Mat<T> A, const T* __restrict__ x, T* __restrict__ y)
{
    constexpr int R = AmulShape<T>::R, G = AmulShape<T>::G;
    const int stride = gridDim.x * blockDim.x;
    if (PipeShape<T>::stand_alone && A.ell_w > 0 && A.ell_w <= PipeShape<T>::G) {
        ell_amul_pipelined<T, PipeShape<T>::R, PipeShape<T>::G>(A, x, blockIdx.x * blockDim.x + threadIdx.x, stride, n,
                                                                [&](int p, T yv, T) { __stcs(y + p, yv); });
        return;
    }
    for (int pb = blockIdx.x * blockDim.x + threadIdx.x; pb < n; pb += R * stride) {
        int p[R];
        T yy[R], xp[R];
#pragma unroll
        for (int k = 0; k < R; k++) p[k] = pb + k * stride;
        amul_rows<T, R, G, false>(A, x, p, n, yy, xp);
#pragma unroll
        for (int k = 0; k < R; k++)
            if (p[k] < n) __stcs(y + p[k], yy[k]);
    }
}

// Stand-alone Amul on the fixed-width layout alone (no row-extent branch in
// the kernel, rows of at most W entries): its registers stay within 32 per
// thread, so that 2048 threads per SM are resident and enough loads are in
// flight; one wave of 8 blocks per SM walks the rows (FP64: 140 -> 130.6 us
// at 200^3 against the kernel shared with the row-extent path).  Each row: d_p x_p, then
// its entries in layout order (lower ascending, then upper ascending), one
// FMA each: the same sums as the solver's Amul phase.
template <class T, int W>
__global__ void __launch_bounds__(256, 8) k_amul_ell(int n, Mat<T> A, const T* __restrict__ x, T* __restrict__ y)
{
    const int stride = gridDim.x * blockDim.x;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        int c[W];
        T a[W], v[W];
#pragma unroll
        for (int j = 0; j < W; j++) {
            const bool ok = j < A.ell_w;
            const size_t e = (size_t)j * A.ell_stride + p;
            c[j] = ok ? __ldcs(A.Ecol + e) : -1;
            a[j] = ok ? __ldcs(A.Ea + e) : T(0);
        }
        const T xp = x[p];
        const T d = __ldcs(A.d + p);
#pragma unroll
        for (int j = 0; j < W; j++) v[j] = c[j] >= 0 ? x[c[j]] : T(0);
        T yy = mul_rn(d, xp);
#pragma unroll
        for (int j = 0; j < W; j++)
            if (c[j] >= 0) yy = fmadd(a[j], v[j], yy);
        __stcs(y + p, yy);
    }
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
// Row mapping of the DIC sweeps: 1 (default) contiguous level chunks per
// block, 0 strided (SPUMA_SWEEP=0, a measurement override).
static int sweep_mode()
{
    static const int m = [] {
        const char* e = getenv("SPUMA_SWEEP");
        return (e && atoi(e) == 0) ? 0 : 1;
    }();
    return m;
}

SolveArgs make_args(spuma_ldu_t h)
{
    SolveArgs a{};
    const Layout& L = h->L;
    a.n = h->n;
    a.nf = h->nf;
    a.nlev = h->nlev;
    a.tail_from = h->nlev;

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
    a.lower_orig = nullptr;
    a.LaT64 = L.asym ? h->at<double>(L.LaT64) : nullptr;
    a.UaT64 = L.asym ? h->at<double>(L.UaT64) : nullptr;
    a.LcT64 = L.asym ? h->at<double>(L.LcT64) : nullptr;
    a.UcT64 = L.asym ? h->at<double>(L.UcT64) : nullptr;
    a.pT = L.asym ? h->at<double>(L.pT64) : nullptr;
    a.EaT64 = L.asym ? h->at<double>(L.EaT64) : nullptr;
    a.Ecol = h->at<int>(L.Ecol);
    a.Ea64 = h->at<double>(L.Ea64);
    a.Ea32 = h->at<float>(L.Ea32);
    a.ell_w = h->ell_w;
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
    a.sweep = sweep_mode();
    return a;
}

static int kind_of(const SolveArgs& a)
{
    if (a.mode != MODE_SOLVE) return KIND_SETUP;
    if (a.lower_orig) return KIND_PBICG;
    if (a.precision == SPUMA_MIXED) return KIND_MIXED;
    if (a.precision == SPUMA_MIXED_RESTART) return KIND_MIXED_RESTART;
    return KIND_F64;
}

static const void* solve_kernel(int kind)
{
    switch (kind) {
    case KIND_SETUP: return (const void*)k_solve<KIND_SETUP>;
    case KIND_MIXED: return (const void*)k_solve<KIND_MIXED>;
    case KIND_MIXED_RESTART: return (const void*)k_solve<KIND_MIXED_RESTART>;
    case KIND_PBICG: return (const void*)k_solve<KIND_PBICG>;
    default: return (const void*)k_solve<KIND_F64>;
    }
}

template <int MAXT>
static const void* batch_kernel_t(int kind)
{
    switch (kind) {
    case KIND_MIXED: return (const void*)k_solve_batch<KIND_MIXED, MAXT>;
    case KIND_MIXED_RESTART: return (const void*)k_solve_batch<KIND_MIXED_RESTART, MAXT>;
    default: return (const void*)k_solve_batch<KIND_F64, MAXT>;
    }
}

static const void* batch_kernel(int kind, int threads)
{
    if (threads <= 256) return batch_kernel_t<256>(kind);
    if (threads <= 512) return batch_kernel_t<512>(kind);
    return batch_kernel_t<1024>(kind);
}

static std::mutex g_occ_mu;
static std::map<long long, int> g_occ;   // (kernel, block threads, ring) -> co-resident blocks per SM

int solve_blocks_per_sm(int threads, bool batch, int kind, size_t dyn = 0)
{
    std::lock_guard<std::mutex> lk(g_occ_mu);
    const long long key = (((long long)(threads * 2 + (batch ? 1 : 0)) * 8 + kind) << 20) + (long long)dyn;
    auto it = g_occ.find(key);
    if (it != g_occ.end()) return it->second;
    const void* k = batch ? batch_kernel(kind, threads) : solve_kernel(kind);
    int nb = 0;
    cudaError_t e = cudaSuccess;
    if (dyn) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, dyn);
    if (e != cudaSuccess) {
        cudaGetLastError();
        nb = 0;
    }
    g_occ[key] = nb;
    return nb;
}

int default_threads(const spuma_solver_controls* ctl)
{
    if (ctl && ctl->block_threads > 0) return ctl->block_threads;
    return 1024;
}

// Blocks of the persistent single-system solver: one per row chunk of
// `threads` rows, at most all co-resident blocks (SPUMA_SOLVE_BLOCKS_PER_SM
// caps the blocks per SM, a tuning override).  0 when the kernel cannot be
// resident.
int solve_grid(spuma_ldu_t h, int threads, int kind, size_t dyn)
{
    int per_sm = solve_blocks_per_sm(threads, false, kind, dyn);
    if (per_sm < 1) return 0;
    if (const char* env = getenv("SPUMA_SOLVE_BLOCKS_PER_SM")) {
        int v = atoi(env);
        if (v >= 1 && v < per_sm) per_sm = v;
    }
    int64_t want = ((int64_t)h->n + threads - 1) / threads;
    int64_t maxg = std::min<int64_t>((int64_t)per_sm * h->num_sms, kMaxBlocks);
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, maxg));
}

// First level of the run of small last levels (each with at most `threads`
// rows) that the solver's first block handles alone; SPUMA_TAIL_ROWS
// overrides the row limit (0 disables).
int tail_level(spuma_ldu_t h, int threads)
{
    int limit = threads;
    if (const char* e = getenv("SPUMA_TAIL_ROWS")) limit = atoi(e);
    int t = h->nlev;
    while (t > 1 && (int64_t)h->h_lvl[t] - h->h_lvl[t - 1] <= limit) t--;
    // keep at least two levels in the tail, else the single grid barrier saves nothing
    return (h->nlev - t >= 2) ? t : h->nlev;
}

spuma_status launch_solve(spuma_ldu_t h, const SolveArgs& a, int threads, cudaStream_t s)
{
    if (threads < 32 || threads > 1024 || threads % 32) {
        set_error("block_threads must be a multiple of 32 in [32, 1024]");
        return SPUMA_ERR_INVALID_ARG;
    }
    const int kind = kind_of(a);
    const int grid = solve_grid(h, threads, kind, 0);
    if (grid < 1) { set_error("solver kernel cannot be resident"); return SPUMA_ERR_CUDA; }
    SPUMA_CUDA(cudaMemsetAsync(h->at<char>(h->L.bar), 0, h->L.status + 256 - h->L.bar, s));
    unsigned long long tns = barrier_timeout_ns();
    SolveArgs b = a;
    b.tail_from = tail_level(h, threads);
    // SPUMA_AMUL_CHUNKS=1: the Amul phase walks level chunks when the levels
    // are wide (an average level gives every block at least a block's worth
    // of rows).  Off by default: measured at 200^3, Amul phase 101.9 -> 112.7
    // us per FP32 iteration, mixed solve 328.8 -> 338.1 ms
    static const bool amul_chunks_env = getenv("SPUMA_AMUL_CHUNKS") && atoi(getenv("SPUMA_AMUL_CHUNKS")) != 0;
    b.amul_chunks = amul_chunks_env && b.sweep != 0 && h->nlev > 0 &&
                    (int64_t)h->n / h->nlev >= (int64_t)grid * threads;
    if (getenv("SPUMA_PHASE_CLOCKS")) {
        b.phase_clk = h->at<long long>(h->L.clk);
        SPUMA_CUDA(cudaMemsetAsync(b.phase_clk, 0, 8 * 256, s));
    }
    void* args[] = {(void*)&b, (void*)&tns};
    SPUMA_CUDA(cudaLaunchCooperativeKernel(solve_kernel(kind), grid, threads, args, 0, s));
    count_launch();
    if (b.mode == MODE_SOLVE) {
        // the report's true residual (the solver's x in internal order is still in the workspace)
        const int tg = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)h->n + 255) / 256, (int64_t)h->num_sms * 8));
        k_true_residual_part<<<tg, 256, 0, s>>>(b, kind == KIND_PBICG ? 1 : 0);
        k_true_residual_final<<<1, 32, 0, s>>>(b, tg);
        count_launch(2);
        SPUMA_CUDA(cudaGetLastError());
    }
    return SPUMA_OK;
}

spuma_status launch_batch_kernel(const BatchTable& t, int grid, int threads, int kind, cudaStream_t s)
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
    BatchTable tt = t;
    void* args[] = {(void*)&tt, (void*)&tns};
    SPUMA_CUDA(cudaLaunchKernelExC(&cfg, batch_kernel(kind, threads), args));
    return SPUMA_OK;
}

int batch_kind(int precision)
{
    if (precision == SPUMA_MIXED) return KIND_MIXED;
    if (precision == SPUMA_MIXED_RESTART) return KIND_MIXED_RESTART;
    return KIND_F64;
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
    if (c->precision != SPUMA_F64 && c->precision != SPUMA_MIXED && c->precision != SPUMA_MIXED_RESTART) return false;
    if (!(c->tolerance >= 0.0) || !(c->rel_tol >= 0.0) || c->max_iter < 0 || c->min_iter < 0) return false;
    if ((c->precision == SPUMA_MIXED || c->precision == SPUMA_MIXED_RESTART) &&
        (!(c->inner_rel_tol > 0.0) || c->max_outer < 0))
        return false;
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

spuma_status spuma_pbicg_solve(spuma_ldu_t h, const double* diag, const double* lower, const double* upper,
                               const double* b, double* x, const spuma_solver_controls* ctl, spuma_solver_perf* perf,
                               spuma_stream_t stream)
{
    if (!h || !ctl || (ctl->precond != SPUMA_PRECOND_NONE && ctl->precond != SPUMA_PRECOND_DIAGONAL &&
                       ctl->precond != SPUMA_PRECOND_DILU) ||
        ctl->precision != SPUMA_F64 || !(ctl->tolerance >= 0.0) || !(ctl->rel_tol >= 0.0) || ctl->max_iter < 0 ||
        ctl->min_iter < 0 || (h->n > 0 && (!diag || !b || !x)) || (h->nf > 0 && (!lower || !upper))) {
        set_error("spuma_pbicg_solve: bad argument (precond NONE, DIAGONAL or DILU; precision F64)");
        return SPUMA_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (h->n == 0) {
        if (perf) {
            spuma_solver_perf z{};
            z.converged = 1;
            SPUMA_CUDA(cudaMemcpyAsync(perf, &z, sizeof(z), cudaMemcpyHostToDevice, s));
        }
        return SPUMA_OK;
    }
    if (!h->L.asym) {
        set_error("spuma_pbicg_solve: the workspace was not sized with SPUMA_WORKSPACE_ASYMMETRIC");
        return SPUMA_ERR_WORKSPACE_TOO_SMALL;
    }
    SolveArgs a = make_args(h);
    fill_controls(a, ctl);
    a.mode = MODE_SOLVE;
    a.zero_x0 = 0;
    a.diag_orig = diag;
    a.upper_orig = upper;
    a.lower_orig = lower;
    a.b_orig = b;
    a.x_orig = x;
    a.perf = perf;
    h->prepared_precond = -1;
    return launch_solve(h, a, default_threads(ctl), s);
}

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
        Mat<double> A{a.Lptr, a.Lcol, a.La64, a.Lc64, a.Uptr, a.Ucol, a.Ua64, a.Uc64, a.d64, a.rD64,
                      a.Ecol, a.Ea64, a.ell_w, a.n};
        const int ge = std::min(g, h->num_sms * 8);
        if (a.ell_w > 0 && a.ell_w <= 6)
            k_amul_ell<double, 6><<<ge, 256, 0, s>>>(h->n, A, (const double*)x, (double*)y);
        else if (a.ell_w > 0)
            k_amul_ell<double, kEllMax><<<ge, 256, 0, s>>>(h->n, A, (const double*)x, (double*)y);
        else
            k_amul_prepared<double><<<g, 256, 0, s>>>(h->n, A, (const double*)x, (double*)y);
    } else {
        Mat<float> A{a.Lptr, a.Lcol, a.La32, a.Lc32, a.Uptr, a.Ucol, a.Ua32, a.Uc32, a.d32, a.rD32,
                     a.Ecol, a.Ea32, a.ell_w, a.n};
        // FP32: the software-pipelined kernel measured faster than the
        // 32-register one (90.4 against 92.8 us at 200^3)
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

spuma_status spuma_read_phase_clocks(spuma_ldu_t h, int64_t* out, int32_t n, spuma_stream_t stream)
{
    if (!h || !out || n < 0 || n > 256) { set_error("spuma_read_phase_clocks: bad argument"); return SPUMA_ERR_INVALID_ARG; }
    SPUMA_CUDA(cudaMemcpyAsync(out, h->at<long long>(h->L.clk), 8 * (size_t)n, cudaMemcpyDeviceToHost,
                               (cudaStream_t)stream));
    SPUMA_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return SPUMA_OK;
}

spuma_status spuma_pcg_solve(spuma_ldu_t h, const double* diag, const double* upper, const double* b, double* x,
                             const spuma_solver_controls* ctl, spuma_solver_perf* perf, spuma_stream_t stream)
{
    return pcg_solve_internal(h, diag, upper, b, x, ctl, perf, (cudaStream_t)stream, 0);
}

}  // extern "C"
