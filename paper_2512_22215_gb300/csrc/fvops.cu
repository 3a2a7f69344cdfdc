// fvops.cu -- the finite-volume operators around the pressure solve in the
// paper's SIMPLE loop (fvSchemes listing: gradSchemes Gauss linear,
// interpolationSchemes linear, laplacianSchemes Gauss linear corrected,
// snGradSchemes corrected; fvSolution: nNonOrthogonalCorrectors 0):
// interpolation weights, the Gauss linear gradient, the explicit
// non-orthogonal correction and the right-hand side of A p = b, the flux
// reconstruction after the solve, and the integrated divergence.
//
// Per-cell results are gathers over the face-to-cell lists (no atomics):
// a cell takes its neighbour-side faces, then its owner-side faces (together
// this is ascending face order, since faces are sorted by (l, u)), then its
// boundary faces in ascending order, each contribution rounded as in the
// sequential face loop, so every result is bit-identical to it.
#include <algorithm>

#include "common.cuh"

namespace spuma {

spuma_status scan_exclusive_ext(const int* in, int64_t n, int* out, int* tmp, cudaStream_t s);

static int grid_fv(int64_t work, int threads, int num_sms)
{
    int64_t g = (work + threads - 1) / threads;
    g = std::min<int64_t>(g, (int64_t)num_sms * 16);
    return (int)std::max<int64_t>(g, 1);
}

// w_f = |S.(C_u - C_f)| / (|S.(C_f - C_l)| + |S.(C_u - C_f)|): the weight of
// the owner value in the linear interpolation p_f = w p_l + (1 - w) p_u.
__global__ void k_fv_weights(int nf, const int* __restrict__ l, const int* __restrict__ u,
                             const double* __restrict__ sf, const double* __restrict__ cf,
                             const double* __restrict__ c, double* __restrict__ w)
{
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
        const double* s = sf + 3 * (size_t)f;
        const double* x = cf + 3 * (size_t)f;
        const double* cl = c + 3 * (size_t)l[f];
        const double* cu = c + 3 * (size_t)u[f];
        const double own = fabs(__dadd_rn(__dadd_rn(__dmul_rn(s[0], __dsub_rn(x[0], cl[0])),
                                                    __dmul_rn(s[1], __dsub_rn(x[1], cl[1]))),
                                          __dmul_rn(s[2], __dsub_rn(x[2], cl[2]))));
        const double nei = fabs(__dadd_rn(__dadd_rn(__dmul_rn(s[0], __dsub_rn(cu[0], x[0])),
                                                    __dmul_rn(s[1], __dsub_rn(cu[1], x[1]))),
                                          __dmul_rn(s[2], __dsub_rn(cu[2], x[2]))));
        w[f] = __ddiv_rn(nei, __dadd_rn(own, nei));
    }
}

// Per-cell lists of all boundary faces, ascending within each cell.
__global__ void k_fv_bcount(int nb, const int* __restrict__ bcell, int* cnt)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x)
        atomicAdd(cnt + bcell[b], 1);
}
__global__ void k_fv_bfill(int nb, const int* __restrict__ bcell, int* cursor, int* blist)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x)
        blist[atomicAdd(cursor + bcell[b], 1)] = b;
}
__global__ void k_fv_bsort(int n, const int* __restrict__ bstart, int* blist)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int b0 = bstart[i], b1 = bstart[i + 1];
        for (int k = b0 + 1; k < b1; k++) {
            const int v = blist[k];
            int j = k - 1;
            while (j >= b0 && blist[j] > v) {
                blist[j + 1] = blist[j];
                j--;
            }
            blist[j + 1] = v;
        }
    }
}

// Gauss linear gradient, in two passes.  Face pass (face order, coalesced):
// t_f = S_f p_f with p_f = w p_l + (1 - w) p_u, each component a rounded
// product, padded to 32 bytes (one sector per face).  Cell pass: grad_i =
// (1/V_i) (sum over the neighbour-side faces of -t_f, then the owner-side
// faces of +t_f, ascending face order, then S_b p_b over the boundary faces,
// p_b = 0 on Dirichlet faces, p_i on zero-gradient ones).  The sequential
// loop computes the same p_f and S_f p_f from either side of a face, so the
// result is bit-identical to it.
__global__ void __launch_bounds__(256, 8) k_fv_grad_face(int nf, const int* __restrict__ l,
                                                         const int* __restrict__ u, const double* __restrict__ sf,
                                                         const double* __restrict__ w, const double* __restrict__ p,
                                                         double4* __restrict__ t)
{
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
        const double wf = w[f];
        const double pf = __dadd_rn(__dmul_rn(wf, p[l[f]]), __dmul_rn(__dsub_rn(1.0, wf), p[u[f]]));
        const double* s = sf + 3 * (size_t)f;
        t[f] = make_double4(__dmul_rn(s[0], pf), __dmul_rn(s[1], pf), __dmul_rn(s[2], pf), 0.0);
    }
}

// one 32-byte face record of the gradient's face pass, evict-first
__device__ __forceinline__ double4 ld_t4(const double4* t, int f)
{
    const double2* q = reinterpret_cast<const double2*>(t + f);
    const double2 a = __ldcs(q), b = __ldcs(q + 1);
    return make_double4(a.x, a.y, b.x, b.y);
}

__global__ void __launch_bounds__(256, 6) k_fv_grad_cell(int n, const int* __restrict__ lo_start,
                                                         const int* __restrict__ lo_face,
                                                         const int* __restrict__ own_start,
                                                         const double4* __restrict__ t, const double* __restrict__ p,
                                                         const int* __restrict__ bstart, const int* __restrict__ blist,
                                                         const double* __restrict__ bsf,
                                                         const int8_t* __restrict__ btype,
                                                         const double* __restrict__ v, double* __restrict__ grad)
{
    // a cell's faces as one list (neighbour side, then owner side: ascending
    // face order) in groups of G, so that an interior hex cell (six faces,
    // two full groups) issues no idle sums: GB300's FP64 pipe, not memory,
    // bounds these kernels, and a predicated-off FP64 add costs as much as a
    // live one (G = 3 keeps the records within 32 registers)
    constexpr int G = 3;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int k0 = lo_start[i], nl = lo_start[i + 1] - k0, f0 = own_start[i], nt = nl + own_start[i + 1] - f0;
        double gx = 0.0, gy = 0.0, gz = 0.0;
        for (int jb = 0; jb < nt; jb += G) {
            double4 tv[G];
#pragma unroll
            for (int j = 0; j < G; j++) {
                const int e = jb + j;
                if (e < nt) {
                    const double4 q = ld_t4(t, e < nl ? __ldcs(lo_face + k0 + e) : f0 + (e - nl));
                    // i = u(f): -t_f (an exact negation), i = l(f): +t_f
                    tv[j] = e < nl ? make_double4(-q.x, -q.y, -q.z, 0.0) : q;
                } else {
                    tv[j] = make_double4(0.0, 0.0, 0.0, 0.0);
                }
            }
#pragma unroll
            for (int j = 0; j < G; j++)
                if (jb + j < nt) {
                    gx = __dadd_rn(gx, tv[j].x);
                    gy = __dadd_rn(gy, tv[j].y);
                    gz = __dadd_rn(gz, tv[j].z);
                }
        }
        if (bstart) {
            const double pi = p[i];
            for (int k = bstart[i]; k < bstart[i + 1]; k++) {
                const int b = blist[k];
                const double pb = btype[b] == 1 ? 0.0 : pi;
                gx = __dadd_rn(gx, __dmul_rn(bsf[3 * (size_t)b + 0], pb));
                gy = __dadd_rn(gy, __dmul_rn(bsf[3 * (size_t)b + 1], pb));
                gz = __dadd_rn(gz, __dmul_rn(bsf[3 * (size_t)b + 2], pb));
            }
        }
        const double vi = v[i];
        grad[3 * (size_t)i + 0] = __ddiv_rn(gx, vi);
        grad[3 * (size_t)i + 1] = __ddiv_rn(gy, vi);
        grad[3 * (size_t)i + 2] = __ddiv_rn(gz, vi);
    }
}

// The same two cell passes over the fixed-width face lists (entry j of cell
// i at FL[j n + i]: -(f + 1) neighbour side, f + 1 owner side, 0 padding; the
// neighbour-side faces first, each side ascending: the face order): a
// thread's face indices arrive in W coalesced loads with no extents to load
// first, then its values in one gather round.
__device__ __forceinline__ int fl_face(int v) { return v > 0 ? v - 1 : -v - 1; }

// Exact negation (the sign bit flipped) when neg, on the integer pipe: GB300
// issues FP64 instructions at a small fraction of its integer rate, and a
// floating-point negation or select would take an FP64 issue slot.
__device__ __forceinline__ double flip_sign(double q, bool neg)
{
    return __longlong_as_double(__double_as_longlong(q) ^ (neg ? (long long)0x8000000000000000ull : 0ll));
}

template <int W>
__global__ void __launch_bounds__(256, 6) k_fv_grad_cell_fl(int n, int w, const int* __restrict__ FL,
                                                            const double4* __restrict__ t,
                                                            const double* __restrict__ p,
                                                            const int* __restrict__ bstart,
                                                            const int* __restrict__ blist,
                                                            const double* __restrict__ bsf,
                                                            const int8_t* __restrict__ btype,
                                                            const double* __restrict__ v, double* __restrict__ grad)
{
    constexpr int H = (W + 1) / 2;   // records gathered in two rounds of H (registers)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int e[W];   // the list's width w <= W columns; the rest read as padding
#pragma unroll
        for (int j = 0; j < W; j++) e[j] = j < w ? __ldcs(FL + (size_t)j * n + i) : 0;
        double gx = 0.0, gy = 0.0, gz = 0.0;
#pragma unroll
        for (int h = 0; h < W; h += H) {
            double4 tv[H];
#pragma unroll
            for (int j = 0; j < H; j++) {
                const int ej = h + j < W ? e[h + j] : 0;
                const double4 q = ej != 0 ? ld_t4(t, fl_face(ej)) : make_double4(0.0, 0.0, 0.0, 0.0);
                tv[j] = make_double4(flip_sign(q.x, ej < 0), flip_sign(q.y, ej < 0), flip_sign(q.z, ej < 0), 0.0);
            }
#pragma unroll
            for (int j = 0; j < H; j++)
                if (h + j < W && e[h + j] != 0) {
                    gx = __dadd_rn(gx, tv[j].x);
                    gy = __dadd_rn(gy, tv[j].y);
                    gz = __dadd_rn(gz, tv[j].z);
                }
        }
        if (bstart) {
            const double pi = p[i];
            for (int k = bstart[i]; k < bstart[i + 1]; k++) {
                const int b = blist[k];
                const double pb = btype[b] == 1 ? 0.0 : pi;
                gx = __dadd_rn(gx, __dmul_rn(bsf[3 * (size_t)b + 0], pb));
                gy = __dadd_rn(gy, __dmul_rn(bsf[3 * (size_t)b + 1], pb));
                gz = __dadd_rn(gz, __dmul_rn(bsf[3 * (size_t)b + 2], pb));
            }
        }
        const double vi = v[i];
        grad[3 * (size_t)i + 0] = __ddiv_rn(gx, vi);
        grad[3 * (size_t)i + 1] = __ddiv_rn(gy, vi);
        grad[3 * (size_t)i + 2] = __ddiv_rn(gz, vi);
    }
}

template <int W>
__global__ void __launch_bounds__(256, 8) k_fv_cell_sum_fl(int n, int w, const int* __restrict__ FL,
                                                           const double* __restrict__ val,
                                                           const int* __restrict__ bstart,
                                                           const int* __restrict__ blist,
                                                           const double* __restrict__ bphi, int bsign,
                                                           double* __restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int e[W];   // the list's width w <= W columns; the rest read as padding
#pragma unroll
        for (int j = 0; j < W; j++) e[j] = j < w ? __ldcs(FL + (size_t)j * n + i) : 0;
        double t[W];
#pragma unroll
        for (int j = 0; j < W; j++) {
            const double q = e[j] != 0 ? __ldcs(val + fl_face(e[j])) : 0.0;
            t[j] = flip_sign(q, e[j] < 0);   // the neighbour side subtracts
        }
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < W; j++)
            if (e[j] != 0) acc = __dadd_rn(acc, t[j]);
        if (bstart) {
            if (bsign < 0)
                for (int k = bstart[i]; k < bstart[i + 1]; k++) acc = __dsub_rn(acc, bphi[blist[k]]);
            else
                for (int k = bstart[i]; k < bstart[i + 1]; k++) acc = __dadd_rn(acc, bphi[blist[k]]);
        }
        __stcs(out + i, acc);
    }
}

// Explicit non-orthogonal correction flux of the corrected laplacian:
// corr_f = (gamma_f |S|) (k . (w grad_l + (1 - w) grad_u)), k = S/|S| - d delta,
// delta = 1/max(n.d, 0.05 |d|) (the implicit part's coefficient).
// dcp_f = corr_f - phi_f as well, the face term of the right-hand side.
__global__ void k_fv_corr(int nf, const int* __restrict__ l, const int* __restrict__ u,
                          const double* __restrict__ sf, const double* __restrict__ c,
                          const double* __restrict__ w, const double* __restrict__ gamma,
                          const double* __restrict__ grad, const double* __restrict__ phi, double* __restrict__ corr,
                          double* __restrict__ dcp)
{
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
        const double* s = sf + 3 * (size_t)f;
        const double* cl = c + 3 * (size_t)l[f];
        const double* cu = c + 3 * (size_t)u[f];
        const double* gl = grad + 3 * (size_t)l[f];
        const double* gu = grad + 3 * (size_t)u[f];
        const double dx = __dsub_rn(cu[0], cl[0]), dy = __dsub_rn(cu[1], cl[1]), dz = __dsub_rn(cu[2], cl[2]);
        const double mags =
            __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(s[0], s[0]), __dmul_rn(s[1], s[1])), __dmul_rn(s[2], s[2])));
        const double magd = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
        const double ndotd =
            __ddiv_rn(__dadd_rn(__dadd_rn(__dmul_rn(s[0], dx), __dmul_rn(s[1], dy)), __dmul_rn(s[2], dz)), mags);
        const double delta = __ddiv_rn(1.0, fmax(ndotd, __dmul_rn(0.05, magd)));
        const double kx = __dsub_rn(__ddiv_rn(s[0], mags), __dmul_rn(dx, delta));
        const double ky = __dsub_rn(__ddiv_rn(s[1], mags), __dmul_rn(dy, delta));
        const double kz = __dsub_rn(__ddiv_rn(s[2], mags), __dmul_rn(dz, delta));
        const double wf = w[f], wu = __dsub_rn(1.0, wf);
        const double gx = __dadd_rn(__dmul_rn(wf, gl[0]), __dmul_rn(wu, gu[0]));
        const double gy = __dadd_rn(__dmul_rn(wf, gl[1]), __dmul_rn(wu, gu[1]));
        const double gz = __dadd_rn(__dmul_rn(wf, gl[2]), __dmul_rn(wu, gu[2]));
        const double cf = __dmul_rn(__dmul_rn(gamma[f], mags),
                                    __dadd_rn(__dadd_rn(__dmul_rn(kx, gx), __dmul_rn(ky, gy)), __dmul_rn(kz, gz)));
        corr[f] = cf;
        dcp[f] = __dsub_rn(cf, phi[f]);
    }
}

// out_i = sum over the faces of i of -val_f (neighbour side) and +val_f
// (owner side), ascending face order, then over its boundary faces of
// bsign bphi_b.  Right-hand side: val = corr - phi, bsign = -1 (A p = b for
// laplacian(gamma, p) = div(phiHbyA), A = -(implicit laplacian)); integrated
// divergence: val = phi, bsign = +1.  All loads of a group of faces are
// issued together, the sums taken in order.
__global__ void __launch_bounds__(256, 8) k_fv_cell_sum(int n, const int* __restrict__ lo_start,
                                                        const int* __restrict__ lo_face,
                                                        const int* __restrict__ own_start,
                                                        const double* __restrict__ val,
                                                        const int* __restrict__ bstart, const int* __restrict__ blist,
                                                        const double* __restrict__ bphi, int bsign,
                                                        double* __restrict__ out)
{
    // one list per cell (neighbour side, then owner side), groups of G: an
    // interior hex cell issues its six FP64 adds once (see k_fv_grad_cell)
    constexpr int G = 6;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int k0 = lo_start[i], nl = lo_start[i + 1] - k0, f0 = own_start[i], nt = nl + own_start[i + 1] - f0;
        double acc = 0.0;
        for (int jb = 0; jb < nt; jb += G) {
            double t[G];
#pragma unroll
            for (int j = 0; j < G; j++) {
                const int e = jb + j;
                if (e < nt) {
                    const double q = __ldcs(val + (e < nl ? __ldcs(lo_face + k0 + e) : f0 + (e - nl)));
                    t[j] = e < nl ? -q : q;   // neighbour side subtracts (an exact negation)
                } else {
                    t[j] = 0.0;
                }
            }
#pragma unroll
            for (int j = 0; j < G; j++)
                if (jb + j < nt) acc = __dadd_rn(acc, t[j]);
        }
        if (bstart) {
            if (bsign < 0)
                for (int k = bstart[i]; k < bstart[i + 1]; k++) acc = __dsub_rn(acc, bphi[blist[k]]);
            else
                for (int k = bstart[i]; k < bstart[i + 1]; k++) acc = __dadd_rn(acc, bphi[blist[k]]);
        }
        __stcs(out + i, acc);
    }
}

// Cell sums of one face array over whichever face lists the handle has.
static void launch_cell_sum(spuma_ldu_t h, const double* val, const int* bstart, const int* blist,
                            const double* bphi, int bsign, double* out, cudaStream_t s)
{
    const Layout& L = h->L;
    const int g = std::min(grid_fv(h->n, 256, h->num_sms), h->num_sms * 8);
    if (h->ell_w > 0 && h->ell_w <= 6)
        k_fv_cell_sum_fl<6><<<g, 256, 0, s>>>(h->n, h->ell_w, h->at<int>(L.FL), val, bstart, blist, bphi, bsign, out);
    else
        k_fv_cell_sum<<<g, 256, 0, s>>>(h->n, h->at<int>(L.lo_start), h->at<int>(L.lo_face), h->at<int>(L.own_start),
                                        val, bstart, blist, bphi, bsign, out);
    count_launch();
}

// phi_f = phiHbyA_f - (a_f (p_u - p_l) + corr_f), a_f = -upper_f.
__global__ void k_fv_flux(int nf, const int* __restrict__ l, const int* __restrict__ u,
                          const double* __restrict__ upper, const double* __restrict__ corr,
                          const double* __restrict__ p, const double* __restrict__ phi, double* __restrict__ out)
{
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x)
        out[f] = __dsub_rn(phi[f], __dadd_rn(__dmul_rn(-upper[f], __dsub_rn(p[u[f]], p[l[f]])), corr[f]));
}

// Boundary: Dirichlet phi_b = phiHbyA_b + a_b p_cell (a_b the assembly's
// boundary coefficient), zero gradient phiHbyA_b.
__global__ void k_fv_bflux(int nb, const int* __restrict__ bcell, const int8_t* __restrict__ btype,
                           const double* __restrict__ bsf, const double* __restrict__ bcf,
                           const double* __restrict__ bgamma, const double* __restrict__ c,
                           const double* __restrict__ p, const double* __restrict__ bphi, double* __restrict__ out)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        if (btype[b] != 1) {
            out[b] = bphi[b];
            continue;
        }
        const int i = bcell[b];
        const double* s = bsf + 3 * (size_t)b;
        const double* cb = bcf + 3 * (size_t)b;
        const double* ci = c + 3 * (size_t)i;
        const double ab = face_coeff(s[0], s[1], s[2], __dsub_rn(cb[0], ci[0]), __dsub_rn(cb[1], ci[1]),
                                     __dsub_rn(cb[2], ci[2]), bgamma[b]);
        out[b] = __dadd_rn(bphi[b], __dmul_rn(ab, p[i]));
    }
}

// Per-cell boundary lists: bstart[n+1], blist[nb].  Built once per boundary
// (bface_cell pointer and count) into the handle's boundary region and reused
// by later calls; a boundary with more than 2 faces per cell on average is
// built on every call into the (idle) vector region instead.
static spuma_status boundary_lists(spuma_ldu_t h, int nb, const int* bcell, int** bstart_out, int** blist_out,
                                   cudaStream_t s)
{
    *bstart_out = nullptr;
    *blist_out = nullptr;
    if (nb <= 0) return SPUMA_OK;
    if ((int64_t)nb > 10LL * h->n) {
        set_error("more than 10 boundary faces per cell");
        return SPUMA_ERR_WORKSPACE_TOO_SMALL;
    }
    const Layout& L = h->L;
    const bool cached = (size_t)nb <= L.blist_cap;
    int* bstart = cached ? h->at<int>(L.bstart) : h->at<int>(L.x64);
    int* blist = cached ? h->at<int>(L.blist) : h->at<int>(L.p64);
    *bstart_out = bstart;
    *blist_out = blist;
    if (cached && h->bl_cell == bcell && h->bl_nb == nb) return SPUMA_OK;
    const int T = 256;
    int* cursor = h->at<int>(L.r64);
    int* tmp = h->at<int>(L.w64);
    SPUMA_CUDA(cudaMemsetAsync(bstart, 0, 4 * (size_t)(h->n + 1), s));
    k_fv_bcount<<<grid_fv(nb, T, h->num_sms), T, 0, s>>>(nb, bcell, bstart);
    count_launch();
    spuma_status st = scan_exclusive_ext(bstart, h->n, bstart, tmp, s);
    if (st != SPUMA_OK) return st;
    SPUMA_CUDA(cudaMemcpyAsync(cursor, bstart, 4 * (size_t)h->n, cudaMemcpyDeviceToDevice, s));
    k_fv_bfill<<<grid_fv(nb, T, h->num_sms), T, 0, s>>>(nb, bcell, cursor, blist);
    k_fv_bsort<<<grid_fv(h->n, T, h->num_sms), T, 0, s>>>(h->n, bstart, blist);
    count_launch(2);
    SPUMA_CUDA(cudaGetLastError());
    if (cached) {
        h->bl_cell = bcell;
        h->bl_nb = nb;
    }
    return SPUMA_OK;
}

// Face-indexed scratch of the operators: the matrix region (La64 .. Uc64,
// 32F bytes at least); a matrix prepared with spuma_matrix_prepare() is no
// longer valid afterwards.
static char* face_scratch(spuma_ldu_t h)
{
    h->prepared_precond = -1;
    return h->at<char>(h->L.La64);
}

}  // namespace spuma

using namespace spuma;

extern "C" {

spuma_status spuma_fv_weights(spuma_ldu_t h, const double* face_sf, const double* face_cf, const double* cell_c,
                              double* w, spuma_stream_t stream)
{
    if (!h || (h->nf > 0 && (!face_sf || !face_cf || !cell_c || !w))) {
        set_error("spuma_fv_weights: bad argument");
        return SPUMA_ERR_INVALID_ARG;
    }
    if (h->nf == 0) return SPUMA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_fv_weights<<<grid_fv(h->nf, 256, h->num_sms), 256, 0, s>>>(h->nf, h->at<int>(h->L.laddr),
                                                                 h->at<int>(h->L.uaddr), face_sf, face_cf, cell_c, w);
    count_launch();
    SPUMA_CUDA(cudaGetLastError());
    return SPUMA_OK;
}

spuma_status spuma_fv_grad(spuma_ldu_t h, const double* face_sf, const double* w, const double* cell_v,
                           int32_t n_bfaces, const int32_t* bface_cell, const double* bface_sf,
                           const int8_t* bface_type, const double* p, double* grad, spuma_stream_t stream)
{
    if (!h || n_bfaces < 0 || (h->n > 0 && (!cell_v || !p || !grad)) || (h->nf > 0 && (!face_sf || !w)) ||
        (n_bfaces > 0 && (!bface_cell || !bface_sf || !bface_type))) {
        set_error("spuma_fv_grad: bad argument");
        return SPUMA_ERR_INVALID_ARG;
    }
    if (h->n == 0) return SPUMA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int *bstart, *blist;
    spuma_status st = boundary_lists(h, n_bfaces, bface_cell, &bstart, &blist, s);
    if (st != SPUMA_OK) return st;
    const Layout& L = h->L;
    double4* t = reinterpret_cast<double4*>(face_scratch(h));
    if (h->nf > 0) {
        k_fv_grad_face<<<std::min(grid_fv(h->nf, 256, h->num_sms), h->num_sms * 8), 256, 0, s>>>(
            h->nf, h->at<int>(L.laddr), h->at<int>(L.uaddr), face_sf, w, p, t);
        count_launch();
    }
    const int gc = std::min(grid_fv(h->n, 256, h->num_sms), h->num_sms * 6);
    if (h->ell_w > 0 && h->ell_w <= 6)
        k_fv_grad_cell_fl<6><<<gc, 256, 0, s>>>(h->n, h->ell_w, h->at<int>(L.FL), t, p, bstart, blist, bface_sf,
                                                bface_type, cell_v, grad);
    else
        k_fv_grad_cell<<<gc, 256, 0, s>>>(h->n, h->at<int>(L.lo_start), h->at<int>(L.lo_face),
                                          h->at<int>(L.own_start), t, p, bstart, blist, bface_sf, bface_type, cell_v,
                                          grad);
    count_launch();
    SPUMA_CUDA(cudaGetLastError());
    return SPUMA_OK;
}

spuma_status spuma_pressure_rhs(spuma_ldu_t h, const double* face_sf, const double* cell_c, const double* w,
                                const double* face_gamma, const double* grad, const double* phi,
                                int32_t n_bfaces, const int32_t* bface_cell, const double* bphi, double* corr,
                                double* b, spuma_stream_t stream)
{
    if (!h || n_bfaces < 0 || (h->n > 0 && (!cell_c || !grad || !b)) ||
        (h->nf > 0 && (!face_sf || !w || !face_gamma || !phi || !corr)) || (n_bfaces > 0 && (!bface_cell || !bphi))) {
        set_error("spuma_pressure_rhs: bad argument");
        return SPUMA_ERR_INVALID_ARG;
    }
    if (h->n == 0) return SPUMA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const Layout& L = h->L;
    double* dcp = reinterpret_cast<double*>(face_scratch(h));
    if (h->nf > 0) {
        k_fv_corr<<<grid_fv(h->nf, 256, h->num_sms), 256, 0, s>>>(h->nf, h->at<int>(L.laddr), h->at<int>(L.uaddr),
                                                                  face_sf, cell_c, w, face_gamma, grad, phi, corr,
                                                                  dcp);
        count_launch();
    }
    int *bstart, *blist;
    spuma_status st = boundary_lists(h, n_bfaces, bface_cell, &bstart, &blist, s);
    if (st != SPUMA_OK) return st;
    launch_cell_sum(h, dcp, bstart, blist, bphi, -1, b, s);
    SPUMA_CUDA(cudaGetLastError());
    return SPUMA_OK;
}

spuma_status spuma_pressure_flux(spuma_ldu_t h, const double* upper, const double* corr, const double* p,
                                 const double* phi, int32_t n_bfaces, const int32_t* bface_cell,
                                 const double* bface_sf, const double* bface_cf, const double* bface_gamma,
                                 const int8_t* bface_type, const double* cell_c, const double* bphi,
                                 double* phi_out, double* bphi_out, spuma_stream_t stream)
{
    if (!h || n_bfaces < 0 || (h->n > 0 && !p) || (h->nf > 0 && (!upper || !corr || !phi || !phi_out)) ||
        (n_bfaces > 0 && (!bface_cell || !bface_sf || !bface_cf || !bface_gamma || !bface_type || !cell_c ||
                          !bphi || !bphi_out))) {
        set_error("spuma_pressure_flux: bad argument");
        return SPUMA_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const Layout& L = h->L;
    if (h->nf > 0) {
        k_fv_flux<<<grid_fv(h->nf, 256, h->num_sms), 256, 0, s>>>(h->nf, h->at<int>(L.laddr), h->at<int>(L.uaddr),
                                                                  upper, corr, p, phi, phi_out);
        count_launch();
    }
    if (n_bfaces > 0) {
        k_fv_bflux<<<grid_fv(n_bfaces, 256, h->num_sms), 256, 0, s>>>(n_bfaces, bface_cell, bface_type, bface_sf,
                                                                      bface_cf, bface_gamma, cell_c, p, bphi, bphi_out);
        count_launch();
    }
    SPUMA_CUDA(cudaGetLastError());
    return SPUMA_OK;
}

spuma_status spuma_fv_div(spuma_ldu_t h, const double* phi, int32_t n_bfaces, const int32_t* bface_cell,
                          const double* bphi, double* div, spuma_stream_t stream)
{
    if (!h || n_bfaces < 0 || (h->n > 0 && !div) || (h->nf > 0 && !phi) || (n_bfaces > 0 && (!bface_cell || !bphi))) {
        set_error("spuma_fv_div: bad argument");
        return SPUMA_ERR_INVALID_ARG;
    }
    if (h->n == 0) return SPUMA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int *bstart, *blist;
    spuma_status st = boundary_lists(h, n_bfaces, bface_cell, &bstart, &blist, s);
    if (st != SPUMA_OK) return st;
    const Layout& L = h->L;
    launch_cell_sum(h, phi, bstart, blist, bphi, 1, div, s);
    SPUMA_CUDA(cudaGetLastError());
    return SPUMA_OK;
}

}  // extern "C"
