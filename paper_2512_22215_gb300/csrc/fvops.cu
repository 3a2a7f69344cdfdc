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

// Gauss linear gradient: grad_i = (1/V_i) sum_f S_f p_f with the outward S
// (+S_f for the owner, -S_f for the neighbour); boundary p_b = 0 on
// Dirichlet faces, p_cell on zero-gradient ones.
__global__ void k_fv_grad(int n, const int* __restrict__ lo_start, const int* __restrict__ lo_face,
                          const int* __restrict__ own_start, const int* __restrict__ l, const int* __restrict__ u,
                          const double* __restrict__ sf, const double* __restrict__ w, const double* __restrict__ p,
                          const int* __restrict__ bstart, const int* __restrict__ blist,
                          const double* __restrict__ bsf, const int8_t* __restrict__ btype,
                          const double* __restrict__ v, double* __restrict__ grad)
{
    constexpr int G = 4;   // faces whose loads are issued together
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double g[3] = {0.0, 0.0, 0.0};
        const double pi = p[i];
        const int k1 = lo_start[i + 1];
        for (int k0 = lo_start[i]; k0 < k1; k0 += G) {   // i = u(f)
            int f[G];
            double wf[G], po[G], s[G][3];
#pragma unroll
            for (int j = 0; j < G; j++) f[j] = k0 + j < k1 ? lo_face[k0 + j] : -1;
#pragma unroll
            for (int j = 0; j < G; j++) {
                const bool ok = f[j] >= 0;
                wf[j] = ok ? w[f[j]] : 0.0;
                po[j] = ok ? p[l[f[j]]] : 0.0;
#pragma unroll
                for (int d = 0; d < 3; d++) s[j][d] = ok ? sf[3 * (size_t)f[j] + d] : 0.0;
            }
#pragma unroll
            for (int j = 0; j < G; j++)
                if (f[j] >= 0) {
                    const double pf = __dadd_rn(__dmul_rn(wf[j], po[j]), __dmul_rn(__dsub_rn(1.0, wf[j]), pi));
#pragma unroll
                    for (int d = 0; d < 3; d++) g[d] = __dsub_rn(g[d], __dmul_rn(s[j][d], pf));
                }
        }
        const int f1 = own_start[i + 1];
        for (int f0 = own_start[i]; f0 < f1; f0 += G) {  // i = l(f)
            double wf[G], po[G], s[G][3];
#pragma unroll
            for (int j = 0; j < G; j++) {
                const int f = f0 + j;
                const bool ok = f < f1;
                wf[j] = ok ? w[f] : 0.0;
                po[j] = ok ? p[u[f]] : 0.0;
#pragma unroll
                for (int d = 0; d < 3; d++) s[j][d] = ok ? sf[3 * (size_t)f + d] : 0.0;
            }
#pragma unroll
            for (int j = 0; j < G; j++)
                if (f0 + j < f1) {
                    const double pf = __dadd_rn(__dmul_rn(wf[j], pi), __dmul_rn(__dsub_rn(1.0, wf[j]), po[j]));
#pragma unroll
                    for (int d = 0; d < 3; d++) g[d] = __dadd_rn(g[d], __dmul_rn(s[j][d], pf));
                }
        }
        if (bstart) {
            for (int k = bstart[i]; k < bstart[i + 1]; k++) {
                const int b = blist[k];
                const double pb = btype[b] == 1 ? 0.0 : pi;
#pragma unroll
                for (int d = 0; d < 3; d++) g[d] = __dadd_rn(g[d], __dmul_rn(bsf[3 * (size_t)b + d], pb));
            }
        }
        const double vi = v[i];
#pragma unroll
        for (int d = 0; d < 3; d++) grad[3 * (size_t)i + d] = __ddiv_rn(g[d], vi);
    }
}

// Explicit non-orthogonal correction flux of the corrected laplacian:
// corr_f = (gamma_f |S|) (k . (w grad_l + (1 - w) grad_u)), k = S/|S| - d delta,
// delta = 1/max(n.d, 0.05 |d|) (the implicit part's coefficient).
__global__ void k_fv_corr(int nf, const int* __restrict__ l, const int* __restrict__ u,
                          const double* __restrict__ sf, const double* __restrict__ c,
                          const double* __restrict__ w, const double* __restrict__ gamma,
                          const double* __restrict__ grad, double* __restrict__ corr)
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
        corr[f] = __dmul_rn(__dmul_rn(gamma[f], mags),
                            __dadd_rn(__dadd_rn(__dmul_rn(kx, gx), __dmul_rn(ky, gy)), __dmul_rn(kz, gz)));
    }
}

// b_i = sum over the faces of i of +-(corr_f - phi_f) (+ owner, - neighbour),
// then minus the boundary fluxes of i: A p = b for laplacian(gamma, p) =
// div(phiHbyA) with A = -(implicit laplacian).  With corr = NULL: the
// integrated divergence sum +-phi_f + boundary fluxes instead.
__global__ void k_fv_cell_sum(int n, const int* __restrict__ lo_start, const int* __restrict__ lo_face,
                              const int* __restrict__ own_start, const double* __restrict__ corr,
                              const double* __restrict__ phi, const int* __restrict__ bstart,
                              const int* __restrict__ blist, const double* __restrict__ bphi, double* __restrict__ out)
{
    constexpr int G = 4;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double acc = 0.0;
        const int k1 = lo_start[i + 1], f1 = own_start[i + 1];
        // neighbour-side faces subtract, owner-side faces add; with corr the
        // face term is corr_f - phi_f, else phi_f; loads issued G at a time
        for (int k0 = lo_start[i]; k0 < k1; k0 += G) {
            int f[G];
            double t[G];
#pragma unroll
            for (int j = 0; j < G; j++) f[j] = k0 + j < k1 ? lo_face[k0 + j] : -1;
#pragma unroll
            for (int j = 0; j < G; j++)
                t[j] = f[j] < 0 ? 0.0 : (corr ? __dsub_rn(corr[f[j]], phi[f[j]]) : phi[f[j]]);
#pragma unroll
            for (int j = 0; j < G; j++)
                if (f[j] >= 0) acc = __dsub_rn(acc, t[j]);
        }
        for (int f0 = own_start[i]; f0 < f1; f0 += G) {
            double t[G];
#pragma unroll
            for (int j = 0; j < G; j++) {
                const int f = f0 + j;
                t[j] = f >= f1 ? 0.0 : (corr ? __dsub_rn(corr[f], phi[f]) : phi[f]);
            }
#pragma unroll
            for (int j = 0; j < G; j++)
                if (f0 + j < f1) acc = __dadd_rn(acc, t[j]);
        }
        if (bstart) {
            if (corr)
                for (int k = bstart[i]; k < bstart[i + 1]; k++) acc = __dsub_rn(acc, bphi[blist[k]]);
            else
                for (int k = bstart[i]; k < bstart[i + 1]; k++) acc = __dadd_rn(acc, bphi[blist[k]]);
        }
        out[i] = acc;
    }
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

// Builds the per-cell boundary lists in the handle's (idle) vector region:
// bstart[n+1] in x64, blist[nb] from p64 on.
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
    const int T = 256;
    int* bstart = h->at<int>(L.x64);
    int* cursor = h->at<int>(L.r64);
    int* tmp = h->at<int>(L.w64);
    int* blist = h->at<int>(L.p64);
    SPUMA_CUDA(cudaMemsetAsync(bstart, 0, 4 * (size_t)(h->n + 1), s));
    k_fv_bcount<<<grid_fv(nb, T, h->num_sms), T, 0, s>>>(nb, bcell, bstart);
    count_launch();
    spuma_status st = scan_exclusive_ext(bstart, h->n, bstart, tmp, s);
    if (st != SPUMA_OK) return st;
    SPUMA_CUDA(cudaMemcpyAsync(cursor, bstart, 4 * (size_t)h->n, cudaMemcpyDeviceToDevice, s));
    k_fv_bfill<<<grid_fv(nb, T, h->num_sms), T, 0, s>>>(nb, bcell, cursor, blist);
    k_fv_bsort<<<grid_fv(h->n, T, h->num_sms), T, 0, s>>>(h->n, bstart, blist);
    count_launch(2);
    *bstart_out = bstart;
    *blist_out = blist;
    return SPUMA_OK;
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
    k_fv_grad<<<grid_fv(h->n, 256, h->num_sms), 256, 0, s>>>(
        h->n, h->at<int>(L.lo_start), h->at<int>(L.lo_face), h->at<int>(L.own_start), h->at<int>(L.laddr),
        h->at<int>(L.uaddr), face_sf, w, p, bstart, blist, bface_sf, bface_type, cell_v, grad);
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
    if (h->nf > 0) {
        k_fv_corr<<<grid_fv(h->nf, 256, h->num_sms), 256, 0, s>>>(h->nf, h->at<int>(L.laddr), h->at<int>(L.uaddr),
                                                                  face_sf, cell_c, w, face_gamma, grad, corr);
        count_launch();
    }
    int *bstart, *blist;
    spuma_status st = boundary_lists(h, n_bfaces, bface_cell, &bstart, &blist, s);
    if (st != SPUMA_OK) return st;
    k_fv_cell_sum<<<grid_fv(h->n, 256, h->num_sms), 256, 0, s>>>(h->n, h->at<int>(L.lo_start), h->at<int>(L.lo_face),
                                                                 h->at<int>(L.own_start), corr, phi, bstart, blist,
                                                                 bphi, b);
    count_launch();
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
    k_fv_cell_sum<<<grid_fv(h->n, 256, h->num_sms), 256, 0, s>>>(h->n, h->at<int>(L.lo_start), h->at<int>(L.lo_face),
                                                                 h->at<int>(L.own_start), nullptr, phi, bstart, blist,
                                                                 bphi, div);
    count_launch();
    SPUMA_CUDA(cudaGetLastError());
    return SPUMA_OK;
}

}  // extern "C"
