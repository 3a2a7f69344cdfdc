// ops.cu -- face/cell stream kernels on the caller's original ordering:
// laplacian assembly ("Gauss linear corrected"), the LDU Amul through the
// face-to-cell gather lists, and the adjoint's face gradient.
#include <algorithm>

#include "solve.cuh"

namespace spuma {

SolveArgs make_args(spuma_ldu_t h);
spuma_status launch_solve(spuma_ldu_t h, const SolveArgs& a, int threads, cudaStream_t s);
spuma_status scan_exclusive_ext(const int* in, int64_t n, int* out, int* tmp, cudaStream_t s);
spuma_status pcg_solve_internal(spuma_ldu_t h, const double* diag, const double* upper, const double* b, double* x,
                                const spuma_solver_controls* ctl, spuma_solver_perf* perf, cudaStream_t s,
                                int zero_x0);

static int grid1d(int64_t work, int threads, int num_sms)
{
    int64_t g = (work + threads - 1) / threads;
    g = std::min<int64_t>(g, (int64_t)num_sms * 16);
    return (int)std::max<int64_t>(g, 1);
}


__global__ void k_face_coeff(int nf, const int* __restrict__ l, const int* __restrict__ u,
                             const double* __restrict__ sf, const double* __restrict__ c,
                             const double* __restrict__ gamma, double* __restrict__ upper)
{
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
        const int lf = l[f], uf = u[f];
        const double* s = sf + 3 * (size_t)f;
        const double* cl = c + 3 * (size_t)lf;
        const double* cu = c + 3 * (size_t)uf;
        upper[f] = -face_coeff(s[0], s[1], s[2], __dsub_rn(cu[0], cl[0]), __dsub_rn(cu[1], cl[1]),
                               __dsub_rn(cu[2], cl[2]), gamma[f]);
    }
}

// Reverse mode of the assembly with respect to gamma: d a / d gamma is the
// face coefficient at gamma = 1 (a is linear in gamma).
__global__ void k_gamma_grad(int nf, const int* __restrict__ l, const int* __restrict__ u,
                             const double* __restrict__ sf, const double* __restrict__ c,
                             const double* __restrict__ gu, const double* __restrict__ gd, double* gg)
{
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
        const double* s = sf + 3 * (size_t)f;
        const double* cl = c + 3 * (size_t)l[f];
        const double* cu = c + 3 * (size_t)u[f];
        const double da = face_coeff(s[0], s[1], s[2], __dsub_rn(cu[0], cl[0]), __dsub_rn(cu[1], cl[1]),
                                     __dsub_rn(cu[2], cl[2]), 1.0);
        gg[f] = __dmul_rn(__dsub_rn(__dadd_rn(gd[l[f]], gd[u[f]]), gu[f]), da);
    }
}

__global__ void k_bgamma_grad(int nb, const int* __restrict__ bcell, const int8_t* __restrict__ btype,
                              const double* __restrict__ bsf, const double* __restrict__ bcf,
                              const double* __restrict__ c, const double* __restrict__ gd, double* gb)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        if (btype[b] != 1) {
            gb[b] = 0.0;
            continue;
        }
        const int i = bcell[b];
        const double* s = bsf + 3 * (size_t)b;
        const double* cb = bcf + 3 * (size_t)b;
        const double* ci = c + 3 * (size_t)i;
        const double da = face_coeff(s[0], s[1], s[2], __dsub_rn(cb[0], ci[0]), __dsub_rn(cb[1], ci[1]),
                                     __dsub_rn(cb[2], ci[2]), 1.0);
        gb[b] = __dmul_rn(gd[i], da);
    }
}

__global__ void k_bcount(int nb, const int* __restrict__ bcell, const int8_t* __restrict__ btype, int* cnt)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x)
        if (btype[b] == 1) atomicAdd(cnt + bcell[b], 1);
}

__global__ void k_bfill(int nb, const int* __restrict__ bcell, const int8_t* __restrict__ btype, int* cursor,
                        int* blist)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x)
        if (btype[b] == 1) blist[atomicAdd(cursor + bcell[b], 1)] = b;
}

// diag_i = sum over the faces of i in face order (neighbour side ascending,
// owner side ascending) of a_f = -upper_f, then the Dirichlet faces of i in
// ascending order.
__global__ void k_diag(int n, const int* __restrict__ lo_start, const int* __restrict__ lo_face,
                       const int* __restrict__ own_start, const double* __restrict__ upper,
                       const int* __restrict__ bstart, int* __restrict__ blist, const double* __restrict__ c,
                       const double* __restrict__ bsf, const double* __restrict__ bcf,
                       const double* __restrict__ bgamma, double* __restrict__ diag)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int k = lo_start[i]; k < lo_start[i + 1]; k++) d = __dadd_rn(d, -upper[lo_face[k]]);
        for (int f = own_start[i]; f < own_start[i + 1]; f++) d = __dadd_rn(d, -upper[f]);
        if (bstart) {
            const int b0 = bstart[i], b1 = bstart[i + 1];
            for (int k = b0 + 1; k < b1; k++) {   // ascending boundary-face order
                int v = blist[k], j = k - 1;
                while (j >= b0 && blist[j] > v) {
                    blist[j + 1] = blist[j];
                    j--;
                }
                blist[j + 1] = v;
            }
            for (int k = b0; k < b1; k++) {
                const int b = blist[k];
                const double* s = bsf + 3 * (size_t)b;
                const double* cb = bcf + 3 * (size_t)b;
                const double* ci = c + 3 * (size_t)i;
                d = __dadd_rn(d, face_coeff(s[0], s[1], s[2], __dsub_rn(cb[0], ci[0]), __dsub_rn(cb[1], ci[1]),
                                            __dsub_rn(cb[2], ci[2]), bgamma[b]));
            }
        }
        diag[i] = d;
    }
}

template <class T>
__global__ void k_amul_ldu(int n, const int* __restrict__ lo_start, const int* __restrict__ lo_face,
                           const int* __restrict__ lo_col, const int* __restrict__ own_start,
                           const int* __restrict__ uaddr, const T* __restrict__ diag, const T* __restrict__ upper,
                           const T* __restrict__ x, T* __restrict__ y)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T acc = mul_rn(diag[i], x[i]);
        for (int k = lo_start[i]; k < lo_start[i + 1]; k++) acc = fmadd(upper[lo_face[k]], x[lo_col[k]], acc);
        for (int f = own_start[i]; f < own_start[i + 1]; f++) acc = fmadd(upper[f], x[uaddr[f]], acc);
        y[i] = acc;
    }
}

__global__ void k_face_gradient(int nf, int n, const int* __restrict__ l, const int* __restrict__ u,
                                const double* __restrict__ lam, const double* __restrict__ x,
                                double* __restrict__ dupper, double* __restrict__ ddiag)
{
    const int stride = gridDim.x * blockDim.x;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += stride) {
        const int lf = l[f], uf = u[f];
        dupper[f] = -(lam[lf] * x[uf] + lam[uf] * x[lf]);
    }
    if (ddiag)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) ddiag[i] = -(lam[i] * x[i]);
}

}  // namespace spuma

using namespace spuma;

extern "C" {

spuma_status spuma_assemble_laplacian(spuma_ldu_t h, const double* face_sf, const double* cell_c,
                                      const double* face_gamma, int32_t n_bfaces, const int32_t* bface_cell,
                                      const double* bface_sf, const double* bface_cf, const double* bface_gamma,
                                      const int8_t* bface_type, double* upper, double* diag, spuma_stream_t stream)
{
    if (!h || n_bfaces < 0 || (h->n > 0 && (!cell_c || !diag)) || (h->nf > 0 && (!face_sf || !face_gamma || !upper)) ||
        (n_bfaces > 0 && (!bface_cell || !bface_sf || !bface_cf || !bface_gamma || !bface_type))) {
        set_error("spuma_assemble_laplacian: bad argument");
        return SPUMA_ERR_INVALID_ARG;
    }
    if (h->n == 0) return SPUMA_OK;
    // temporaries in the (idle) FP64 vector region: bstart[n+1], cursor[n], blist[<=B]
    const Layout& L = h->L;
    if ((int64_t)n_bfaces > 10LL * h->n) {
        set_error("more than 10 boundary faces per cell");
        return SPUMA_ERR_WORKSPACE_TOO_SMALL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int T = 256;
    if (h->nf > 0) {
        k_face_coeff<<<grid1d(h->nf, T, h->num_sms), T, 0, s>>>(h->nf, h->at<int>(L.laddr), h->at<int>(L.uaddr), face_sf,
                                                                cell_c, face_gamma, upper);
        count_launch();
    }
    int* bstart = nullptr;
    int* blist = nullptr;
    if (n_bfaces > 0) {
        bstart = h->at<int>(L.x64);           // n+1 ints (x64 holds 2n)
        int* cursor = h->at<int>(L.r64);      // n ints
        int* tmp = h->at<int>(L.w64);         // scan temporaries
        blist = h->at<int>(L.p64);            // <= 10n ints: p64, q64, b64, x32.. are contiguous (>= 11n ints)
        SPUMA_CUDA(cudaMemsetAsync(bstart, 0, 4 * (size_t)(h->n + 1), s));
        k_bcount<<<grid1d(n_bfaces, T, h->num_sms), T, 0, s>>>(n_bfaces, bface_cell, bface_type, bstart);
        count_launch();
        spuma_status st = scan_exclusive_ext(bstart, h->n, bstart, tmp, s);
        if (st != SPUMA_OK) return st;
        SPUMA_CUDA(cudaMemcpyAsync(cursor, bstart, 4 * (size_t)h->n, cudaMemcpyDeviceToDevice, s));
        k_bfill<<<grid1d(n_bfaces, T, h->num_sms), T, 0, s>>>(n_bfaces, bface_cell, bface_type, cursor, blist);
        count_launch();
    }
    if (h->nf > 0 || n_bfaces > 0) {
        k_diag<<<grid1d(h->n, T, h->num_sms), T, 0, s>>>(h->n, h->at<int>(L.lo_start), h->at<int>(L.lo_face),
                                                         h->at<int>(L.own_start), upper, bstart, blist, cell_c,
                                                         bface_sf, bface_cf, bface_gamma, diag);
    } else {
        SPUMA_CUDA(cudaMemsetAsync(diag, 0, 8 * (size_t)h->n, s));
    }
    count_launch();
    SPUMA_CUDA(cudaGetLastError());
    return SPUMA_OK;
}

spuma_status spuma_assemble_laplacian_adjoint(spuma_ldu_t h, const double* face_sf, const double* cell_c,
                                              int32_t n_bfaces, const int32_t* bface_cell, const double* bface_sf,
                                              const double* bface_cf, const int8_t* bface_type,
                                              const double* dldupper, const double* dlddiag, double* dldgamma,
                                              double* dldbgamma, spuma_stream_t stream)
{
    if (!h || n_bfaces < 0 || (h->n > 0 && (!cell_c || !dlddiag)) ||
        (h->nf > 0 && (!face_sf || !dldupper || !dldgamma)) ||
        (n_bfaces > 0 && dldbgamma && (!bface_cell || !bface_sf || !bface_cf || !bface_type))) {
        set_error("spuma_assemble_laplacian_adjoint: bad argument");
        return SPUMA_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int T = 256;
    const Layout& L = h->L;
    if (h->nf > 0) {
        k_gamma_grad<<<grid1d(h->nf, T, h->num_sms), T, 0, s>>>(h->nf, h->at<int>(L.laddr), h->at<int>(L.uaddr),
                                                                face_sf, cell_c, dldupper, dlddiag, dldgamma);
        count_launch();
    }
    if (n_bfaces > 0 && dldbgamma) {
        k_bgamma_grad<<<grid1d(n_bfaces, T, h->num_sms), T, 0, s>>>(n_bfaces, bface_cell, bface_type, bface_sf,
                                                                    bface_cf, cell_c, dlddiag, dldbgamma);
        count_launch();
    }
    SPUMA_CUDA(cudaGetLastError());
    return SPUMA_OK;
}

spuma_status spuma_amul(spuma_ldu_t h, int32_t precision, const void* diag, const void* upper, const void* x,
                        void* y, spuma_stream_t stream)
{
    if (!h || (precision != SPUMA_F64 && precision != SPUMA_F32) || (h->n > 0 && (!diag || !x || !y)) ||
        (h->nf > 0 && !upper)) {
        set_error("spuma_amul: bad argument");
        return SPUMA_ERR_INVALID_ARG;
    }
    if (h->n == 0) return SPUMA_OK;
    const Layout& L = h->L;
    cudaStream_t s = (cudaStream_t)stream;
    const int T = 256;
    int g = grid1d(h->n, T, h->num_sms);
    if (precision == SPUMA_F64)
        k_amul_ldu<double><<<g, T, 0, s>>>(h->n, h->at<int>(L.lo_start), h->at<int>(L.lo_face), h->at<int>(L.lo_col),
                                           h->at<int>(L.own_start), h->at<int>(L.uaddr), (const double*)diag,
                                           (const double*)upper, (const double*)x, (double*)y);
    else
        k_amul_ldu<float><<<g, T, 0, s>>>(h->n, h->at<int>(L.lo_start), h->at<int>(L.lo_face), h->at<int>(L.lo_col),
                                          h->at<int>(L.own_start), h->at<int>(L.uaddr), (const float*)diag,
                                          (const float*)upper, (const float*)x, (float*)y);
    count_launch();
    SPUMA_CUDA(cudaGetLastError());
    return SPUMA_OK;
}

spuma_status spuma_pcg_adjoint(spuma_ldu_t h, const double* diag, const double* upper, const double* x,
                               const double* dldx, double* dldb, double* dldupper, double* dlddiag,
                               const spuma_solver_controls* ctl, spuma_solver_perf* perf, spuma_stream_t stream)
{
    if (!h || !ctl || ctl->precision != SPUMA_F64 || (h->n > 0 && (!diag || !x || !dldx || !dldb)) ||
        (h->nf > 0 && (!upper || !dldupper))) {
        set_error("spuma_pcg_adjoint: bad argument (FP64 controls required)");
        return SPUMA_ERR_INVALID_ARG;
    }
    if (h->n == 0) return SPUMA_OK;
    // A lambda = dL/dx from lambda = 0 (A^T = A), written to dldb
    spuma_status st = pcg_solve_internal(h, diag, upper, dldx, dldb, ctl, perf, (cudaStream_t)stream, 1);
    if (st != SPUMA_OK) return st;
    const int T = 256;
    int g = grid1d(std::max(h->nf, h->n), T, h->num_sms);
    k_face_gradient<<<g, T, 0, (cudaStream_t)stream>>>(h->nf, h->n, h->at<int>(h->L.laddr), h->at<int>(h->L.uaddr),
                                                       dldb, x, dldupper, dlddiag);
    count_launch();
    SPUMA_CUDA(cudaGetLastError());
    return SPUMA_OK;
}

}  // extern "C"
