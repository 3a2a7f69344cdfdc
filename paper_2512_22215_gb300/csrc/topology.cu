// topology.cu -- handle creation: validation of the LDU addressing, the
// face-to-cell gather lists (CSR transpose of owner/neighbour, no atomics at
// solve time), DIC level sets and the level-ordered internal layout.
// Also the library's host-side diagnostics (status strings, last error,
// launch counter, barrier time limit).
#include <atomic>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace spuma {

// ------------------------------------------------------------ diagnostics --
static thread_local std::string g_last_error;
static std::atomic<uint64_t> g_launches{0};
static std::atomic<uint64_t> g_timeout_ns{2000000000ull};

void set_error(const std::string& msg) { g_last_error = msg; }
spuma_status cuda_fail(cudaError_t e, const char* what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return SPUMA_ERR_CUDA;
}
void count_launch(uint64_t n) { g_launches += n; }
uint64_t barrier_timeout_ns() { return g_timeout_ns.load(); }

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

Layout make_layout(int64_t n, int64_t nf, bool asym)
{
    Layout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    const size_t i4n = 4 * (size_t)n, i4n1 = 4 * (size_t)(n + 1), i4f = 4 * (size_t)nf;
    L.perm = take(i4n);
    L.iperm = take(i4n);
    L.lvl = take(i4n1);
    L.Lptr = take(i4n1);
    L.Uptr = take(i4n1);
    L.Lcol = take(i4f);
    L.Ucol = take(i4f);
    L.Lface = take(i4f);
    L.Uface = take(i4f);
    L.own_start = take(i4n1);
    L.lo_start = take(i4n1);
    L.lo_face = take(i4f);
    L.lo_col = take(i4f);
    L.laddr = take(i4f);
    L.uaddr = take(i4f);
    const size_t d8f = 8 * (size_t)nf, d8n = 8 * (size_t)n, f4f = 4 * (size_t)nf, f4n = 4 * (size_t)n;
    L.La64 = take(d8f);
    L.Ua64 = take(d8f);
    L.Lc64 = take(d8f);
    L.Uc64 = take(d8f);
    L.d64 = take(d8n);
    L.rD64 = take(d8n);
    L.La32 = take(f4f);
    L.Ua32 = take(f4f);
    L.Lc32 = take(f4f);
    L.Uc32 = take(f4f);
    L.d32 = take(f4n);
    L.rD32 = take(f4n);
    // fixed-width Amul layout: used when the widest row times n fits 2F + n
    // slots (no more than one padding slot per row on average)
    L.ell_slots = 2 * (size_t)nf + (size_t)n;
    L.Ecol = take(4 * L.ell_slots);
    L.FL = take(4 * L.ell_slots);
    L.Ea64 = take(8 * L.ell_slots);
    L.Ea32 = take(4 * L.ell_slots);
    L.x64 = take(d8n);
    L.r64 = take(d8n);
    L.w64 = take(d8n);
    L.p64 = take(d8n);
    L.q64 = take(d8n);
    L.b64 = take(d8n);
    L.x32 = take(f4n);
    L.r32 = take(f4n);
    L.w32 = take(f4n);
    L.p32 = take(f4n);
    L.q32 = take(f4n);
    L.partials = take(8 * (size_t)kMaxBlocks * kSlots);
    L.bar = take(1024);
    L.status = take(256);
    L.args = take(4096);
    L.clk = take(8 * 256);
    // per-cell boundary-face lists of the pressure-step operators, built once
    // per boundary (up to 2 boundary faces per cell on average)
    L.bstart = take(i4n1);
    L.blist_cap = 2 * (size_t)n;
    L.blist = take(4 * L.blist_cap);
    if (asym) {
        L.asym = true;
        L.LaT64 = take(d8f);
        L.UaT64 = take(d8f);
        L.LcT64 = take(d8f);
        L.UcT64 = take(d8f);
        L.pT64 = take(d8n);
        L.EaT64 = take(8 * L.ell_slots);
    }
    L.bytes = off;
    return L;
}

// ---------------------------------------------------------------- kernels --
__global__ void k_validate(int n, int nf, const int* __restrict__ l, const int* __restrict__ u, int* st)
{
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
        int lf = l[f], uf = u[f];
        bool ok = lf >= 0 && uf < n && lf < uf;
        if (ok && f > 0) {
            int lp = l[f - 1], up = u[f - 1];
            ok = (lp < lf) || (lp == lf && up < uf);
        }
        if (!ok) flag_error(st, SPUMA_ERR_NOT_UPPER_TRIANGULAR, f);
    }
}

__global__ void k_copy_count(int nf, const int* __restrict__ l, const int* __restrict__ u, int* laddr, int* uaddr,
                             int* own_cnt, int* lo_cnt)
{
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
        int lf = l[f], uf = u[f];
        laddr[f] = lf;
        uaddr[f] = uf;
        atomicAdd(own_cnt + lf, 1);
        atomicAdd(lo_cnt + uf, 1);
    }
}

// Exclusive scan of int32 (n+1 outputs: out[n] = total), three phases.
constexpr int kScanItems = 4;
constexpr int kScanThreads = 1024;
constexpr int kScanTile = kScanItems * kScanThreads;

__device__ __forceinline__ int block_exclusive_scan(int v, int* smem, int* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) smem[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int s = lane < (int)(blockDim.x >> 5) ? smem[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        smem[lane] = s;
    }
    __syncthreads();
    int excl = x - v + (warp > 0 ? smem[warp - 1] : 0);
    *total = smem[(blockDim.x >> 5) - 1];
    __syncthreads();
    return excl;
}

__global__ void k_scan_tiles(const int* __restrict__ in, int64_t n, int* tile_sums)
{
    __shared__ int sm[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++)
        if (base + k < n) s += in[base + k];
    int tot;
    block_exclusive_scan(s, sm, &tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int* tile_sums, int ntiles)
{
    __shared__ int sm[32];
    int carry = 0;
    for (int b = 0; b < ntiles; b += blockDim.x) {
        int i = b + threadIdx.x;
        int v = i < ntiles ? tile_sums[i] : 0;
        int tot;
        int e = block_exclusive_scan(v, sm, &tot);
        if (i < ntiles) tile_sums[i] = carry + e;
        carry += tot;
    }
    if (threadIdx.x == 0) tile_sums[ntiles] = carry;
}

__global__ void k_scan_apply(const int* __restrict__ in, int64_t n, const int* __restrict__ tile_sums, int* out)
{
    __shared__ int sm[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        v[k] = base + k < n ? in[base + k] : 0;
        s += v[k];
    }
    int tot;
    int e = block_exclusive_scan(s, sm, &tot) + tile_sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        if (base + k < n) out[base + k] = e;
        e += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = tile_sums[gridDim.x];
}

// out[0..n] = exclusive scan of in[0..n-1]; tmp needs ceil(n/kScanTile)+1 ints.
// in and out may alias.
static spuma_status scan_exclusive(const int* in, int64_t n, int* out, int* tmp, cudaStream_t s)
{
    int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles == 0) {
        SPUMA_CUDA(cudaMemsetAsync(out, 0, sizeof(int), s));
        return SPUMA_OK;
    }
    k_scan_tiles<<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, n, tmp);
    k_scan_sums<<<1, kScanThreads, 0, s>>>(tmp, (int)ntiles);
    k_scan_apply<<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, n, tmp, out);
    count_launch(3);
    SPUMA_CUDA(cudaGetLastError());
    return SPUMA_OK;
}

__global__ void k_fill_losort(int nf, const int* __restrict__ u, int* cursor, int* lo_face)
{
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
        int pos = atomicAdd(cursor + u[f], 1);
        lo_face[pos] = f;
    }
}

// Each row's neighbour-side faces in ascending face order (insertion sort of a
// short row), and their columns l(f).
__global__ void k_sort_losort(int n, const int* __restrict__ lo_start, int* lo_face, const int* __restrict__ l,
                              int* lo_col)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int b = lo_start[i], e = lo_start[i + 1];
        for (int k = b + 1; k < e; k++) {
            int v = lo_face[k];
            int j = k - 1;
            while (j >= b && lo_face[j] > v) {
                lo_face[j + 1] = lo_face[j];
                j--;
            }
            lo_face[j + 1] = v;
        }
        for (int k = b; k < e; k++) lo_col[k] = l[lo_face[k]];
    }
}

// level(i) = 0 without lower neighbours, else 1 + max level of the lower
// neighbours.  Monotone in-place relaxation: each thread walks a chunk of rows
// in ascending order, so chains inside a chunk settle in one pass.
constexpr int kLevelChunk = 16;
__global__ void k_level_relax(int n, const int* __restrict__ lo_start, const int* __restrict__ lo_col, int* level,
                              int* st)
{
    int nchunks = (n + kLevelChunk - 1) / kLevelChunk;
    bool changed = false;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nchunks; c += gridDim.x * blockDim.x) {
        int i0 = c * kLevelChunk, i1 = min(n, i0 + kLevelChunk);
        for (int i = i0; i < i1; i++) {
            int b = lo_start[i], e = lo_start[i + 1];
            int lv = 0;
            for (int k = b; k < e; k++) lv = max(lv, ld_volatile_int(level + lo_col[k]) + 1);
            if (lv > ld_volatile_int(level + i)) {
                *(volatile int*)(level + i) = lv;
                changed = true;
            }
        }
    }
    if (changed) st[DS_LEVELS_CHANGED] = 1;
}

__global__ void k_max_level(int n, const int* __restrict__ level, int* st)
{
    int m = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) m = max(m, level[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(st + DS_MAXLEVEL, m);
}

// Stable partition by bucket: positions 0..n-1 visit the items order[pos]
// (or pos when order is NULL); warp k owns positions [k*C, (k+1)*C).  Used
// for the partition of the rows by DIC level and for the passes of the radix
// sort of the cells by locality key.
__global__ void k_bucket_count(int n, int chunk, int nchunks, const int* __restrict__ order,
                               const int* __restrict__ bucket, int* table)
{
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int k = warp; k < nchunks; k += nwarps) {
        int i0 = k * chunk, i1 = min(n, i0 + chunk);
        for (int i = i0 + lane; i < i1; i += 32) {
            const int item = order ? order[i] : i;
            atomicAdd(table + (size_t)bucket[item] * nchunks + k, 1);
        }
    }
}

__global__ void k_bucket_scatter(int n, int chunk, int nchunks, const int* __restrict__ order,
                                 const int* __restrict__ bucket, int* table, int* out_order, int* out_pos)
{
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    int nwarps = (gridDim.x * blockDim.x) >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int k = warp; k < nchunks; k += nwarps) {
        int i0 = k * chunk, i1 = min(n, i0 + chunk);
        for (int ib = i0; ib < i1; ib += 32) {
            int i = ib + lane;
            bool act = i < i1;
            const int item = act ? (order ? order[i] : i) : 0;
            int bk = act ? bucket[item] : -1;
            unsigned am = __ballot_sync(0xffffffffu, act);
            unsigned peers = __match_any_sync(0xffffffffu, bk);
            int base = 0;
            size_t slot = (size_t)(act ? bk : 0) * nchunks + k;
            if (act) base = table[slot];
            __syncwarp();
            if (act) {
                int pos = base + __popc(peers & lt & am);
                out_order[pos] = item;
                if (out_pos) out_pos[item] = pos;
                if ((peers & lt & am) == 0) table[slot] = base + __popc(peers & am);
            }
            __syncwarp();
        }
    }
}

// Locality key of each cell: a 30-bit Morton code of its centre in the
// bounding box of all centres (10 bits per axis).
__global__ void k_bbox_partial(int n, const double* __restrict__ c, double* part)
{
    __shared__ double sm[6][32];
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int d = 0; d < 3; d++) {
            const double v = c[3 * (size_t)i + d];
            mn[d] = fmin(mn[d], v);
            mx[d] = fmax(mx[d], v);
        }
    for (int d = 0; d < 3; d++)
        for (int o = 16; o > 0; o >>= 1) {
            mn[d] = fmin(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
            mx[d] = fmax(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
        }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
        for (int d = 0; d < 3; d++) {
            sm[d][w] = mn[d];
            sm[3 + d][w] = mx[d];
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int d = 0; d < 3; d++) {
            double a = 1e300, b = -1e300;
            for (int k = 0; k < nw; k++) {
                a = fmin(a, sm[d][k]);
                b = fmax(b, sm[3 + d][k]);
            }
            part[6 * blockIdx.x + d] = a;
            part[6 * blockIdx.x + 3 + d] = b;
        }
    }
}

__device__ __forceinline__ unsigned spread3(unsigned v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void k_morton(int n, int nparts, const double* __restrict__ c, const double* __restrict__ part,
                         unsigned* key)
{
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int k = 0; k < nparts; k++)
        for (int d = 0; d < 3; d++) {
            mn[d] = fmin(mn[d], part[6 * k + d]);
            mx[d] = fmax(mx[d], part[6 * k + 3 + d]);
        }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        unsigned q[3];
        for (int d = 0; d < 3; d++) {
            const double ext = mx[d] - mn[d];
            double t = ext > 0.0 ? (c[3 * (size_t)i + d] - mn[d]) / ext : 0.0;
            int qi = (int)(t * 1024.0);
            q[d] = (unsigned)min(1023, max(0, qi));
        }
        key[i] = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
    }
}

__global__ void k_digit(int n, const unsigned* __restrict__ key, int shift, int* digit)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        digit[i] = (int)((key[i] >> shift) & 255u);
}

__global__ void k_level_starts(int nlev, int nchunks, const int* __restrict__ table, int n, int* lvl)
{
    for (int L = blockIdx.x * blockDim.x + threadIdx.x; L <= nlev; L += gridDim.x * blockDim.x)
        lvl[L] = L < nlev ? table[(size_t)L * nchunks] : n;
}

__global__ void k_internal_counts(int n, const int* __restrict__ perm, const int* __restrict__ lo_start,
                                  const int* __restrict__ own_start, int* Lcnt, int* Ucnt)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        int i = perm[p];
        Lcnt[p] = lo_start[i + 1] - lo_start[i];
        Ucnt[p] = own_start[i + 1] - own_start[i];
    }
}

__global__ void k_internal_fill(int n, const int* __restrict__ perm, const int* __restrict__ iperm,
                                const int* __restrict__ lo_start, const int* __restrict__ lo_face,
                                const int* __restrict__ lo_col, const int* __restrict__ own_start,
                                const int* __restrict__ uaddr, const int* __restrict__ Lptr,
                                const int* __restrict__ Uptr, int* Lcol, int* Lface, int* Ucol, int* Uface)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        int i = perm[p];
        int e = Lptr[p];
        for (int k = lo_start[i]; k < lo_start[i + 1]; k++, e++) {
            Lface[e] = lo_face[k];
            Lcol[e] = iperm[lo_col[k]];
        }
        e = Uptr[p];
        for (int f = own_start[i]; f < own_start[i + 1]; f++, e++) {
            Uface[e] = f;
            Ucol[e] = iperm[uaddr[f]];
        }
    }
}

// Widest row of the Amul (lower + upper entries) into *w (atomic max).
__global__ void k_row_width(int n, const int* __restrict__ Lptr, const int* __restrict__ Uptr, int* w)
{
    int m = 0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
        m = max(m, Lptr[p + 1] - Lptr[p] + Uptr[p + 1] - Uptr[p]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(w, m);
}

// Whether the fixed-width Amul layout is used for a widest row of w entries.
__host__ __device__ inline bool ell_fits(int w, int64_t n, size_t slots)
{
    return w >= 1 && w <= kEllMax && (size_t)w * (size_t)n <= slots;
}

// Columns of the fixed-width Amul layout: entry j of row p (its lower
// entries in ascending face order, then its upper ones) at j n + p, -1 past
// the row's end.  Does nothing unless the layout fits.
__global__ void k_ell_fill(int n, size_t slots, const int* __restrict__ wptr, const int* __restrict__ Lptr,
                           const int* __restrict__ Lcol, const int* __restrict__ Uptr, const int* __restrict__ Ucol,
                           int* Ecol)
{
    const int w = *wptr;
    if (!ell_fits(w, n, slots)) return;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int l0 = Lptr[p], nl = Lptr[p + 1] - l0, u0 = Uptr[p], nt = nl + Uptr[p + 1] - u0;
        for (int j = 0; j < w; j++)
            Ecol[(size_t)j * n + p] = j < nl ? Lcol[l0 + j] : (j < nt ? Ucol[u0 + j - nl] : -1);
    }
}

// The cells' faces in the same fixed-width column-major form, in the caller's
// (original) cell order, for the pressure-step operators: entry j of cell i
// at j n + i, its neighbour-side faces (ascending) then its owner-side faces
// (ascending), -(f + 1) for a face where i is the neighbour, f + 1 where it
// is the owner, 0 past the cell's end.  The width is the Amul layout's (a
// cell's face count is its row's entry count).
__global__ void k_face_list_fill(int n, size_t slots, const int* __restrict__ wptr, const int* __restrict__ lo_start,
                                 const int* __restrict__ lo_face, const int* __restrict__ own_start, int* FL)
{
    const int w = *wptr;
    if (!ell_fits(w, n, slots)) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int k0 = lo_start[i], nl = lo_start[i + 1] - k0, f0 = own_start[i], nt = nl + own_start[i + 1] - f0;
        for (int j = 0; j < w; j++)
            FL[(size_t)j * n + i] = j < nl ? -(lo_face[k0 + j] + 1) : (j < nt ? f0 + (j - nl) + 1 : 0);
    }
}

spuma_status scan_exclusive_ext(const int* in, int64_t n, int* out, int* tmp, cudaStream_t s)
{
    return scan_exclusive(in, n, out, tmp, s);
}

static int grid_for(int64_t work, int threads, int num_sms)
{
    int64_t g = (work + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms * 16;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

}  // namespace spuma

using namespace spuma;

extern "C" {

const char* spuma_status_string(int32_t s)
{
    switch (s) {
    case SPUMA_OK: return "ok";
    case SPUMA_ERR_INVALID_ARG: return "invalid argument";
    case SPUMA_ERR_NOT_UPPER_TRIANGULAR: return "addressing not upper-triangular (l < u, sorted by (l,u), in range)";
    case SPUMA_ERR_CUDA: return "CUDA runtime error";
    case SPUMA_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case SPUMA_ERR_SINGULAR: return "singular matrix (p.Ap vanished)";
    case SPUMA_ERR_NOT_SPD: return "matrix not SPD (non-positive DIC pivot)";
    case SPUMA_ERR_NONFINITE: return "non-finite input";
    case SPUMA_ERR_DEVICE_TIMEOUT: return "device grid barrier timed out";
    case SPUMA_ERR_HOST: return "host allocation or thread failed";
    default: return "unknown status";
    }
}

const char* spuma_last_error(void) { return g_last_error.c_str(); }
uint64_t spuma_launch_count(void) { return g_launches.load(); }
void spuma_set_barrier_timeout_ns(uint64_t ns) { g_timeout_ns = ns; }

size_t spuma_workspace_bytes(int32_t n_cells, int32_t n_faces, int32_t flags)
{
    if (n_cells < 0 || n_faces < 0) return 0;
    return make_layout(n_cells, n_faces, (flags & SPUMA_WORKSPACE_ASYMMETRIC) != 0).bytes;
}

spuma_status spuma_ldu_create(int32_t n, int32_t nf, const int32_t* l, const int32_t* u, void* workspace,
                              size_t workspace_bytes, spuma_stream_t stream, spuma_ldu_t* out)
{
    return spuma_ldu_create_with_centres(n, nf, l, u, nullptr, workspace, workspace_bytes, stream, out);
}

static spuma_status ldu_create(int32_t n, int32_t nf, const int32_t* l, const int32_t* u, const double* cell_c,
                               void* workspace, size_t workspace_bytes, spuma_stream_t stream, spuma_ldu_t* out);

spuma_status spuma_ldu_create_with_centres(int32_t n, int32_t nf, const int32_t* l, const int32_t* u,
                                           const double* cell_c, void* workspace, size_t workspace_bytes,
                                           spuma_stream_t stream, spuma_ldu_t* out)
{
    return host_guard("spuma_ldu_create",
                      [&] { return ldu_create(n, nf, l, u, cell_c, workspace, workspace_bytes, stream, out); });
}

static spuma_status ldu_create(int32_t n, int32_t nf, const int32_t* l, const int32_t* u, const double* cell_c,
                               void* workspace, size_t workspace_bytes, spuma_stream_t stream, spuma_ldu_t* out)
{
    if (!out) { set_error("out is NULL"); return SPUMA_ERR_INVALID_ARG; }
    *out = nullptr;
    if (n < 0 || nf < 0) { set_error("negative size"); return SPUMA_ERR_INVALID_ARG; }
    if (nf > 0 && (!l || !u)) { set_error("addressing pointer is NULL"); return SPUMA_ERR_INVALID_ARG; }
    if (!workspace) { set_error("workspace is NULL"); return SPUMA_ERR_INVALID_ARG; }
    if (((uintptr_t)workspace & 255u) != 0) { set_error("workspace must be 256-byte aligned"); return SPUMA_ERR_INVALID_ARG; }
    Layout L = make_layout(n, nf);
    {
        // the asymmetric regions follow the symmetric layout when they fit
        const Layout La = make_layout(n, nf, true);
        if (workspace_bytes >= La.bytes) L = La;
    }
    if (workspace_bytes < L.bytes) {
        set_error("workspace needs " + std::to_string(L.bytes) + " bytes");
        return SPUMA_ERR_WORKSPACE_TOO_SMALL;
    }
    if (nf > 0 && (int64_t)nf > 3LL * n * n) { set_error("more faces than cell pairs"); return SPUMA_ERR_NOT_UPPER_TRIANGULAR; }
    cudaStream_t s = (cudaStream_t)stream;
    spuma_ldu* h = new spuma_ldu();
    h->n = n;
    h->nf = nf;
    h->ws = (char*)workspace;
    h->ws_bytes = workspace_bytes;
    h->L = L;
    auto fail = [&](spuma_status st) { delete h; return st; };
    if (cudaGetDevice(&h->device) != cudaSuccess) return fail(cuda_fail(cudaGetLastError(), "cudaGetDevice"));
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);

    int* st = h->at<int>(L.status);
    int* own_start = h->at<int>(L.own_start);
    int* lo_start = h->at<int>(L.lo_start);
    int* lo_face = h->at<int>(L.lo_face);
    int* lo_col = h->at<int>(L.lo_col);
    int* laddr = h->at<int>(L.laddr);
    int* uaddr = h->at<int>(L.uaddr);
    // temporaries live in the vector/matrix regions (not yet in use)
    int* tmp_scan = h->at<int>(L.x64);               // >= 2N ints
    int* cursor = h->at<int>(L.r64);
    int* level = h->at<int>(L.w64);
    int* Lcnt = h->at<int>(L.p64);
    int* Ucnt = h->at<int>(L.q64);

    const int T = 256;
#define CHK(x) do { spuma_status s_ = (x); if (s_ != SPUMA_OK) return fail(s_); } while (0)
#define CU(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return fail(cuda_fail(e_, #x)); } while (0)
    CU(cudaMemsetAsync(st, 0, 256, s));
    CU(cudaMemsetAsync(own_start, 0, 4 * (size_t)(n + 1), s));
    CU(cudaMemsetAsync(lo_start, 0, 4 * (size_t)(n + 1), s));
    if (nf > 0) {
        k_validate<<<grid_for(nf, T, h->num_sms), T, 0, s>>>(n, nf, l, u, st);
        count_launch();
        int hst[4];
        CU(cudaMemcpyAsync(hst, st, sizeof(hst), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (hst[DS_STATUS] != 0) {
            set_error("face " + std::to_string(hst[DS_INDEX]) + " breaks l < u, range or (l,u) order");
            return fail(SPUMA_ERR_NOT_UPPER_TRIANGULAR);
        }
        k_copy_count<<<grid_for(nf, T, h->num_sms), T, 0, s>>>(nf, l, u, laddr, uaddr, own_start, lo_start);
        count_launch();
    }
    CHK(scan_exclusive(own_start, n, own_start, tmp_scan, s));
    CHK(scan_exclusive(lo_start, n, lo_start, tmp_scan, s));
    if (nf > 0) {
        CU(cudaMemcpyAsync(cursor, lo_start, 4 * (size_t)n, cudaMemcpyDeviceToDevice, s));
        k_fill_losort<<<grid_for(nf, T, h->num_sms), T, 0, s>>>(nf, u, cursor, lo_face);
        count_launch();
    }
    if (n > 0) {
        k_sort_losort<<<grid_for(n, T, h->num_sms), T, 0, s>>>(n, lo_start, lo_face, laddr, lo_col);
        count_launch();
    }

    // DIC levels
    int nlev = 0;
    if (n > 0) {
        CU(cudaMemsetAsync(level, 0, 4 * (size_t)n, s));
        int nchunks_lv = (n + kLevelChunk - 1) / kLevelChunk;
        int g = grid_for(nchunks_lv, T, h->num_sms);
        for (int64_t sweep = 0;; sweep += 8) {
            CU(cudaMemsetAsync(st + DS_LEVELS_CHANGED, 0, 4, s));
            for (int k = 0; k < 8; k++) k_level_relax<<<g, T, 0, s>>>(n, lo_start, lo_col, level, st);
            count_launch(8);
            int changed = 0;
            CU(cudaMemcpyAsync(&changed, st + DS_LEVELS_CHANGED, 4, cudaMemcpyDeviceToHost, s));
            CU(cudaStreamSynchronize(s));
            if (!changed) break;
            if (sweep > 4LL * n + 64) { set_error("level relaxation did not settle"); return fail(SPUMA_ERR_CUDA); }
        }
        k_max_level<<<grid_for(n, T, h->num_sms), T, 0, s>>>(n, level, st);
        count_launch();
        int hmax = 0;
        CU(cudaMemcpyAsync(&hmax, st + DS_MAXLEVEL, 4, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        nlev = hmax + 1;

        // Stable partitions: the count table and its scan temporaries use the
        // matrix region (48F + 24N bytes, not yet in use).
        int* table = h->at<int>(L.La64);
        const int64_t cap_ints = (int64_t)(L.x64 - L.La64) / 4;
        auto partition = [&](const int* order, const int* bucket, int nb, int* out_order, int* out_pos,
                             int* lvl_out) -> spuma_status {
            int64_t chunk = 1024;
            auto need = [&](int64_t c) {
                int64_t tab = (int64_t)nb * ((n + c - 1) / c);
                return tab + 64 + tab / kScanTile + 64;
            };
            while (need(chunk) > cap_ints && chunk < n) chunk *= 2;
            if (need(chunk) > cap_ints) { set_error("partition table does not fit"); return SPUMA_ERR_WORKSPACE_TOO_SMALL; }
            int nchunks = (int)((n + chunk - 1) / chunk);
            size_t tab_n = (size_t)nb * nchunks;
            int* tscan = table + tab_n + 64;
            SPUMA_CUDA(cudaMemsetAsync(table, 0, 4 * (tab_n + 1), s));
            int gw = grid_for((int64_t)nchunks * 32, T, h->num_sms);
            k_bucket_count<<<gw, T, 0, s>>>(n, (int)chunk, nchunks, order, bucket, table);
            count_launch();
            spuma_status ss = scan_exclusive(table, (int64_t)tab_n, table, tscan, s);
            if (ss != SPUMA_OK) return ss;
            if (lvl_out) {
                k_level_starts<<<grid_for(nb + 1, T, h->num_sms), T, 0, s>>>(nb, nchunks, table, n, lvl_out);
                count_launch();
            }
            k_bucket_scatter<<<gw, T, 0, s>>>(n, (int)chunk, nchunks, order, bucket, table, out_order, out_pos);
            count_launch();
            SPUMA_CUDA(cudaGetLastError());
            return SPUMA_OK;
        };
        // optional locality order: cells sorted by the Morton code of their
        // centre (LSD radix sort, four stable passes of 8 bits)
        const int* key_order = nullptr;
        if (cell_c) {
            unsigned* key = h->at<unsigned>(L.b64);
            int* digit = h->at<int>(L.x32);
            int* ord_a = h->at<int>(L.r32);
            int* ord_b = h->at<int>(L.w32);
            double* bbox = h->at<double>(L.q32);       // 6 doubles per partial block
            const int nparts = std::min(grid_for(n, T, h->num_sms), (int)((4 * (size_t)n) / 48));
            const int np = std::max(1, nparts);
            k_bbox_partial<<<np, T, 0, s>>>(n, cell_c, bbox);
            k_morton<<<grid_for(n, T, h->num_sms), T, 0, s>>>(n, np, cell_c, bbox, key);
            count_launch(2);
            const int* in = nullptr;
            int* outs[2] = {ord_a, ord_b};
            for (int pass = 0; pass < 4; pass++) {
                k_digit<<<grid_for(n, T, h->num_sms), T, 0, s>>>(n, key, 8 * pass, digit);
                count_launch();
                CHK(partition(in, digit, 256, outs[pass & 1], nullptr, nullptr));
                in = outs[pass & 1];
            }
            key_order = in;
        }
        int* lvl = h->at<int>(L.lvl);
        CHK(partition(key_order, level, nlev, h->at<int>(L.perm), h->at<int>(L.iperm), lvl));

        // internal CSR (level order): lower part = neighbour-side faces,
        // upper part = owner-side faces, each in ascending face order
        int* Lptr = h->at<int>(L.Lptr);
        int* Uptr = h->at<int>(L.Uptr);
        k_internal_counts<<<grid_for(n, T, h->num_sms), T, 0, s>>>(n, h->at<int>(L.perm), lo_start, own_start, Lcnt,
                                                                 Ucnt);
        count_launch();
        CHK(scan_exclusive(Lcnt, n, Lptr, tmp_scan, s));
        CHK(scan_exclusive(Ucnt, n, Uptr, tmp_scan, s));
        k_internal_fill<<<grid_for(n, T, h->num_sms), T, 0, s>>>(
            n, h->at<int>(L.perm), h->at<int>(L.iperm), lo_start, lo_face, lo_col, own_start, uaddr, Lptr, Uptr,
            h->at<int>(L.Lcol), h->at<int>(L.Lface), h->at<int>(L.Ucol), h->at<int>(L.Uface));
        count_launch();
        // fixed-width Amul layout (the widest row decides; read back below)
        int* wdev = h->at<int>(L.args);
        CU(cudaMemsetAsync(wdev, 0, sizeof(int), s));
        k_row_width<<<grid_for(n, T, h->num_sms), T, 0, s>>>(n, Lptr, Uptr, wdev);
        k_ell_fill<<<grid_for(n, T, h->num_sms), T, 0, s>>>(n, L.ell_slots, wdev, Lptr, h->at<int>(L.Lcol), Uptr,
                                                            h->at<int>(L.Ucol), h->at<int>(L.Ecol));
        k_face_list_fill<<<grid_for(n, T, h->num_sms), T, 0, s>>>(n, L.ell_slots, wdev, lo_start, lo_face, own_start,
                                                                  h->at<int>(L.FL));
        count_launch(3);
        CU(cudaMemcpyAsync(&h->ell_w, wdev, sizeof(int), cudaMemcpyDeviceToHost, s));
        h->h_lvl.resize(nlev + 1);
        CU(cudaMemcpyAsync(h->h_lvl.data(), lvl, 4 * (size_t)(nlev + 1), cudaMemcpyDeviceToHost, s));
    }
    CU(cudaMemsetAsync(h->at<char>(L.bar), 0, 1024, s));
    CU(cudaMemsetAsync(st, 0, 256, s));
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(s));
#undef CHK
#undef CU
    h->nlev = nlev;
    if (!ell_fits(h->ell_w, n, L.ell_slots)) h->ell_w = 0;
    *out = h;
    return SPUMA_OK;
}

spuma_status spuma_ldu_destroy(spuma_ldu_t h)
{
    delete h;
    return SPUMA_OK;
}

spuma_status spuma_ldu_info(spuma_ldu_t h, int32_t* n_cells, int32_t* n_faces, int32_t* n_levels)
{
    if (!h) { set_error("handle is NULL"); return SPUMA_ERR_INVALID_ARG; }
    if (n_cells) *n_cells = h->n;
    if (n_faces) *n_faces = h->nf;
    if (n_levels) *n_levels = h->nlev;
    return SPUMA_OK;
}

spuma_status spuma_ldu_device_status(spuma_ldu_t h, spuma_stream_t stream)
{
    if (!h) { set_error("handle is NULL"); return SPUMA_ERR_INVALID_ARG; }
    int hst[2] = {0, 0};
    SPUMA_CUDA(cudaMemcpyAsync(hst, h->at<int>(h->L.status), sizeof(hst), cudaMemcpyDeviceToHost,
                               (cudaStream_t)stream));
    SPUMA_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if (hst[0] != 0) set_error(std::string(spuma_status_string(hst[0])) + " (index " + std::to_string(hst[1]) + ")");
    return (spuma_status)hst[0];
}

}  // extern "C"
