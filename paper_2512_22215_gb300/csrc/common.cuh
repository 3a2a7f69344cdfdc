// common.cuh -- shared device helpers, the handle and the workspace layout of
// the LDU pressure-solve library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <exception>
#include <string>
#include <vector>

#include "../../include/spuma.h"

namespace spuma {

constexpr int kMaxBlocks = 4096;       // partial-sum slots per reduction
constexpr int kEllMax = 8;             // widest row of the fixed-width Amul layout
constexpr int kSlots = 8;              // reduction slots
constexpr int kMaxBatch = 1024;        // systems per batched launch
constexpr int kWarp = 32;

// ---------------------------------------------------------------- errors --
void set_error(const std::string& msg);
spuma_status cuda_fail(cudaError_t e, const char* what);

// An entry point's body run so that no C++ exception crosses the C
// interface: a failed host allocation or thread returns SPUMA_ERR_HOST.
template <class F>
inline spuma_status host_guard(const char* where, F f)
{
    try {
        return f();
    } catch (const std::exception& e) {
        set_error(std::string(where) + ": host failure: " + e.what());
    } catch (...) {
        set_error(std::string(where) + ": host failure");
    }
    return SPUMA_ERR_HOST;
}
void count_launch(uint64_t n = 1);
uint64_t barrier_timeout_ns();

#define SPUMA_CUDA(call)                                   \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// Device status words (int32): [0] status, [1] first offending cell/face,
// [32..33] the grid barrier's 64-bit arrival word (its own 128-byte line),
// whose top bit tells every waiting block that an error was recorded.  The
// count has 63 bits: a launch makes blocks x barriers arrivals, and 2^63 is out
// of reach of any solve (a 32-bit count could carry into the error bit after
// about 12 thousand iterations on a mesh with 600 DIC levels).
enum DevStatus { DS_STATUS = 0, DS_INDEX = 1, DS_LEVELS_CHANGED = 2, DS_MAXLEVEL = 3, DS_BARRIER = 32 };
constexpr unsigned long long kErrBit = 1ull << 63;

__device__ __forceinline__ void flag_error(int* st, int code, int index)
{
    if (atomicCAS(st + DS_STATUS, 0, code) == 0) st[DS_INDEX] = index;
    __threadfence();
    atomicOr(reinterpret_cast<unsigned long long*>(st + DS_BARRIER), kErrBit);
}

// ------------------------------------------------------- memory helpers --
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long atom_add_acq_rel(unsigned long long* p, unsigned long long v)
{
    unsigned long long old;
    asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}
__device__ __forceinline__ unsigned long long global_timer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ int ld_volatile_int(const int* p)
{
    return *(const volatile int*)p;
}

// Fused multiply-add in the working precision.
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }

// --------------------------------------------------------- grid barrier --
// A group of co-resident blocks (a cooperative launch guarantees residency)
// synchronises on one arrival word that only grows during a launch: a block
// arriving as the k-th (0-based) waits until the word reaches the next
// multiple of the group size.  No generation read before arriving, no status
// reload after: an error sets the word's top bit, which ends every wait.
// Every wait is bounded by a time limit: when it expires the block records
// SPUMA_ERR_DEVICE_TIMEOUT and the caller unwinds.  Ordering needs no extra
// fence: the arrival is a gpu-scope acquire-release add made after the
// block's threads met (release is cumulative over the writes they made
// before), and the wait ends on a gpu-scope acquire load of the word that the
// last arrival's add wrote; the block's threads meet again after it.
struct Group {
    unsigned long long* word;  // arrival word (status + DS_BARRIER)
    int* status;           // device status words
    int nblocks;           // blocks in the group
    int bid;               // this block's index in the group
    unsigned long long timeout_ns;
};

// Returns true when the caller may continue (no error recorded anywhere).
__device__ __forceinline__ bool group_sync(const Group& g)
{
    __shared__ int s_err;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long old = atom_add_acq_rel(g.word, 1ull);
        bool err = (old & kErrBit) != 0;
        if (!err) {
            const unsigned long long nb = (unsigned long long)g.nblocks;
            const unsigned long long cnt = old & ~kErrBit;
            const unsigned long long target = (cnt / nb + 1ull) * nb;
            if (cnt + 1ull != target) {
                const unsigned long long t0 = global_timer_ns();
                for (;;) {
                    const unsigned long long w = ld_acquire(g.word);
                    if (w & kErrBit) {
                        err = true;
                        break;
                    }
                    if ((w & ~kErrBit) >= target) break;
                    if (global_timer_ns() - t0 > g.timeout_ns) {
                        flag_error(g.status, SPUMA_ERR_DEVICE_TIMEOUT, g.bid);
                        err = true;
                        break;
                    }
                }
            }
        }
        s_err = err ? 1 : 0;
    }
    __syncthreads();
    return s_err == 0;
}

// a = (gamma |S|) / max(n.d, 0.05 |d|), no contraction (bit-identical to the
// sequential definition).
__device__ __forceinline__ double face_coeff(double sx, double sy, double sz, double dx, double dy, double dz,
                                             double gamma)
{
    const double mags = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(sx, sx), __dmul_rn(sy, sy)), __dmul_rn(sz, sz)));
    const double magd = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
    const double ndotd =
        __ddiv_rn(__dadd_rn(__dadd_rn(__dmul_rn(sx, dx), __dmul_rn(sy, dy)), __dmul_rn(sz, dz)), mags);
    const double denom = fmax(ndotd, __dmul_rn(0.05, magd));
    return __ddiv_rn(__dmul_rn(gamma, mags), denom);
}

// ------------------------------------------------------------ reductions --
// Block-level sums of NV doubles, written as this block's partials; after a
// group_sync every block reads all partials of a slot in the same fixed order,
// so the grid-wide result is deterministic and identical in every block.
template <int NV>
__device__ __forceinline__ void block_reduce_store(double (&v)[NV], double* partials, int slot0, int bid)
{
    __shared__ double red[NV][32];
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double s = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        v[k] = s;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) red[k][warp] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) {
            double s = lane < nw ? red[k][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) partials[(size_t)(slot0 + k) * kMaxBlocks + bid] = s;
        }
    }
}

template <int NV>
__device__ __forceinline__ void block_max_store(double (&v)[NV], double* partials, int slot0, int bid)
{
    __shared__ double redm[NV][32];
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double s = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
        v[k] = s;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) redm[k][warp] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) {
            double s = lane < nw ? redm[k][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
            if (lane == 0) partials[(size_t)(slot0 + k) * kMaxBlocks + bid] = s;
        }
    }
}

// Grid-wide value of slot0..slot0+NV-1 (sum or max), broadcast to the block.
template <int NV, bool MAX = false>
__device__ __forceinline__ void grid_reduce_read(double (&out)[NV], const double* partials, int slot0, int nblocks)
{
    __shared__ double bc[NV];
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
#pragma unroll
        for (int k = 0; k < NV; k++) {
            const volatile double* ps = partials + (size_t)(slot0 + k) * kMaxBlocks;
            double s = 0.0;
            for (int j = lane; j < nblocks; j += 32) s = MAX ? fmax(s, ps[j]) : s + ps[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                double t = __shfl_xor_sync(0xffffffffu, s, o);
                s = MAX ? fmax(s, t) : s + t;
            }
            if (lane == 0) bc[k] = s;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; k++) out[k] = bc[k];
    __syncthreads();
}

// ------------------------------------------------------- internal matrix --
template <class T>
struct Mat {
    const int* Lptr;   // [n+1] lower (neighbour-side) entries of each row
    const int* Lcol;   // internal column
    const T* La;       // a_f
    const T* Lc;       // rD_row * a_f   (DIC sweep coefficient)
    const int* Uptr;   // [n+1] upper (owner-side) entries of each row
    const int* Ucol;
    const T* Ua;
    const T* Uc;
    const T* d;        // diagonal
    const T* rD;       // DIC / diagonal reciprocal
    // the Amul's entries of each row (lower ascending, then upper ascending)
    // in a column-major fixed-width layout: entry j of row p at j * ell_stride
    // + p (column -1: padding); ell_w = 0 when the mesh does not use it
    const int* Ecol;
    const T* Ea;
    int ell_w;
    int ell_stride;
};

// Workspace layout: one carve function used for sizing and for create.
struct Layout {
    size_t bytes = 0;
    // topology (int32)
    size_t perm, iperm, lvl, Lptr, Uptr, Lcol, Ucol, Lface, Uface;
    size_t own_start, lo_start, lo_face, lo_col, laddr, uaddr;
    // matrix
    size_t La64, Ua64, Lc64, Uc64, d64, rD64;
    size_t La32, Ua32, Lc32, Uc32, d32, rD32;
    // fixed-width Amul layout: ell_slots entries
    size_t ell_slots, Ecol, Ea64, Ea32;
    // the cells' faces, fixed-width column-major in original cell order (same width)
    size_t FL;
    // vectors
    size_t x64, r64, w64, p64, q64, b64;
    size_t x32, r32, w32, p32, q32;
    // control
    size_t partials, bar, status, args, clk;
    // cached per-cell boundary-face lists (pressure-step operators)
    size_t bstart, blist, blist_cap;
    // asymmetric matrices (PBiCG), present when the workspace was sized with
    // SPUMA_WORKSPACE_ASYMMETRIC: A^T's coefficients in the internal CSR, the
    // transposed DILU sweep coefficients, the transposed search direction
    size_t LaT64, UaT64, LcT64, UcT64, pT64;
    size_t EaT64;  // A^T's coefficients in the fixed-width Amul layout (A's go to Ea64)
    bool asym = false;
};

Layout make_layout(int64_t n, int64_t nf, bool asym = false);

}  // namespace spuma

// Host-side handle.
struct spuma_ldu {
    int32_t n = 0, nf = 0, nlev = 0;
    int device = 0;
    int num_sms = 0;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    spuma::Layout L;
    int prepared_precond = -1;
    const int32_t* bl_cell = nullptr;  // boundary (bface_cell pointer, count) whose lists are cached
    int32_t bl_nb = -1;
    int ell_w = 0;                     // width of the fixed-width Amul layout (0: not used)
    std::vector<int32_t> h_lvl;
    template <class T>
    T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }
};
