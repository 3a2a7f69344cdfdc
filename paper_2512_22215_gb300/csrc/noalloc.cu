// noalloc.cu -- a pressure solve that allocates no device memory.
//
// Some callers cannot call cudaMalloc: a solver plugin inside a host
// application that owns the device allocator (and forbids others from
// allocating), a code path that must not pay cudaMalloc's implicit device
// synchronisation, or a process whose device memory is fully reserved up
// front.  spuma_pcg_solve_static() serves them: its whole workspace (mesh
// topology, prepared matrix, solver vectors) lives in one file-scope device
// array of fixed size that the library image carries; the caller passes only
// the inputs and the outputs.
#include <cstdio>
#include <string>

#include "common.cuh"

namespace spuma {
spuma_status pcg_solve_internal(spuma_ldu_t h, const double* diag, const double* upper, const double* b, double* x,
                                const spuma_solver_controls* ctl, spuma_solver_perf* perf, cudaStream_t s,
                                int zero_x0);
bool ctl_ok(const spuma_solver_controls* c);
}  // namespace spuma

using namespace spuma;

// 32 MiB: enough for hex meshes of about 65 thousand cells.  Every GPU that
// loads the library holds this array until the process exits.
constexpr size_t kStaticWorkspaceBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_static_workspace[kStaticWorkspaceBytes];

// In host code the array's name is only a host-side stand-in: its device
// address is looked up with the current device, on every call (a cached
// address would outlive a reset of the device's primary context; the lookup
// costs little next to the topology build).
static spuma_status static_workspace(void** out)
{
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_workspace);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static workspace)");
    *out = p;
    return SPUMA_OK;
}

extern "C" {

size_t spuma_static_workspace_bytes(void) { return kStaticWorkspaceBytes; }

spuma_status spuma_pcg_solve_static(int32_t n_cells, int32_t n_faces, const int32_t* lower_addr,
                                    const int32_t* upper_addr, const double* diag, const double* upper,
                                    const double* b, double* x, const spuma_solver_controls* ctl,
                                    spuma_solver_perf* perf, spuma_stream_t stream)
{
    // every argument is checked before the shared array is touched, so that a
    // call that is going to be rejected never disturbs another user of it
    if (n_cells < 0 || n_faces < 0) {
        set_error("spuma_pcg_solve_static: negative size");
        return SPUMA_ERR_INVALID_ARG;
    }
    const size_t need = spuma_workspace_bytes(n_cells, n_faces, 0);
    if (need > kStaticWorkspaceBytes) {
        set_error("spuma_pcg_solve_static: this mesh needs " + std::to_string(need) +
                  " bytes of workspace; the static workspace holds " + std::to_string(kStaticWorkspaceBytes) +
                  " (use spuma_ldu_create with a caller-provided workspace)");
        return SPUMA_ERR_WORKSPACE_TOO_SMALL;
    }
    if (!ctl_ok(ctl) || (n_cells > 0 && (!diag || !b || !x)) ||
        (n_faces > 0 && (!upper || !lower_addr || !upper_addr))) {
        set_error("spuma_pcg_solve_static: bad argument (controls, or a NULL array)");
        return SPUMA_ERR_INVALID_ARG;
    }
    void* ws = nullptr;
    spuma_status st = static_workspace(&ws);
    if (st != SPUMA_OK) return st;
    spuma_ldu_t h = nullptr;
    st = spuma_ldu_create(n_cells, n_faces, lower_addr, upper_addr, ws, kStaticWorkspaceBytes, stream, &h);
    if (st != SPUMA_OK) return st;
    st = pcg_solve_internal(h, diag, upper, b, x, ctl, perf, (cudaStream_t)stream, 0);
    spuma_ldu_destroy(h);
    return st;
}

}  // extern "C"
