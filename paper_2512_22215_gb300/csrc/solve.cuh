// solve.cuh -- arguments of the persistent solver kernel (shared by the single
// and the batched launch).
#pragma once
#include "common.cuh"

namespace spuma {

enum SolveMode { MODE_PREPARE = 0, MODE_SOLVE = 1, MODE_PRECONDITION = 2 };

struct SolveArgs {
    int n, nf, nlev;
    int mode;              // SolveMode
    int precond;           // spuma_precond
    int precision;         // spuma_precision (F64 or MIXED)
    int zero_x0;           // start from x = 0 instead of reading x_orig
    int no_store;          // leave x_orig untouched (autotuner trial runs)
    int tail_from;         // levels >= tail_from are small enough for the group's first block alone
    int max_iter, min_iter, max_outer;
    double tol, rel_tol, inner_rel_tol;
    const int* lvl;        // [nlev+1] level starts (internal order)
    const int* perm;       // internal -> original
    // original-order inputs/outputs
    const double* diag_orig;
    const double* upper_orig;
    const double* lower_orig;  // asymmetric matrix (PBiCG): lower coefficients; NULL when symmetric
    const double* b_orig;
    double* x_orig;
    // internal matrix
    const int *Lptr, *Lcol, *Lface, *Uptr, *Ucol, *Uface;
    double *La64, *Ua64, *Lc64, *Uc64, *d64, *rD64;
    float *La32, *Ua32, *Lc32, *Uc32, *d32, *rD32;
    double *LaT64, *UaT64, *LcT64, *UcT64, *pT;  // asymmetric regions (NULL without them)
    double* EaT64;         // asymmetric: A^T in the fixed-width layout (A in Ea64)
    const int* Ecol;       // fixed-width Amul layout (ell_w > 0): columns, entry j of row p at j n + p
    double* Ea64;
    float* Ea32;
    int ell_w;
    // internal vectors
    double *x, *r, *w, *p, *q, *b;
    float *xi, *ri, *wi, *pi, *qi;
    // control
    double* partials;
    unsigned* bar;
    int* status;
    spuma_solver_perf* perf;
    long long* phase_clk;  // optional per-phase SM-clock totals of group block 0 (diagnostics)
    int sweep;             // DIC sweep row mapping: 1 contiguous level chunks per block, 0 strided
    int amul_chunks;       // the Amul phase walks each block's chunk of every level (levels wide enough)
};

struct BatchTable {
    int n_sys;
    int split[257];                  // block ranges per system
    const SolveArgs* args[256];      // device copies
};

}  // namespace spuma
