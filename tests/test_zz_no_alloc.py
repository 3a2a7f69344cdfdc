"""The solve entry point that allocates no device memory, for callers that
cannot call cudaMalloc (its workspace is a static device array inside the
library).  Called through the C ABI and checked against the regular entry
point (spuma_ldu_create + spuma_pcg_solve) on two calls in a row, and against
the oracle's FP64 DIC-PCG at the same iteration count (relative solution
error within 1e-10, the FP64 bound of the other parity tests).  This file is
collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

import hexmesh

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_static_solve_matches_regular_solve_twice():
    import oracle
    from paper_2512_22215_gb300 import LduMesh, SolverControls, lib
    from paper_2512_22215_gb300._lib import check, ptr, stream_ptr
    from paper_2512_22215_gb300.core import perf_tensor, read_perf

    L = lib()
    ctl = SolverControls(precond=2, tolerance=1e-10)
    cctl = ctl.c()
    for seed, n in [(51, 18), (52, (21, 13, 9))]:
        c = hexmesh.pressure_case(n, jitter=0.2, permute=True, seed=seed, lognormal_gamma=True)
        m = c.mesh
        assert L.spuma_workspace_bytes(m.n_cells, m.n_faces, 0) <= L.spuma_static_workspace_bytes()
        up, dg = oracle.assemble_laplacian(m, c.gamma, c.bgamma, c.btype)
        lo, ua, d, u, b = _dev(m.lower), _dev(m.upper_addr), _dev(dg), _dev(up), _dev(c.b)
        # regular entry point: caller-provided workspace
        x_ref, p_ref = LduMesh(m.lower, m.upper_addr, m.n_cells).solve(d, u, b, None, ctl)
        # no-allocation entry point
        x = torch.zeros_like(b)
        perf = perf_tensor(1)
        check(L.spuma_pcg_solve_static(m.n_cells, m.n_faces, ptr(lo), ptr(ua), ptr(d), ptr(u), ptr(b), ptr(x),
                                       C.byref(cctl), ptr(perf), stream_ptr()), "spuma_pcg_solve_static")
        p = read_perf(perf)[0]
        assert p["status"] == 0 and p["converged"] == 1
        assert p["n_iter"] == p_ref["n_iter"]
        assert torch.linalg.norm(x - x_ref) <= 1e-10 * torch.linalg.norm(x_ref)
        xo, _ = oracle.pcg(m.lower, m.upper_addr, dg, up, c.b, precond=2, tol=0.0, max_iter=p["n_iter"])
        xs = x.cpu().numpy()
        assert np.linalg.norm(xs - xo) <= 1e-10 * np.linalg.norm(xo)


def test_static_solve_rejects_oversized_mesh():
    from paper_2512_22215_gb300 import SolverControls, lib
    L = lib()
    cap = L.spuma_static_workspace_bytes()
    n = 2_000_000
    assert L.spuma_workspace_bytes(n, 3 * n, 0) > cap
    cctl = SolverControls().c()
    st = L.spuma_pcg_solve_static(n, 3 * n, None, None, None, None, None, None, C.byref(cctl), None, None)
    assert st == 4
    assert b"static workspace" in L.spuma_last_error()
    # a mesh that fits, with no controls: rejected before the array is touched
    st = L.spuma_pcg_solve_static(8, 12, None, None, None, None, None, None, None, None, None)
    assert st == 1
