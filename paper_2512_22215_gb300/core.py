"""Tensor-level wrappers around the C ABI: a mesh handle that owns its
workspace tensor, solver controls, batched solves.  Marshalling only."""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import torch

from ._lib import (BATCH_ALLOW_DIRECT, BATCH_AUTOTUNE, BATCH_NO_GRAPH, F32, F64, MIXED, PERF_BYTES, PRECOND_DIC,
                   PRECOND_DILU, WORKSPACE_ASYMMETRIC, Controls, Perf,
                   SpumaError, check, lib, ptr, stream_ptr)


@dataclass
class SolverControls:
    precond: int = PRECOND_DIC
    precision: int = F64
    tolerance: float = 1e-8
    rel_tol: float = 0.0
    inner_rel_tol: float = 1e-2
    max_iter: int = 20000
    min_iter: int = 0
    max_outer: int = 30
    block_threads: int = 0

    def c(self) -> Controls:
        return Controls(self.precond, self.precision, self.tolerance, self.rel_tol, self.inner_rel_tol,
                        self.max_iter, self.min_iter, self.max_outer, self.block_threads)


def perf_tensor(n: int = 1, device="cuda") -> torch.Tensor:
    return torch.zeros(n * PERF_BYTES, dtype=torch.uint8, device=device)


def read_perf(t: torch.Tensor) -> list[dict]:
    raw = t.cpu().numpy().tobytes()
    out = []
    for k in range(len(raw) // PERF_BYTES):
        p = Perf.from_buffer_copy(raw[k * PERF_BYTES:(k + 1) * PERF_BYTES])
        out.append({f: getattr(p, f) for f, _ in Perf._fields_})
    return out


class LduMesh:
    """A mesh's LDU addressing on the device plus the library workspace."""

    def __init__(self, lower, upper_addr, n_cells: int, device="cuda", centres=None, asymmetric=False):
        L = lib()
        dev = torch.device(device)
        lower = torch.as_tensor(lower, dtype=torch.int32).to(dev).contiguous()
        upper_addr = torch.as_tensor(upper_addr, dtype=torch.int32).to(dev).contiguous()
        self.n_cells = int(n_cells)
        self.n_faces = int(lower.numel())
        self.device = dev
        nbytes = L.spuma_workspace_bytes(self.n_cells, self.n_faces, WORKSPACE_ASYMMETRIC if asymmetric else 0)
        # 256-byte alignment: the caching allocator returns 512-byte aligned blocks
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        h = C.c_void_p()
        cc = None
        if centres is not None:
            cc = torch.as_tensor(centres, dtype=torch.float64).to(dev).contiguous()
        st = L.spuma_ldu_create_with_centres(self.n_cells, self.n_faces, ptr(lower), ptr(upper_addr), ptr(cc),
                                             self._ws_ptr, nbytes, stream_ptr(), C.byref(h))
        check(st, "spuma_ldu_create")
        self.handle = h
        self.lower = lower
        self.upper_addr = upper_addr
        n, f, lv = C.c_int32(), C.c_int32(), C.c_int32()
        check(L.spuma_ldu_info(h, C.byref(n), C.byref(f), C.byref(lv)), "spuma_ldu_info")
        self.n_levels = lv.value

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                lib().spuma_ldu_destroy(h)
            except Exception:
                pass
            self.handle = None

    # ------------------------------------------------------------ ops ----
    def device_status(self) -> int:
        return lib().spuma_ldu_device_status(self.handle, stream_ptr())

    def assemble_laplacian(self, sf, c, gamma, bface_cell=None, bface_sf=None, bface_cf=None, bgamma=None,
                           btype=None):
        upper = torch.empty(self.n_faces, dtype=torch.float64, device=self.device)
        diag = torch.empty(self.n_cells, dtype=torch.float64, device=self.device)
        nb = 0 if bface_cell is None else int(bface_cell.numel())
        check(lib().spuma_assemble_laplacian(self.handle, ptr(sf), ptr(c), ptr(gamma), nb, ptr(bface_cell),
                                             ptr(bface_sf), ptr(bface_cf), ptr(bgamma), ptr(btype),
                                             ptr(upper), ptr(diag), stream_ptr()), "spuma_assemble_laplacian")
        return upper, diag

    def assemble_laplacian_adjoint(self, sf, c, dl_dupper, dl_ddiag, bface_cell=None, bface_sf=None, bface_cf=None,
                                   btype=None):
        """(dL/dgamma[F], dL/dbgamma[B] or None) from dL/dupper and dL/ddiag."""
        gg = torch.empty(self.n_faces, dtype=torch.float64, device=self.device)
        nb = 0 if bface_cell is None else int(bface_cell.numel())
        gb = torch.empty(nb, dtype=torch.float64, device=self.device) if nb else None
        check(lib().spuma_assemble_laplacian_adjoint(self.handle, ptr(sf), ptr(c), nb, ptr(bface_cell),
                                                     ptr(bface_sf), ptr(bface_cf), ptr(btype),
                                                     ptr(dl_dupper.contiguous()), ptr(dl_ddiag.contiguous()),
                                                     ptr(gg), ptr(gb), stream_ptr()),
              "spuma_assemble_laplacian_adjoint")
        return gg, gb

    # ------------------------------------------ pressure-correction step --
    def fv_weights(self, sf, cf, c):
        w = torch.empty(self.n_faces, dtype=torch.float64, device=self.device)
        check(lib().spuma_fv_weights(self.handle, ptr(sf), ptr(cf), ptr(c), ptr(w), stream_ptr()), "spuma_fv_weights")
        return w

    def fv_grad(self, sf, w, v, p, bface_cell=None, bface_sf=None, btype=None):
        g = torch.empty((self.n_cells, 3), dtype=torch.float64, device=self.device)
        nb = 0 if bface_cell is None else int(bface_cell.numel())
        check(lib().spuma_fv_grad(self.handle, ptr(sf), ptr(w), ptr(v), nb, ptr(bface_cell), ptr(bface_sf),
                                  ptr(btype), ptr(p), ptr(g), stream_ptr()), "spuma_fv_grad")
        return g

    def pressure_rhs(self, sf, c, w, gamma, grad, phi, bface_cell=None, bphi=None):
        corr = torch.empty(self.n_faces, dtype=torch.float64, device=self.device)
        b = torch.empty(self.n_cells, dtype=torch.float64, device=self.device)
        nb = 0 if bface_cell is None else int(bface_cell.numel())
        check(lib().spuma_pressure_rhs(self.handle, ptr(sf), ptr(c), ptr(w), ptr(gamma), ptr(grad), ptr(phi), nb,
                                       ptr(bface_cell), ptr(bphi), ptr(corr), ptr(b), stream_ptr()),
              "spuma_pressure_rhs")
        return corr, b

    def pressure_flux(self, upper, corr, p, phi, c, bface_cell=None, bface_sf=None, bface_cf=None, bgamma=None,
                      btype=None, bphi=None):
        out = torch.empty(self.n_faces, dtype=torch.float64, device=self.device)
        nb = 0 if bface_cell is None else int(bface_cell.numel())
        bout = torch.empty(nb, dtype=torch.float64, device=self.device)
        check(lib().spuma_pressure_flux(self.handle, ptr(upper), ptr(corr), ptr(p), ptr(phi), nb, ptr(bface_cell),
                                        ptr(bface_sf), ptr(bface_cf), ptr(bgamma), ptr(btype), ptr(c), ptr(bphi),
                                        ptr(out), ptr(bout), stream_ptr()), "spuma_pressure_flux")
        return out, bout

    def fv_div(self, phi, bface_cell=None, bphi=None):
        d = torch.empty(self.n_cells, dtype=torch.float64, device=self.device)
        nb = 0 if bface_cell is None else int(bface_cell.numel())
        check(lib().spuma_fv_div(self.handle, ptr(phi), nb, ptr(bface_cell), ptr(bphi), ptr(d), stream_ptr()),
              "spuma_fv_div")
        return d

    def pressure_step(self, geom, gamma, bgamma, btype, phi, bphi, p_old, controls=None):
        """One pressure correction (nNonOrthogonalCorrectors 0): assemble A,
        b from div(phiHbyA) and the explicit correction with grad(p_old),
        solve, reconstruct the flux.  geom = (sf, cf, c, v, bface_cell,
        bface_sf, bface_cf).  Returns (p, phi, bphi, perf)."""
        sf, cf, c, v, bcell, bsf, bcf = geom
        upper, diag = self.assemble_laplacian(sf, c, gamma, bcell, bsf, bcf, bgamma, btype)
        w = self.fv_weights(sf, cf, c)
        g = self.fv_grad(sf, w, v, p_old, bcell, bsf, btype)
        corr, b = self.pressure_rhs(sf, c, w, gamma, g, phi, bcell, bphi)
        p, perf = self.solve(diag, upper, b, None, controls or SolverControls())
        phin, bphin = self.pressure_flux(upper, corr, p, phi, c, bcell, bsf, bcf, bgamma, btype, bphi)
        return p, phin, bphin, perf

    def amul(self, diag, upper, x, out=None):
        prec = F32 if x.dtype == torch.float32 else F64
        y = out if out is not None else torch.empty_like(x)
        check(lib().spuma_amul(self.handle, prec, ptr(diag), ptr(upper), ptr(x), ptr(y), stream_ptr()),
              "spuma_amul")
        return y

    def prepare(self, diag, upper, precond=PRECOND_DIC):
        check(lib().spuma_matrix_prepare(self.handle, ptr(diag), ptr(upper), int(precond), stream_ptr()),
              "spuma_matrix_prepare")

    def read_rD(self):
        out = torch.empty(self.n_cells, dtype=torch.float64, device=self.device)
        check(lib().spuma_read_rD(self.handle, ptr(out), stream_ptr()), "spuma_read_rD")
        return out

    def amul_prepared(self, x_internal, out=None):
        prec = F32 if x_internal.dtype == torch.float32 else F64
        y = out if out is not None else torch.empty_like(x_internal)
        check(lib().spuma_amul_prepared(self.handle, prec, ptr(x_internal), ptr(y), stream_ptr()),
              "spuma_amul_prepared")
        return y

    def to_internal(self, v):
        out = torch.empty_like(v)
        check(lib().spuma_permute(self.handle, 0, ptr(v), ptr(out), stream_ptr()), "spuma_permute")
        return out

    def from_internal(self, v):
        out = torch.empty_like(v)
        check(lib().spuma_permute(self.handle, 1, ptr(v), ptr(out), stream_ptr()), "spuma_permute")
        return out

    def precondition(self, r, precond=PRECOND_DIC):
        w = torch.empty_like(r)
        check(lib().spuma_precondition(self.handle, int(precond), ptr(r), ptr(w), stream_ptr()),
              "spuma_precondition")
        return w

    def solve(self, diag, upper, b, x=None, controls: SolverControls | None = None, perf=None, check_status=True):
        """Solve A x = b in place of x (x0 = 0 when x is None).  Returns (x, perf dict | perf tensor)."""
        ctl = (controls or SolverControls()).c()
        if x is None:
            x = torch.zeros_like(b)
        own_perf = perf is None
        if own_perf:
            perf = perf_tensor(1, self.device)
        check(lib().spuma_pcg_solve(self.handle, ptr(diag), ptr(upper), ptr(b), ptr(x), C.byref(ctl), ptr(perf),
                                    stream_ptr()), "spuma_pcg_solve")
        if not own_perf:
            return x, perf
        p = read_perf(perf)[0]
        if check_status and p["status"] != 0:
            raise SpumaError(p["status"], "device-side status of spuma_pcg_solve")
        return x, p

    def pbicg_solve(self, diag, lower, upper, b, x=None, controls: SolverControls | None = None, perf=None,
                    check_status=True):
        """PBiCG on the asymmetric A (A_{u,l} = lower_f, A_{l,u} = upper_f), in place of x
        (x0 = 0 when x is None); the mesh must be created with asymmetric=True."""
        ctl = (controls or SolverControls(precond=PRECOND_DILU)).c()
        if x is None:
            x = torch.zeros_like(b)
        own_perf = perf is None
        if own_perf:
            perf = perf_tensor(1, self.device)
        check(lib().spuma_pbicg_solve(self.handle, ptr(diag), ptr(lower), ptr(upper), ptr(b), ptr(x), C.byref(ctl),
                                      ptr(perf), stream_ptr()), "spuma_pbicg_solve")
        if not own_perf:
            return x, perf
        p = read_perf(perf)[0]
        if check_status and p["status"] != 0:
            raise SpumaError(p["status"], "device-side status of spuma_pbicg_solve")
        return x, p

    def adjoint(self, diag, upper, x, dldx, controls: SolverControls | None = None, want_diag=True,
                check_status=True):
        ctl = (controls or SolverControls(tolerance=1e-12)).c()
        dldb = torch.empty_like(dldx)
        dldu = torch.empty(self.n_faces, dtype=torch.float64, device=self.device)
        dldd = torch.empty_like(dldx) if want_diag else None
        perf = perf_tensor(1, self.device)
        check(lib().spuma_pcg_adjoint(self.handle, ptr(diag), ptr(upper), ptr(x), ptr(dldx), ptr(dldb), ptr(dldu),
                                      ptr(dldd), C.byref(ctl), ptr(perf), stream_ptr()), "spuma_pcg_adjoint")
        p = read_perf(perf)[0]
        if check_status and p["status"] != 0:
            raise SpumaError(p["status"], "device-side status of spuma_pcg_adjoint")
        return dldb, dldu, dldd, p


class GamgSolver:
    """GAMG for a mesh's symmetric pressure matrices: the level hierarchy from
    the face weights (e.g. |S_f|), built once, then any number of solves."""

    def __init__(self, mesh: LduMesh, face_weight, smoother: int = 0, coarsest_precond: int = 1):
        """smoother 0 Richardson (damped Jacobi), 1 two-stage Gauss-Seidel;
        coarsest_precond 1 diagonal, 2 DIC."""
        L = lib()
        self.mesh = mesh
        fw = torch.as_tensor(face_weight, dtype=torch.float64).to(mesh.device).contiguous()
        h = C.c_void_p()
        check(L.spuma_gamg_create(mesh.handle, ptr(fw), stream_ptr(), C.byref(h)), "spuma_gamg_create")
        self.handle = h
        nbytes = L.spuma_gamg_workspace_bytes(h)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=mesh.device)
        base = (self.workspace.data_ptr() + 255) // 256 * 256
        check(L.spuma_gamg_bind(h, base, nbytes, stream_ptr()), "spuma_gamg_bind")
        check(L.spuma_gamg_set_options(h, int(smoother), int(coarsest_precond)), "spuma_gamg_set_options")
        nl = C.c_int32()
        cells = (C.c_int32 * 64)()
        check(L.spuma_gamg_info(h, C.byref(nl), C.cast(cells, C.c_void_p), 64), "spuma_gamg_info")
        self.level_cells = [cells[k] for k in range(min(nl.value, 64))]

    def set_options(self, smoother: int = 0, coarsest_precond: int = 1):
        """Smoother (0 Richardson, 1 two-stage Gauss-Seidel) and coarsest-level
        preconditioner (1 diagonal, 2 DIC) of later solves; the hierarchy is kept."""
        check(lib().spuma_gamg_set_options(self.handle, int(smoother), int(coarsest_precond)),
              "spuma_gamg_set_options")

    def solve(self, diag, upper, b, x=None, controls: SolverControls | None = None, perf=None, check_status=True):
        ctl = (controls or SolverControls()).c()
        if x is None:
            x = torch.zeros_like(b)
        own_perf = perf is None
        if own_perf:
            perf = perf_tensor(1, self.mesh.device)
        check(lib().spuma_gamg_solve(self.handle, ptr(diag), ptr(upper), ptr(b), ptr(x), C.byref(ctl), ptr(perf),
                                     stream_ptr()), "spuma_gamg_solve")
        if not own_perf:
            return x, perf
        p = read_perf(perf)[0]
        if check_status and p["status"] != 0:
            raise SpumaError(p["status"], "device-side status of spuma_gamg_solve")
        return x, p

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                lib().spuma_gamg_destroy(h)
            except Exception:
                pass


class BatchSolve:
    """Many systems in one persistent launch, replayed from a CUDA graph
    (capture failure raises unless allow_direct=True)."""

    def __init__(self, meshes, diags, uppers, bs, xs, controls: SolverControls | None = None, autotune=True,
                 allow_direct=False, graph=True):
        n = len(meshes)
        self.meshes, self.diags, self.uppers, self.bs, self.xs = meshes, diags, uppers, bs, xs
        self.ctl = (controls or SolverControls()).c()
        self.perf = perf_tensor(n, meshes[0].device)
        H = (C.c_void_p * n)(*[m.handle.value for m in meshes])
        arr = lambda ts: (C.c_void_p * n)(*[ptr(t) for t in ts])
        self._keep = (H, arr(diags), arr(uppers), arr(bs), arr(xs))
        flags = ((BATCH_AUTOTUNE if autotune else 0) | (BATCH_ALLOW_DIRECT if allow_direct else 0)
                 | (0 if graph else BATCH_NO_GRAPH))
        h = C.c_void_p()
        check(lib().spuma_batch_create(n, self._keep[0], self._keep[1], self._keep[2], self._keep[3], self._keep[4],
                                       C.byref(self.ctl), ptr(self.perf), flags, stream_ptr(), C.byref(h)),
              "spuma_batch_create")
        self.handle = h
        t, g, ms, cap = C.c_int32(), C.c_int32(), C.c_double(), C.c_int32()
        check(lib().spuma_batch_info(h, C.byref(t), C.byref(g), C.byref(ms), C.byref(cap)), "spuma_batch_info")
        self.block_threads, self.grid_blocks, self.tuned_ms = t.value, g.value, ms.value
        self.graph_captured = bool(cap.value)
        nt = lib().spuma_batch_trials(h, 0, None, None, None, None)
        if nt > 0:
            tt, pp, gg, mm = (C.c_int32 * nt)(), (C.c_int32 * nt)(), (C.c_int32 * nt)(), (C.c_double * nt)()
            lib().spuma_batch_trials(h, nt, C.cast(tt, C.c_void_p), C.cast(pp, C.c_void_p), C.cast(gg, C.c_void_p),
                                     C.cast(mm, C.c_void_p))
            self.trials = [dict(block_threads=tt[k], split_policy=pp[k], grid_blocks=gg[k], ms=round(mm[k], 3))
                           for k in range(nt)]
        else:
            self.trials = []

    def run(self):
        check(lib().spuma_batch_run(self.handle, stream_ptr()), "spuma_batch_run")

    def results(self):
        return read_perf(self.perf)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                lib().spuma_batch_destroy(h)
            except Exception:
                pass
            self.handle = None


def solve_host(mesh: LduMesh, diag, upper, b_host, controls: SolverControls | None = None):
    """End-to-end call with host buffers: copies b (pinned host) in, solves,
    copies x back.  Returns (x_host, perf dict)."""
    b = b_host.to(mesh.device, non_blocking=True)
    x = torch.zeros_like(b)
    x, p = mesh.solve(diag, upper, b, x, controls)
    return x.cpu(), p
