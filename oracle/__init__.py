"""CPU oracle of the LDU pressure-solve path (test infrastructure only).

A plain, sequential FP64 C implementation (``oracle.c``) loaded with ctypes,
plus numpy glue.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the CUDA library shares
no code with it.  See the header of ``oracle.c`` for each function's
definition and the paper passage it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PRECOND_NONE, PRECOND_DIAGONAL, PRECOND_DIC = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i8p = np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_i32 = C.c_int32
_f64 = C.c_double


def _declare(L):
    L.oracle_assemble_laplacian.argtypes = [_i32, _i32, _i32p, _i32p, _f64p, _f64p, _f64p, _i32,
                                            _i32p, _f64p, _f64p, _f64p, _i8p, _f64p, _f64p]
    L.oracle_assemble_laplacian.restype = None
    L.oracle_assembly_adjoint.argtypes = [_i32, _i32p, _i32p, _f64p, _f64p, _i32, _i32p, _f64p, _f64p, _i8p,
                                          _f64p, _f64p, _f64p, _f64p]
    L.oracle_assembly_adjoint.restype = None
    L.oracle_dot.argtypes = [_i32, _f64p, _f64p]
    L.oracle_dot.restype = _f64
    L.oracle_jacobi_sweep.argtypes = [_i32, _i32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p]
    L.oracle_jacobi_sweep.restype = None
    L.oracle_gs2_sweep.argtypes = [_i32, _i32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p]
    L.oracle_gs2_sweep.restype = None
    L.oracle_amul_asym.argtypes = [_i32, _i32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p, _f64p]
    L.oracle_amul_asym.restype = None
    L.oracle_dilu_factor.argtypes = [_i32, _i32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p]
    L.oracle_dilu_factor.restype = _i32
    L.oracle_dilu_precondition.argtypes = [_i32, _i32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p, _f64p]
    L.oracle_dilu_precondition.restype = None
    L.oracle_pbicg.argtypes = [_i32, _i32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p, _f64p, _i32, _f64, _f64,
                               _i32, _i32, _f64p]
    L.oracle_pbicg.restype = _i32
    L.oracle_fv_weights.argtypes = [_i32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p]
    L.oracle_fv_weights.restype = None
    L.oracle_fv_grad.argtypes = [_i32, _i32, _i32p, _i32p, _f64p, _f64p, _f64p, _i32, _i32p, _f64p, _i8p, _f64p,
                                 _f64p]
    L.oracle_fv_grad.restype = None
    L.oracle_pressure_rhs.argtypes = [_i32, _i32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p, _i32,
                                      _i32p, _f64p, _f64p, _f64p]
    L.oracle_pressure_rhs.restype = None
    L.oracle_pressure_flux.argtypes = [_i32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p, _i32, _i32p, _f64p, _f64p,
                                       _f64p, _i8p, _f64p, _f64p, _f64p, _f64p]
    L.oracle_pressure_flux.restype = None
    L.oracle_fv_div.argtypes = [_i32, _i32, _i32p, _i32p, _f64p, _i32, _i32p, _f64p, _f64p]
    L.oracle_fv_div.restype = None
    L.oracle_amul.argtypes = [_i32, _i32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p]
    L.oracle_amul.restype = None
    L.oracle_amul_f32.argtypes = [_i32, _i32, _i32p, _i32p, _f32p, _f32p, _f32p, _f32p]
    L.oracle_amul_f32.restype = None
    L.oracle_dic_factor.argtypes = [_i32, _i32, _i32p, _i32p, _f64p, _f64p, _f64p]
    L.oracle_dic_factor.restype = _i32
    L.oracle_dic_precondition.argtypes = [_i32, _i32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p]
    L.oracle_dic_precondition.restype = None
    L.oracle_dic_precondition_f32.argtypes = [_i32, _i32, _i32p, _i32p, _f64p, _f64p, _f32p, _f32p]
    L.oracle_dic_precondition_f32.restype = None
    L.oracle_diag_reciprocal.argtypes = [_i32, _f64p, _f64p]
    L.oracle_diag_reciprocal.restype = None
    L.oracle_norm_factor.argtypes = [_i32, _i32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p, _f64p]
    L.oracle_norm_factor.restype = _f64
    L.oracle_pcg.argtypes = [_i32, _i32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p, _i32, _f64, _f64,
                             _i32, _i32, _f64p]
    L.oracle_pcg.restype = _i32
    L.oracle_mixed_ir.argtypes = [_i32, _i32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p, _i32, _f64,
                                  _f64, _i32, _i32, _f64p]
    L.oracle_mixed_ir.restype = _i32
    L.oracle_mixed_reliable.argtypes = [_i32, _i32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p, _i32, _f64,
                                        _f64, _f64, _i32, _f64p]
    L.oracle_mixed_reliable.restype = _i32
    L.oracle_adjoint.argtypes = [_i32, _i32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p, _i32, _f64,
                                 _i32, _f64p, _f64p, _f64p, _f64p]
    L.oracle_adjoint.restype = _i32


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def assemble_laplacian(mesh, gamma, bgamma, btype):
    """(upper[F], diag[N]) of A = -laplacian(gamma, p), Gauss linear corrected."""
    upper = np.empty(mesh.n_faces)
    diag = np.empty(mesh.n_cells)
    lib().oracle_assemble_laplacian(mesh.n_cells, mesh.n_faces, _c(mesh.lower, np.int32),
                                    _c(mesh.upper_addr, np.int32), _c(mesh.sf, np.float64),
                                    _c(mesh.c, np.float64), _c(gamma, np.float64), mesh.n_bfaces,
                                    _c(mesh.bface_cell, np.int32), _c(mesh.bface_sf, np.float64),
                                    _c(mesh.bface_cf, np.float64), _c(bgamma, np.float64),
                                    _c(btype, np.int8), upper, diag)
    return upper, diag


def assembly_adjoint(mesh, gupper, gdiag, btype):
    """(dL/dgamma[F], dL/dbgamma[B]) from dL/dupper and dL/ddiag through the
    assembly above (geometry fixed): the reverse mode of a2, which is linear
    in the diffusivities."""
    gg = np.empty(mesh.n_faces)
    gb = np.empty(mesh.n_bfaces)
    lib().oracle_assembly_adjoint(mesh.n_faces, _c(mesh.lower, np.int32), _c(mesh.upper_addr, np.int32),
                                  _c(mesh.sf, np.float64), _c(mesh.c, np.float64), mesh.n_bfaces,
                                  _c(mesh.bface_cell, np.int32), _c(mesh.bface_sf, np.float64),
                                  _c(mesh.bface_cf, np.float64), _c(btype, np.int8), _c(gupper, np.float64),
                                  _c(gdiag, np.float64), gg, gb)
    return gg, gb


# ---------------------------------------------- pressure-correction step ----
def fv_weights(mesh):
    """Linear interpolation weight of the owner value at each internal face."""
    w = np.empty(mesh.n_faces)
    lib().oracle_fv_weights(mesh.n_faces, _c(mesh.lower, np.int32), _c(mesh.upper_addr, np.int32),
                            _c(mesh.sf, np.float64), _c(mesh.cf, np.float64), _c(mesh.c, np.float64), w)
    return w


def fv_grad(mesh, w, btype, p):
    """Gauss linear gradient [N, 3] (Dirichlet faces p = 0, zero-gradient p_b = p_cell)."""
    g = np.empty((mesh.n_cells, 3))
    lib().oracle_fv_grad(mesh.n_cells, mesh.n_faces, _c(mesh.lower, np.int32), _c(mesh.upper_addr, np.int32),
                         _c(mesh.sf, np.float64), _c(w, np.float64), _c(mesh.v, np.float64), mesh.n_bfaces,
                         _c(mesh.bface_cell, np.int32), _c(mesh.bface_sf, np.float64), _c(btype, np.int8),
                         _c(p, np.float64), g)
    return g


def pressure_rhs(mesh, w, gamma, grad, phi, bphi):
    """(corr[F], b[N]): explicit non-orthogonal correction flux and the
    right-hand side of A p = b for laplacian(gamma, p) = div(phiHbyA)."""
    corr = np.empty(mesh.n_faces)
    b = np.empty(mesh.n_cells)
    lib().oracle_pressure_rhs(mesh.n_cells, mesh.n_faces, _c(mesh.lower, np.int32), _c(mesh.upper_addr, np.int32),
                              _c(mesh.sf, np.float64), _c(mesh.c, np.float64), _c(w, np.float64),
                              _c(gamma, np.float64), _c(grad, np.float64), _c(phi, np.float64), mesh.n_bfaces,
                              _c(mesh.bface_cell, np.int32), _c(bphi, np.float64), corr, b)
    return corr, b


def pressure_flux(mesh, upper, corr, p, phi, bgamma, btype, bphi):
    """(phi[F], bphi[B]) after the solve."""
    out = np.empty(mesh.n_faces)
    bout = np.empty(mesh.n_bfaces)
    lib().oracle_pressure_flux(mesh.n_faces, _c(mesh.lower, np.int32), _c(mesh.upper_addr, np.int32),
                               _c(upper, np.float64), _c(corr, np.float64), _c(p, np.float64), _c(phi, np.float64),
                               mesh.n_bfaces, _c(mesh.bface_cell, np.int32), _c(mesh.bface_sf, np.float64),
                               _c(mesh.bface_cf, np.float64), _c(bgamma, np.float64), _c(btype, np.int8),
                               _c(mesh.c, np.float64), _c(bphi, np.float64), out, bout)
    return out, bout


def fv_div(mesh, phi, bphi):
    """Integrated divergence [N] of face and boundary fluxes."""
    d = np.empty(mesh.n_cells)
    lib().oracle_fv_div(mesh.n_cells, mesh.n_faces, _c(mesh.lower, np.int32), _c(mesh.upper_addr, np.int32),
                        _c(phi, np.float64), mesh.n_bfaces, _c(mesh.bface_cell, np.int32), _c(bphi, np.float64), d)
    return d


# ------------------------------------------- asymmetric matrices: PBiCG ----
def amul_asym(l, u, diag, lower, upper, x):
    """y = A x with A_{u,l} = lower_f, A_{l,u} = upper_f (Tmul: swap lower/upper)."""
    y = np.empty(len(diag))
    lib().oracle_amul_asym(len(diag), len(l), _c(l, np.int32), _c(u, np.int32), _c(diag, np.float64),
                           _c(lower, np.float64), _c(upper, np.float64), _c(x, np.float64), y)
    return y


def dilu_factor(l, u, diag, lower, upper):
    """Returns (rD, first_bad_cell or -1)."""
    rD = np.empty(len(diag))
    bad = lib().oracle_dilu_factor(len(diag), len(l), _c(l, np.int32), _c(u, np.int32), _c(diag, np.float64),
                                   _c(lower, np.float64), _c(upper, np.float64), rD)
    return rD, bad


def dilu_precondition(l, u, lower, upper, rD, r, transpose=False):
    """w = M^-1 r (or M^-T r) for M = (D + L) D^-1 (D + U)."""
    w = np.empty(len(rD))
    lo, up = (upper, lower) if transpose else (lower, upper)
    lib().oracle_dilu_precondition(len(rD), len(l), _c(l, np.int32), _c(u, np.int32), _c(lo, np.float64),
                                   _c(up, np.float64), _c(rD, np.float64), _c(r, np.float64), w)
    return w


def pbicg(l, u, diag, lower, upper, b, x0=None, precond=3, tol=1e-8, rel_tol=0.0, max_iter=20000, min_iter=0):
    """(x, perf) of OpenFOAM PBiCG; precond 0 none, 1 diagonal, 3 DILU."""
    x = np.zeros(len(diag)) if x0 is None else np.array(x0, dtype=np.float64)
    perf = np.zeros(5)
    st = lib().oracle_pbicg(len(diag), len(l), _c(l, np.int32), _c(u, np.int32), _c(diag, np.float64),
                            _c(lower, np.float64), _c(upper, np.float64), _c(b, np.float64), x, int(precond),
                            float(tol), float(rel_tol), int(max_iter), int(min_iter), perf)
    return x, dict(status=st, initial_residual=perf[0], final_residual=perf[1], n_iter=int(perf[2]),
                   singular=int(perf[3]), converged=int(perf[4]))


def dot(a, b):
    """sum a_i b_i in ascending order."""
    return lib().oracle_dot(len(a), _c(a, np.float64), _c(b, np.float64))


def jacobi_sweep(l, u, diag, upper, wrd, r, e):
    """One damped-Jacobi sweep in place: e_i = fma(wrd_i, r_i - (A e)_i, e_i)."""
    q = np.empty(len(diag))
    lib().oracle_jacobi_sweep(len(diag), len(l), _c(l, np.int32), _c(u, np.int32), _c(diag, np.float64),
                              _c(upper, np.float64), _c(wrd, np.float64), _c(r, np.float64), e, q)
    return e


def gs2_sweep(l, u, diag, upper, rD, r, e):
    """One two-stage Gauss-Seidel sweep in place: e += (D^-1 - D^-1 L D^-1)(r - A e),
    in the face order of oracle.c (rD = 1/d)."""
    n = len(diag)
    q, y = np.empty(n), np.empty(n)
    lib().oracle_gs2_sweep(n, len(l), _c(l, np.int32), _c(u, np.int32), _c(diag, np.float64),
                           _c(upper, np.float64), _c(rD, np.float64), _c(r, np.float64), e, q, y)
    return e


def amul(l, u, diag, upper, x):
    n = len(diag)
    if np.asarray(x).dtype == np.float32:
        y = np.empty(n, dtype=np.float32)
        lib().oracle_amul_f32(n, len(l), _c(l, np.int32), _c(u, np.int32), _c(diag, np.float32),
                              _c(upper, np.float32), _c(x, np.float32), y)
        return y
    y = np.empty(n)
    lib().oracle_amul(n, len(l), _c(l, np.int32), _c(u, np.int32), _c(diag, np.float64),
                      _c(upper, np.float64), _c(x, np.float64), y)
    return y


def dic_factor(l, u, diag, upper):
    """Returns (rD, first_bad_cell or -1)."""
    rD = np.empty(len(diag))
    bad = lib().oracle_dic_factor(len(diag), len(l), _c(l, np.int32), _c(u, np.int32),
                                  _c(diag, np.float64), _c(upper, np.float64), rD)
    return rD, int(bad)


def dic_precondition(l, u, upper, rD, r):
    n = len(rD)
    if np.asarray(r).dtype == np.float32:
        w = np.empty(n, dtype=np.float32)
        lib().oracle_dic_precondition_f32(n, len(l), _c(l, np.int32), _c(u, np.int32),
                                          _c(upper, np.float64), _c(rD, np.float64),
                                          _c(r, np.float32), w)
        return w
    w = np.empty(n)
    lib().oracle_dic_precondition(n, len(l), _c(l, np.int32), _c(u, np.int32), _c(upper, np.float64),
                                  _c(rD, np.float64), _c(r, np.float64), w)
    return w


def diag_reciprocal(diag):
    rD = np.empty(len(diag))
    lib().oracle_diag_reciprocal(len(diag), _c(diag, np.float64), rD)
    return rD


def norm_factor(l, u, diag, upper, x, b):
    q = amul(l, u, diag, upper, x)
    return lib().oracle_norm_factor(len(diag), len(l), _c(l, np.int32), _c(u, np.int32),
                                    _c(diag, np.float64), _c(upper, np.float64), _c(x, np.float64),
                                    _c(b, np.float64), q)


def pcg(l, u, diag, upper, b, x0=None, precond=PRECOND_DIC, tol=1e-8, rel_tol=0.0,
        max_iter=20000, min_iter=0):
    """Returns (x, perf dict)."""
    n = len(diag)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    perf = np.zeros(5)
    st = lib().oracle_pcg(n, len(l), _c(l, np.int32), _c(u, np.int32), _c(diag, np.float64),
                          _c(upper, np.float64), _c(b, np.float64), x, int(precond), float(tol),
                          float(rel_tol), int(max_iter), int(min_iter), perf)
    return x, dict(status=int(st), initial_residual=perf[0], final_residual=perf[1],
                   n_iter=int(perf[2]), singular=int(perf[3]), converged=int(perf[4]))


def mixed_ir(l, u, diag, upper, b, x0=None, precond=PRECOND_DIC, tol=1e-8, inner_rel_tol=1e-4,
             max_iter=20000, max_outer=20):
    n = len(diag)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    perf = np.zeros(6)
    st = lib().oracle_mixed_ir(n, len(l), _c(l, np.int32), _c(u, np.int32), _c(diag, np.float64),
                               _c(upper, np.float64), _c(b, np.float64), x, int(precond), float(tol),
                               float(inner_rel_tol), int(max_iter), int(max_outer), perf)
    return x, dict(status=int(st), initial_residual=perf[0], final_residual=perf[1],
                   n_iter=int(perf[2]), singular=int(perf[3]), converged=int(perf[4]),
                   n_outer=int(perf[5]))


def mixed_reliable(l, u, diag, upper, b, x0=None, precond=PRECOND_DIC, tol=1e-8, rel_tol=0.0, delta=0.1,
                   max_iter=20000):
    """FP32 PCG with reliable FP64 updates (residual replacement, no restart)."""
    n = len(diag)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    perf = np.zeros(6)
    st = lib().oracle_mixed_reliable(n, len(l), _c(l, np.int32), _c(u, np.int32), _c(diag, np.float64),
                                     _c(upper, np.float64), _c(b, np.float64), x, int(precond), float(tol),
                                     float(rel_tol), float(delta), int(max_iter), perf)
    return x, dict(status=int(st), initial_residual=perf[0], final_residual=perf[1], n_iter=int(perf[2]),
                   singular=int(perf[3]), converged=int(perf[4]), n_outer=int(perf[5]))


def adjoint(l, u, diag, upper, x, g, precond=PRECOND_DIC, tol=1e-13, max_iter=20000):
    """Returns (lambda, dL/dupper, dL/ddiag, perf)."""
    n, nf = len(diag), len(l)
    lam = np.empty(n)
    du = np.empty(nf)
    dd = np.empty(n)
    perf = np.zeros(5)
    st = lib().oracle_adjoint(n, nf, _c(l, np.int32), _c(u, np.int32), _c(diag, np.float64),
                              _c(upper, np.float64), _c(x, np.float64), _c(g, np.float64),
                              int(precond), float(tol), int(max_iter), lam, du, dd, perf)
    return lam, du, dd, dict(status=int(st), n_iter=int(perf[2]), final_residual=perf[1])
