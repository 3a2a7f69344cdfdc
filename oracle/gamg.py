"""GAMG oracle (test infrastructure only): the paper's production pressure
solver, "GAMG, smoother Richardson" (fvSolution listing; Sec. 4.3 and the
smoother table: Richardson = damped Jacobi on every level, diagonal-PCG at
the coarsest one; the coarsening is OpenFOAM's, unmodified), and the table's
other two options: the two-stage Gauss-Seidel smoother and DIC-PCG at the
coarsest level (the profiling run's "coarsestSolver=DIC+PCG").

Plain, slow, sequential Python over numpy arrays, FP64, each sum in the order
written here.  Only the tests may call it.

Reading (the paper names the method, not its parameters):
  agglomeration  pairwise by face weight (OpenFOAM faceAreaPair): cells in
                 ascending order; an unassigned cell pairs with its
                 unassigned neighbour across the heaviest face (first in face
                 order on ties); a cell whose neighbours are all assigned
                 joins the aggregate across its heaviest face; a cell without
                 faces stays alone.  The coarse graph keeps the faces between
                 different aggregates, (min, max) ordered and sorted, with
                 the weights summed.  Levels are added while the coarse level
                 has more than N_COARSEST cells and fewer cells than its fine
                 level.
  coarse matrix  Galerkin with piecewise-constant prolongation:
                 upper_F = sum of the fine upper_f mapped to F (ascending f);
                 diag_C = sum of the fine diag_i in C (ascending i), then
                 + 2 upper_f for each fine face inside C (ascending f).
  V-cycle        e = V(k, r): at the coarsest level PCG with the diagonal
                 preconditioner from 0 to relative tolerance COARSE_REL_TOL;
                 else no pre-smoothing, r_c = restriction (sum over the
                 aggregate, ascending), e = prolongation of V(k+1, r_c)
                 (injection) scaled by its A-norm optimal step
                 (e.r)/(e.Ae) (OpenFOAM's correction scaling; kept unscaled
                 when e.Ae <= 0), then NU_POST smoothing sweeps:
                 Richardson: damped Jacobi e_i += (OMEGA rD_i) (r_i - (A e)_i)
                 (one FMA, rD = 1/d);
                 two-stage Gauss-Seidel (smoother="gs2", Berger-Vergiat et
                 al.): e += (D^-1 - D^-1 L D^-1)(r - A e), i.e. the
                 Gauss-Seidel lower solve approximated by one Jacobi step and
                 one Jacobi-Richardson sweep, undamped (oracle.c gs2_sweep).
  coarsest       PCG from 0 to COARSE_REL_TOL with the diagonal (default) or
                 the DIC preconditioner (coarsest_precond=2).
  solver         x0 given; r = b - A x; normFactor, residual and the
                 stopping rule of PCG; each iteration x += V(0, r), r = b - A x.
"""
from __future__ import annotations

import numpy as np

from . import amul, dot, gs2_sweep, jacobi_sweep, norm_factor, pcg

OMEGA = 2.0 / 3.0
NU_POST = 2
N_COARSEST = 10
COARSE_REL_TOL = 1e-8
MAX_LEVELS = 50


def cell_faces(n, l, u):
    """Faces of each cell in ascending face order."""
    faces = [[] for _ in range(n)]
    for f in range(len(l)):
        faces[l[f]].append(f)
        faces[u[f]].append(f)
    return faces


def agglomerate(n, l, u, weight):
    """One pairwise level: (agg[n], n_coarse)."""
    faces = cell_faces(n, l, u)
    agg = [-1] * n
    nc = 0
    for i in range(n):
        if agg[i] != -1:
            continue
        best, bw = -1, -np.inf
        for f in faces[i]:
            j = u[f] if l[f] == i else l[f]
            if agg[j] == -1 and weight[f] > bw:
                best, bw = j, weight[f]
        if best >= 0:
            agg[i] = agg[best] = nc
            nc += 1
            continue
        best, bw = -1, -np.inf
        for f in faces[i]:
            j = u[f] if l[f] == i else l[f]
            if weight[f] > bw:
                best, bw = j, weight[f]
        if best >= 0:
            agg[i] = agg[best]
        else:
            agg[i] = nc
            nc += 1
    return np.array(agg, dtype=np.int64), nc


def coarse_graph(l, u, weight, agg):
    """(lc, uc, wc, face_map): coarse faces (sorted by (l, u)) with summed
    weights; face_map[f] = coarse face of fine face f, or -1 inside an aggregate."""
    pairs = {}
    for f in range(len(l)):
        a, b = int(agg[l[f]]), int(agg[u[f]])
        if a == b:
            continue
        key = (min(a, b), max(a, b))
        pairs.setdefault(key, []).append(f)
    keys = sorted(pairs)
    lc = np.array([k[0] for k in keys], dtype=np.int64)
    uc = np.array([k[1] for k in keys], dtype=np.int64)
    wc = np.zeros(len(keys))
    face_map = np.full(len(l), -1, dtype=np.int64)
    for F, k in enumerate(keys):
        s = 0.0
        for f in pairs[k]:
            s += weight[f]
            face_map[f] = F
        wc[F] = s
    return lc, uc, wc, face_map


def hierarchy(n, l, u, weight):
    """List of levels: dict(n, l, u, agg, face_map) (agg / face_map map to the next level)."""
    levels = [dict(n=n, l=np.asarray(l, dtype=np.int64), u=np.asarray(u, dtype=np.int64))]
    w = np.asarray(weight, dtype=np.float64)
    while len(levels) < MAX_LEVELS and levels[-1]["n"] > N_COARSEST:
        lv = levels[-1]
        agg, nc = agglomerate(lv["n"], lv["l"], lv["u"], w)
        if nc >= lv["n"]:
            break
        lc, uc, wc, fmap = coarse_graph(lv["l"], lv["u"], w, agg)
        lv["agg"], lv["face_map"] = agg, fmap
        levels.append(dict(n=nc, l=lc, u=uc))
        w = wc
    return levels


def coarse_matrix(lv, n_coarse, nf_coarse, diag, upper):
    """Galerkin coarse (diag, upper) of one level, sums in the stated order."""
    dc = np.zeros(n_coarse)
    for i in range(lv["n"]):
        dc[lv["agg"][i]] += diag[i]
    uc = np.zeros(nf_coarse)
    for f in range(len(lv["l"])):
        F = lv["face_map"][f]
        if F >= 0:
            uc[F] += upper[f]
    for f in range(len(lv["l"])):
        if lv["face_map"][f] < 0:
            dc[lv["agg"][lv["l"][f]]] += 2.0 * upper[f]
    return dc, uc


def matrices(levels, diag, upper):
    mats = [(np.asarray(diag, dtype=np.float64), np.asarray(upper, dtype=np.float64))]
    for k in range(len(levels) - 1):
        d, u = mats[-1]
        mats.append(coarse_matrix(levels[k], levels[k + 1]["n"], len(levels[k + 1]["l"]), d, u))
    return mats


def vcycle(levels, mats, k, r, smoother="richardson", coarsest_precond=1):
    lv = levels[k]
    d, up = mats[k]
    if k == len(levels) - 1:
        e, _ = pcg(lv["l"], lv["u"], d, up, r, precond=coarsest_precond, tol=0.0, rel_tol=COARSE_REL_TOL,
                   max_iter=2 * lv["n"] + 10)
        return e
    nc = levels[k + 1]["n"]
    rc = np.zeros(nc)
    for i in range(lv["n"]):
        rc[lv["agg"][i]] += r[i]
    ec = vcycle(levels, mats, k + 1, rc, smoother, coarsest_precond)
    e = np.ascontiguousarray(ec[lv["agg"]], dtype=np.float64)
    # scale the prolongated correction by its A-norm optimal step (e.r)/(e.Ae)
    q = amul(lv["l"], lv["u"], d, up, e)
    eq = dot(e, q)
    if eq > 0.0:
        e = e * (dot(e, r) / eq)
    if smoother == "gs2":
        rD = 1.0 / d
        for _ in range(NU_POST):
            gs2_sweep(lv["l"], lv["u"], d, up, rD, r, e)
    else:
        wrd = OMEGA * (1.0 / d)
        for _ in range(NU_POST):
            jacobi_sweep(lv["l"], lv["u"], d, up, wrd, r, e)
    return e


def gamg(l, u, diag, upper, b, weight, x0=None, tol=1e-8, rel_tol=0.0, max_iter=300, min_iter=0,
         smoother="richardson", coarsest_precond=1):
    """(x, perf, levels) of the GAMG solver with the PCG residual and stopping rule;
    smoother "richardson" or "gs2", coarsest-level PCG preconditioner 1 (diagonal) or 2 (DIC)."""
    assert smoother in ("richardson", "gs2") and coarsest_precond in (1, 2)
    n = len(diag)
    levels = hierarchy(n, l, u, weight)
    mats = matrices(levels, diag, upper)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    q = amul(l, u, diag, upper, x)
    r = b - q
    nfac = norm_factor(l, u, diag, upper, x, b)
    res0 = np.abs(r).sum() / nfac
    res = res0
    it = 0

    def conv(rr):
        return rr < tol or (rel_tol > 0 and rr < rel_tol * res0)

    if min_iter > 0 or not conv(res0):
        while True:
            x = x + vcycle(levels, mats, 0, r, smoother, coarsest_precond)
            r = b - amul(l, u, diag, upper, x)
            res = np.abs(r).sum() / nfac
            it += 1
            if not ((it < max_iter and not conv(res)) or it < min_iter):
                break
    perf = dict(initial_residual=res0, final_residual=res, n_iter=it, converged=int(conv(res)),
                n_levels=len(levels))
    return x, perf, levels
