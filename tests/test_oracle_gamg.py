"""Pins of the GAMG oracle (agglomeration, Galerkin coarse matrices, V-cycle,
solver) against closed forms, dense linear algebra and the multigrid
property that the iteration count does not grow with the mesh."""
import numpy as np
import pytest

import hexmesh
import oracle
from oracle import gamg as G


def _case(n, seed, **kw):
    c = hexmesh.pressure_case(n, seed=seed, **kw)
    m = c.mesh
    up, dg = oracle.assemble_laplacian(m, c.gamma, c.bgamma, c.btype)
    return c, m, up, dg, np.linalg.norm(m.sf, axis=1)


def test_agglomeration_of_chains():
    l = np.arange(7)
    u = l + 1
    agg, nc = G.agglomerate(8, l, u, np.ones(7))
    assert nc == 4 and list(agg) == [0, 0, 1, 1, 2, 2, 3, 3]
    agg, nc = G.agglomerate(7, l[:6], u[:6], np.arange(1.0, 7.0))
    assert nc == 3 and list(agg) == [0, 0, 1, 1, 2, 2, 2]     # the last cell joins its neighbour's pair
    agg, nc = G.agglomerate(3, np.array([], dtype=np.int64), np.array([], dtype=np.int64), np.zeros(0))
    assert nc == 3 and list(agg) == [0, 1, 2]                  # no faces: singletons


def test_heaviest_face_wins():
    # star: cell 0 joined to 1, 2, 3 with weights 1, 5, 2 -> pairs (0, 2), then 1 and 3 join across their faces
    l, u, w = np.array([0, 0, 0]), np.array([1, 2, 3]), np.array([1.0, 5.0, 2.0])
    agg, nc = G.agglomerate(4, l, u, w)
    assert agg[0] == agg[2] and nc == 1 and list(agg) == [0, 0, 0, 0]


def test_aggregates_connected_and_covering():
    c, m, up, dg, w = _case(7, 91, jitter=0.2, permute=True, lognormal_gamma=True)
    levels = G.hierarchy(m.n_cells, m.lower, m.upper_addr, w)
    assert levels[-1]["n"] <= G.N_COARSEST or len(levels) == G.MAX_LEVELS
    for k in range(len(levels) - 1):
        lv, nc = levels[k], levels[k + 1]["n"]
        agg = lv["agg"]
        assert set(agg.tolist()) == set(range(nc))
        # connectivity: union-find over the faces inside aggregates
        parent = list(range(lv["n"]))

        def find(a):
            while parent[a] != a:
                parent[a] = parent[parent[a]]
                a = parent[a]
            return a
        for f in range(len(lv["l"])):
            a, b = lv["l"][f], lv["u"][f]
            if agg[a] == agg[b]:
                parent[find(a)] = find(b)
        roots = {}
        for i in range(lv["n"]):
            roots.setdefault(agg[i], set()).add(find(i))
        assert all(len(r) == 1 for r in roots.values())
        assert levels[k + 1]["n"] < lv["n"]


def test_galerkin_coarse_matrices_dense():
    c, m, up, dg, w = _case((6, 5, 4), 92, jitter=0.2, permute=True, lognormal_gamma=True)
    levels = G.hierarchy(m.n_cells, m.lower, m.upper_addr, w)
    mats = G.matrices(levels, dg, up)

    def dense(n, l, u, d, a):
        A = np.zeros((n, n))
        A[np.arange(n), np.arange(n)] = d
        A[l, u] = a
        A[u, l] = a
        return A

    for k in range(len(levels) - 1):
        lv, cv = levels[k], levels[k + 1]
        A = dense(lv["n"], lv["l"], lv["u"], *mats[k])
        P = np.zeros((lv["n"], cv["n"]))
        P[np.arange(lv["n"]), lv["agg"]] = 1.0
        Ac = dense(cv["n"], cv["l"], cv["u"], *mats[k + 1])
        assert np.allclose(Ac, P.T @ A @ P, rtol=1e-13, atol=1e-13 * np.abs(A).max())
        assert np.all(cv["l"] < cv["u"])
        keys = list(zip(cv["l"], cv["u"]))
        assert keys == sorted(set(keys))


def test_gamg_error_decreases_monotonically_in_energy_norm():
    c, m, up, dg, w = _case(6, 93, jitter=0.2, permute=True, lognormal_gamma=True)
    A_l, A_u = m.lower, m.upper_addr
    xs, _ = oracle.pcg(A_l, A_u, dg, up, c.b, tol=1e-15, max_iter=5000)
    errs = []
    for it in range(1, 8):
        x, p, _ = G.gamg(A_l, A_u, dg, up, c.b, w, tol=0.0, max_iter=it)
        e = x - xs
        errs.append(np.dot(e, oracle.amul(A_l, A_u, dg, up, e)))
    assert all(b < a for a, b in zip(errs, errs[1:]))


def test_gamg_matches_dense_solution():
    c, m, up, dg, w = _case(5, 94, jitter=0.2, permute=True, lognormal_gamma=True)
    x, p, _ = G.gamg(m.lower, m.upper_addr, dg, up, c.b, w, tol=1e-13, max_iter=500)
    A = np.zeros((m.n_cells, m.n_cells))
    A[np.arange(m.n_cells), np.arange(m.n_cells)] = dg
    A[m.lower, m.upper_addr] = up
    A[m.upper_addr, m.lower] = up
    assert p["converged"] == 1
    assert np.allclose(x, np.linalg.solve(A, c.b), rtol=1e-9, atol=1e-11)


def test_iterations_do_not_grow_with_the_mesh():
    """The multigrid property (PCG-DIC needs 2x the iterations from 8^3 to 16^3)."""
    its = []
    for n in (8, 16):
        c, m, up, dg, w = _case(n, 95, jitter=0.2, permute=True, lognormal_gamma=True)
        _, p, _ = G.gamg(m.lower, m.upper_addr, dg, up, c.b, w, tol=1e-10)
        its.append(p["n_iter"])
    assert its[1] <= 1.3 * its[0]


def _dense(n, l, u, d, a):
    A = np.zeros((n, n))
    A[np.arange(n), np.arange(n)] = d
    A[l, u] = a
    A[u, l] = a
    return A


def test_gs2_sweep_is_the_truncated_gauss_seidel_step_dense():
    """The face-loop sweep equals the matrix formula e + (D^-1 - D^-1 L D^-1)(r - A e)
    with L = strictly lower part of A (row u(f), column l(f)), on a jittered
    permuted mesh (dense numpy, independent of the face loop)."""
    c, m, up, dg, w = _case((5, 4, 3), 96, jitter=0.2, permute=True, lognormal_gamma=True)
    n = m.n_cells
    A = _dense(n, m.lower, m.upper_addr, dg, up)
    L = np.tril(A, -1)
    Dinv = np.diag(1.0 / dg)
    rng = np.random.default_rng(97)
    r, e0 = rng.standard_normal(n), rng.standard_normal(n)
    e = oracle.gs2_sweep(m.lower, m.upper_addr, dg, up, 1.0 / dg, r, e0.copy())
    ref = e0 + (Dinv - Dinv @ L @ Dinv) @ (r - A @ e0)
    assert np.allclose(e, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    # a sign error in L, or the upper part used instead, is far off
    bad = e0 + (Dinv + Dinv @ L @ Dinv) @ (r - A @ e0)
    assert not np.allclose(e, bad, rtol=1e-6)


def test_gs2_special_cases():
    # no faces: one sweep is the Jacobi solve rD r from e = 0 (both stages give rD r, rounded once)
    d = np.array([2.0, 4.0, 5.0])
    r = np.array([1.0, 2.0, 3.0])
    e = oracle.gs2_sweep(np.zeros(0, np.int64), np.zeros(0, np.int64), d, np.zeros(0), 1.0 / d, r, np.zeros(3))
    assert np.array_equal(e, (1.0 / d) * r) and np.allclose(e, [0.5, 0.5, 0.6], rtol=1e-15)
    # two cells joined by one face: the truncated series is exact for a 2x2 lower solve,
    # so from e = 0 the sweep is the Gauss-Seidel step (D + L)^-1 r
    d = np.array([4.0, 3.0])
    a = np.array([-1.0])
    r = np.array([1.0, 2.0])
    e = oracle.gs2_sweep(np.array([0]), np.array([1]), d, a, 1.0 / d, r, np.zeros(2))
    DL = np.array([[4.0, 0.0], [-1.0, 3.0]])
    assert np.allclose(e, np.linalg.solve(DL, r), rtol=1e-15)


@pytest.mark.parametrize("smoother,coarsest", [("gs2", 1), ("richardson", 2), ("gs2", 2)])
def test_gamg_options_match_dense_solution(smoother, coarsest):
    c, m, up, dg, w = _case(6, 98, jitter=0.2, permute=True, lognormal_gamma=True)
    x, p, levels = G.gamg(m.lower, m.upper_addr, dg, up, c.b, w, tol=1e-13, max_iter=500, smoother=smoother,
                          coarsest_precond=coarsest)
    A = _dense(m.n_cells, m.lower, m.upper_addr, dg, up)
    assert p["converged"] == 1 and len(levels) >= 3
    assert np.allclose(x, np.linalg.solve(A, c.b), rtol=1e-9, atol=1e-11)


def test_gamg_single_level_is_the_coarsest_pcg():
    """A mesh of at most N_COARSEST cells has one level: one GAMG iteration is one
    coarsest-level PCG solve from 0 (DIC or diagonal) to COARSE_REL_TOL."""
    c, m, up, dg, w = _case((3, 3, 1), 99, jitter=0.2, permute=True, lognormal_gamma=True)
    assert m.n_cells <= G.N_COARSEST
    for pc in (1, 2):
        x, p, levels = G.gamg(m.lower, m.upper_addr, dg, up, c.b, w, tol=0.0, max_iter=1, coarsest_precond=pc)
        assert len(levels) == 1
        xo, _ = oracle.pcg(m.lower, m.upper_addr, dg, up, c.b, precond=pc, tol=0.0, rel_tol=G.COARSE_REL_TOL,
                           max_iter=2 * m.n_cells + 10)
        assert np.array_equal(x, xo)


def test_gs2_gamg_error_decreases_in_energy_norm_and_iterations_do_not_grow():
    c, m, up, dg, w = _case(6, 93, jitter=0.2, permute=True, lognormal_gamma=True)
    xs, _ = oracle.pcg(m.lower, m.upper_addr, dg, up, c.b, tol=1e-15, max_iter=5000)
    errs = []
    for it in range(1, 6):
        x, _, _ = G.gamg(m.lower, m.upper_addr, dg, up, c.b, w, tol=0.0, max_iter=it, smoother="gs2")
        e = x - xs
        errs.append(np.dot(e, oracle.amul(m.lower, m.upper_addr, dg, up, e)))
    assert all(b < a for a, b in zip(errs, errs[1:]))
    its = []
    for n in (8, 16):
        c, m, up, dg, w = _case(n, 95, jitter=0.2, permute=True, lognormal_gamma=True)
        _, p, _ = G.gamg(m.lower, m.upper_addr, dg, up, c.b, w, tol=1e-10, smoother="gs2", coarsest_precond=2)
        its.append(p["n_iter"])
    assert its[1] <= 1.3 * its[0], its
