"""Pins of the oracle's asymmetric path (Amul/Tmul, DILU, PBiCG) against
dense linear algebra and against the symmetric path it must reduce to."""
import numpy as np
import pytest

import oracle
from asym_cases import asym_case, dense_asym


@pytest.fixture(scope="module")
def ac():
    c, lower, upper, diag = asym_case(5, seed=71, jitter=0.2, permute=True, lognormal_gamma=True)
    m = c.mesh
    return m, lower, upper, diag, dense_asym(m.lower, m.upper_addr, diag, lower, upper), c.b


def test_amul_and_tmul_dense(ac):
    m, lo, up, d, A, b = ac
    x = np.random.default_rng(72).standard_normal(len(d))
    assert np.allclose(oracle.amul_asym(m.lower, m.upper_addr, d, lo, up, x), A @ x, rtol=1e-13, atol=1e-13)
    assert np.allclose(oracle.amul_asym(m.lower, m.upper_addr, d, up, lo, x), A.T @ x, rtol=1e-13, atol=1e-13)


def test_dilu_reproduces_pattern_and_inverts_m(ac):
    """M = (D + L) D^-1 (D + U) with D = diag(1/rD) equals A on A's pattern
    (hex meshes have no triangles, so the fill-in lies off the pattern)."""
    m, lo, up, d, A, b = ac
    rD, bad = oracle.dilu_factor(m.lower, m.upper_addr, d, lo, up)
    assert bad == -1
    D = np.diag(1.0 / rD)
    L = np.tril(A, -1)
    U = np.triu(A, 1)
    M = (D + L) @ np.diag(rD) @ (D + U)
    pattern = A != 0
    assert np.allclose(M[pattern], A[pattern], rtol=1e-12, atol=1e-12 * np.abs(A).max())
    r = np.random.default_rng(73).standard_normal(len(d))
    w = oracle.dilu_precondition(m.lower, m.upper_addr, lo, up, rD, r)
    assert np.allclose(w, np.linalg.solve(M, r), rtol=1e-10, atol=1e-12)
    wt = oracle.dilu_precondition(m.lower, m.upper_addr, lo, up, rD, r, transpose=True)
    assert np.allclose(wt, np.linalg.solve(M.T, r), rtol=1e-10, atol=1e-12)


def test_symmetric_matrix_reduces_to_dic_and_pcg_bitwise():
    """lower == upper: DILU is DIC and PBiCG's recurrences are PCG's, bit for bit."""
    import hexmesh
    c = hexmesh.pressure_case(6, jitter=0.2, permute=True, seed=74, lognormal_gamma=True)
    m = c.mesh
    up, dg = oracle.assemble_laplacian(m, c.gamma, c.bgamma, c.btype)
    rD1, _ = oracle.dilu_factor(m.lower, m.upper_addr, dg, up, up)
    rD2, _ = oracle.dic_factor(m.lower, m.upper_addr, dg, up)
    assert np.array_equal(rD1, rD2)
    r = np.random.default_rng(75).standard_normal(m.n_cells)
    assert np.array_equal(oracle.dilu_precondition(m.lower, m.upper_addr, up, up, rD1, r),
                          oracle.dic_precondition(m.lower, m.upper_addr, up, rD2, r))
    for pre_b, pre_c in [(3, 2), (1, 1), (0, 0)]:
        xb, pb = oracle.pbicg(m.lower, m.upper_addr, dg, up, up, c.b, precond=pre_b, tol=1e-10, max_iter=300)
        xc, pc = oracle.pcg(m.lower, m.upper_addr, dg, up, c.b, precond=pre_c, tol=1e-10, max_iter=300)
        assert pb["n_iter"] == pc["n_iter"] and np.array_equal(xb, xc)


@pytest.mark.parametrize("precond", [0, 1, 3])
def test_pbicg_matches_dense_solve(ac, precond):
    m, lo, up, d, A, b = ac
    x, p = oracle.pbicg(m.lower, m.upper_addr, d, lo, up, b, precond=precond, tol=1e-13, max_iter=2000)
    assert p["converged"] == 1 and p["status"] == 0
    xs = np.linalg.solve(A, b)
    assert np.allclose(x, xs, rtol=1e-9, atol=1e-11 * np.abs(xs).max())


def test_pbicg_dilu_beats_diagonal(ac):
    m, lo, up, d, A, b = ac
    _, p3 = oracle.pbicg(m.lower, m.upper_addr, d, lo, up, b, precond=3, tol=1e-10)
    _, p1 = oracle.pbicg(m.lower, m.upper_addr, d, lo, up, b, precond=1, tol=1e-10)
    assert p3["n_iter"] < p1["n_iter"]
