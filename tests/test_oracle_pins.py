"""Pins of the CPU oracle against facts that do not come from the oracle itself:
dense linear algebra (numpy), closed forms, invariants, special cases.

Each test names the definition it checks; the oracle's definitions follow the
paper's LDU matrix (Sec. 2.1), Amul (Sec. 4.2), DIC and diagonal
preconditioning (Sec. 4.3, appendix fvSolution listing) and PCG with
tolerance/relTol/maxIter/minIter (appendix).
"""
import json
import os

import numpy as np
import pytest

import hexmesh
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense(l, u, diag, upper):
    n = len(diag)
    A = np.zeros((n, n))
    A[np.arange(n), np.arange(n)] = diag
    A[l, u] = upper
    A[u, l] = upper
    return A


def case(n, **kw):
    c = hexmesh.pressure_case(n, **kw)
    up, dg = oracle.assemble_laplacian(c.mesh, c.gamma, c.bgamma, c.btype)
    return c, up, dg


# ----------------------------------------------------------------- mesh ----
@pytest.mark.parametrize("n,jit,perm", [(4, 0.0, False), (6, 0.2, True), ((5, 3, 4), 0.2, True)])
def test_mesh_closed_and_volume(n, jit, perm):
    m, _ = hexmesh.hex_block(n, jitter=jit, permute=perm, seed=3)
    s = np.zeros((m.n_cells, 3))
    np.add.at(s, m.lower, m.sf)
    np.add.at(s, m.upper_addr, -m.sf)
    np.add.at(s, m.bface_cell, m.bface_sf)
    assert np.abs(s).max() < 1e-15
    assert abs(m.v.sum() - 1.0) < 1e-13
    assert (m.v > 0).all()
    assert (m.lower < m.upper_addr).all()
    key = m.lower.astype(np.int64) * m.n_cells + m.upper_addr
    assert (np.diff(key) > 0).all()          # sorted by (l, u), no duplicates
    # S points from lower to upper: (C_u - C_l) . S > 0 on these meshes
    d = m.c[m.upper_addr] - m.c[m.lower]
    assert (np.einsum("ij,ij->i", d, m.sf) > 0).all()


def test_mesh_uniform_geometry():
    m, _ = hexmesh.hex_block(4)
    h = 0.25
    assert np.allclose(np.linalg.norm(m.sf, axis=1), h * h, rtol=0, atol=1e-16)
    assert np.allclose(m.v, h ** 3, rtol=0, atol=1e-17)
    ijk = m.cell_ijk
    assert np.allclose(m.c, (ijk + 0.5) * h, rtol=0, atol=1e-15)


# ------------------------------------------------------------- assembly ----
def test_assembly_uniform_closed_form():
    """Orthogonal uniform mesh, gamma = 1: a_f = h^2/h = h; a Dirichlet face
    adds h^2/(h/2) = 2h; diag = (number of internal faces) h (+2h)."""
    c, up, dg = case(4)
    h = 0.25
    assert np.allclose(up, -h, rtol=1e-15, atol=0)
    m = c.mesh
    nfaces = np.bincount(m.lower, minlength=m.n_cells) + np.bincount(m.upper_addr, minlength=m.n_cells)
    ndir = np.bincount(m.bface_cell[c.btype == 1], minlength=m.n_cells)
    assert np.allclose(dg, nfaces * h + ndir * 2 * h, rtol=1e-15, atol=0)


def test_assembly_golden_two_cells():
    """Hand-derived coefficients of single faces (tests/golden/assembly_faces.json),
    including a face where the 0.05|d| clamp of the corrected delta is active."""
    with open(os.path.join(GOLDEN, "assembly_faces.json")) as fh:
        g = json.load(fh)
    for rec in g["faces"]:
        m = hexmesh.Mesh(n_cells=2, n_faces=1, lower=np.array([0], np.int32),
                         upper_addr=np.array([1], np.int32), sf=np.array([rec["sf"]], float),
                         cf=np.zeros((1, 3)), c=np.array([rec["c_l"], rec["c_u"]], float),
                         v=np.ones(2), bface_cell=np.zeros(0, np.int32),
                         bface_sf=np.zeros((0, 3)), bface_cf=np.zeros((0, 3)),
                         bface_patch=np.zeros(0, np.int8))
        up, dg = oracle.assemble_laplacian(m, np.array([rec["gamma"]]), np.zeros(0), np.zeros(0, np.int8))
        assert up[0] == pytest.approx(-rec["a"], rel=1e-14)
        assert dg == pytest.approx([rec["a"], rec["a"]], rel=1e-14)


@pytest.mark.parametrize("seed", [2, 7])
def test_assembly_m_matrix_invariants(seed):
    c, up, dg = case(6, jitter=0.2, permute=True, seed=seed, lognormal_gamma=True)
    m = c.mesh
    assert (up < 0).all() and (dg > 0).all()
    rowsum = dg.copy()
    np.add.at(rowsum, m.lower, up)
    np.add.at(rowsum, m.upper_addr, up)
    dir_rows = np.zeros(m.n_cells, bool)
    dir_rows[m.bface_cell[c.btype == 1]] = True
    # interior rows: zero row sums up to the rounding of the diagonal sum
    assert np.all(np.abs(rowsum[~dir_rows]) <= 8 * np.finfo(float).eps * dg[~dir_rows])
    # Dirichlet rows: strictly diagonally dominant
    assert np.all(rowsum[dir_rows] > 0)
    A = dense(m.lower, m.upper_addr, dg, up)
    assert np.linalg.eigvalsh(A).min() > 0


# ----------------------------------------------------------------- Amul ----
@pytest.mark.parametrize("n,perm", [(5, False), (6, True)])
def test_amul_matches_dense(n, perm):
    c, up, dg = case(n, jitter=0.2, permute=perm, seed=4, lognormal_gamma=True)
    m = c.mesh
    x = np.random.default_rng(0).standard_normal(m.n_cells)
    y = oracle.amul(m.lower, m.upper_addr, dg, up, x)
    A = dense(m.lower, m.upper_addr, dg, up)
    ref = A @ x
    scale = np.abs(A) @ np.abs(x)
    assert np.all(np.abs(y - ref) <= 8 * np.finfo(float).eps * scale)


def test_amul_f32_matches_dense():
    c, up, dg = case(5, jitter=0.2, permute=True, seed=5, lognormal_gamma=True)
    m = c.mesh
    x = np.random.default_rng(1).standard_normal(m.n_cells).astype(np.float32)
    y = oracle.amul(m.lower, m.upper_addr, dg.astype(np.float32), up.astype(np.float32), x)
    A = dense(m.lower, m.upper_addr, dg.astype(np.float32).astype(float), up.astype(np.float32).astype(float))
    ref = A @ x.astype(float)
    scale = np.abs(A) @ np.abs(x.astype(float))
    assert np.all(np.abs(y - ref) <= 8 * np.finfo(np.float32).eps * scale)


def _fma32(a, b, c):
    """float32 fused multiply-add: the product of two float32 values is exact in
    float64, so the only rounding left is that of the float64 sum (and its
    rounding to float32; a double rounding there is a one-in-millions event that
    these inputs do not hit, checked below by the agreement itself)."""
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def test_amul_f32_rounding_bitwise():
    """The FP32 Amul restated element by element: d x rounded to float, then
    each face's two terms as float FMAs in face order (float products are exact
    in float64, so a float FMA is the float64 sum rounded to float; see
    _fma32).  The oracle agrees bit for bit; summing the terms with separate
    float roundings does not."""
    c, up, dg = case((6, 5, 4), jitter=0.2, permute=True, seed=5, lognormal_gamma=True)
    m = c.mesh
    d32, u32 = dg.astype(np.float32), up.astype(np.float32)
    x = np.random.default_rng(1).standard_normal(m.n_cells).astype(np.float32)
    y = oracle.amul(m.lower, m.upper_addr, d32, u32, x)

    def restate(term):
        yr = (d32 * x).astype(np.float32)
        for f in range(m.n_faces):
            l_, u = m.lower[f], m.upper_addr[f]
            yr[u] = term(u32[f], x[l_], yr[u])
            yr[l_] = term(u32[f], x[u], yr[l_])
        return yr

    assert np.array_equal(y.view(np.uint32), restate(_fma32).view(np.uint32))
    sep = restate(lambda a, b, c_: np.float32(np.float32(a * b) + c_))
    assert not np.array_equal(y.view(np.uint32), sep.view(np.uint32))


# ------------------------------------------------------------------ DIC ----
@pytest.mark.parametrize("perm", [False, True])
def test_dic_factor_reproduces_diagonal_and_pattern(perm):
    """DIC: M = (P + L) P^-1 (P + L^T) with P = diag(pivots) has diag(M) = diag(A)
    and M = A on A's off-diagonal pattern (hex graphs have no triangles, so the
    fill L P^-1 L^T falls outside the pattern)."""
    c, up, dg = case(5, jitter=0.2, permute=perm, seed=6, lognormal_gamma=True)
    m = c.mesh
    rD, bad = oracle.dic_factor(m.lower, m.upper_addr, dg, up)
    assert bad == -1 and (rD > 0).all()
    A = dense(m.lower, m.upper_addr, dg, up)
    P = np.diag(1.0 / rD)
    L = np.tril(A, -1)
    M = (P + L) @ np.linalg.inv(P) @ (P + L.T)
    pattern = A != 0
    assert np.allclose(M[pattern], A[pattern], rtol=1e-12, atol=0)
    # apply: w = M^-1 r
    r = np.random.default_rng(2).standard_normal(m.n_cells)
    w = oracle.dic_precondition(m.lower, m.upper_addr, up, rD, r)
    assert np.allclose(w, np.linalg.solve(M, r), rtol=1e-10, atol=1e-12 * np.abs(w).max())


def test_dic_f32_sweeps_close_to_f64():
    c, up, dg = case(5, jitter=0.2, permute=True, seed=6, lognormal_gamma=True)
    m = c.mesh
    rD, _ = oracle.dic_factor(m.lower, m.upper_addr, dg, up)
    r = np.random.default_rng(3).standard_normal(m.n_cells)
    w64 = oracle.dic_precondition(m.lower, m.upper_addr, up, rD, r)
    w32 = oracle.dic_precondition(m.lower, m.upper_addr, up, rD, r.astype(np.float32))
    assert w32.dtype == np.float32
    assert np.abs(w32 - w64).max() <= 1e-5 * np.abs(w64).max()


def test_dic_f32_sweeps_rounding_reading_bitwise():
    """The mixed form's FP32 sweeps, restated element by element: the diagonal
    scale is rD rounded to float, each sweep coefficient the FP64 product rD a
    rounded to float, each term one float FMA, faces ascending (forward) then
    descending (backward).  The oracle's FP32 sweeps agree bit for bit; the
    other reading of the coefficient, float(rD) * float(a) in float, gives other
    bits."""
    c, up, dg = case((6, 5, 4), jitter=0.2, permute=True, seed=6, lognormal_gamma=True)
    m = c.mesh
    rD, _ = oracle.dic_factor(m.lower, m.upper_addr, dg, up)
    r = np.random.default_rng(3).standard_normal(m.n_cells).astype(np.float32)
    w32 = oracle.dic_precondition(m.lower, m.upper_addr, up, rD, r)

    def sweep(coef):
        w = (rD.astype(np.float32) * r).astype(np.float32)
        for f in range(m.n_faces):
            u, l_ = m.upper_addr[f], m.lower[f]
            w[u] = _fma32(-coef(u, f), w[l_], w[u])
        for f in range(m.n_faces - 1, -1, -1):
            u, l_ = m.upper_addr[f], m.lower[f]
            w[l_] = _fma32(-coef(l_, f), w[u], w[l_])
        return w

    w_ref = sweep(lambda i, f: np.float32(rD[i] * up[f]))
    assert np.array_equal(w32.view(np.uint32), w_ref.view(np.uint32))
    w_alt = sweep(lambda i, f: np.float32(np.float32(rD[i]) * np.float32(up[f])))
    assert not np.array_equal(w32.view(np.uint32), w_alt.view(np.uint32))


def test_dic_chain_is_exact_cholesky():
    """On a 1-D chain (a tree) DIC has no fill, so M = A and DIC-PCG converges
    in one iteration."""
    c, up, dg = case((12, 1, 1), lognormal_gamma=True, seed=8)
    m = c.mesh
    x, perf = oracle.pcg(m.lower, m.upper_addr, dg, up, c.b, precond=oracle.PRECOND_DIC, tol=1e-14)
    assert perf["n_iter"] == 1
    A = dense(m.lower, m.upper_addr, dg, up)
    assert np.allclose(x, np.linalg.solve(A, c.b), rtol=1e-12)


def test_dic_sign_symmetry_bitwise():
    c, up, dg = case(4, jitter=0.2, permute=True, seed=9, lognormal_gamma=True)
    m = c.mesh
    rD, _ = oracle.dic_factor(m.lower, m.upper_addr, dg, up)
    rDn, bad = oracle.dic_factor(m.lower, m.upper_addr, -dg, -up)
    assert bad == 0                       # negative definite: pivot check fires
    assert np.array_equal(rDn, -rD)
    r = np.random.default_rng(4).standard_normal(m.n_cells)
    w = oracle.dic_precondition(m.lower, m.upper_addr, up, rD, r)
    wn = oracle.dic_precondition(m.lower, m.upper_addr, -up, rDn, -r)
    assert np.array_equal(w, wn)


# ------------------------------------------------------------------ PCG ----
@pytest.mark.parametrize("precond", [0, 1, 2])
@pytest.mark.parametrize("n", [2, 4, (3, 5, 2)])
def test_pcg_matches_dense_solve(precond, n):
    c, up, dg = case(n, jitter=0.2, permute=True, seed=10, lognormal_gamma=True)
    m = c.mesh
    x, perf = oracle.pcg(m.lower, m.upper_addr, dg, up, c.b, precond=precond, tol=1e-14)
    A = dense(m.lower, m.upper_addr, dg, up)
    xs = np.linalg.solve(A, c.b)
    assert perf["converged"] == 1 and perf["singular"] == 0
    assert np.linalg.norm(x - xs) <= 1e-11 * np.linalg.norm(xs)
    if m.n_cells <= 8:
        assert perf["n_iter"] <= m.n_cells + 1      # CG finite termination (+1 rounding)


def test_pcg_matches_dense_8cubed():
    c, up, dg = case(8, jitter=0.2, permute=True, seed=11, lognormal_gamma=True)
    m = c.mesh
    A = dense(m.lower, m.upper_addr, dg, up)
    xs = np.linalg.solve(A, c.b)
    for pc in (1, 2):
        x, perf = oracle.pcg(m.lower, m.upper_addr, dg, up, c.b, precond=pc, tol=1e-14)
        assert np.linalg.norm(x - xs) <= 1e-11 * np.linalg.norm(xs)


def test_pcg_linear_field_exact():
    """Orthogonal graded mesh, gamma = 1, p = 0 on x-max, zero gradient on y/z,
    prescribed flux on x-min (b = -g|S| there): the discrete solution is the
    linear field p = g (x_c - 1) exactly."""
    xs = np.cumsum(np.r_[0.0, 1.15 ** np.arange(10)])
    xs /= xs[-1]
    ys = np.linspace(0, 1, 5)
    zs = np.r_[0.0, 0.3, 0.45, 1.0]
    c = hexmesh.pressure_case((10, 4, 3), coords=(xs, ys, zs), seed=12)
    m = c.mesh
    up, dg = oracle.assemble_laplacian(m, c.gamma, c.bgamma, c.btype)
    g = 2.5
    b = np.zeros(m.n_cells)
    xmin = m.bface_patch == hexmesh.PATCHES.index("xmin")
    np.add.at(b, m.bface_cell[xmin], -g * np.linalg.norm(m.bface_sf[xmin], axis=1))
    for pc in (0, 1, 2):
        x, perf = oracle.pcg(m.lower, m.upper_addr, dg, up, b, precond=pc, tol=1e-15)
        assert np.allclose(x, g * (m.c[:, 0] - 1.0), rtol=0, atol=1e-12)


def test_pcg_sign_flip_bitwise():
    c, up, dg = case(5, jitter=0.2, permute=True, seed=13, lognormal_gamma=True)
    m = c.mesh
    for pc in (0, 1):
        x1, p1 = oracle.pcg(m.lower, m.upper_addr, dg, up, c.b, precond=pc, tol=1e-10)
        x2, p2 = oracle.pcg(m.lower, m.upper_addr, -dg, -up, -c.b, precond=pc, tol=1e-10)
        assert np.array_equal(x1, x2) and p1["n_iter"] == p2["n_iter"]


def test_pcg_norm_factor_closed_forms():
    c, up, dg = case(4, jitter=0.2, permute=True, seed=14, lognormal_gamma=True)
    m = c.mesh
    nf0 = oracle.norm_factor(m.lower, m.upper_addr, dg, up, np.zeros(m.n_cells), c.b)
    assert nf0 == pytest.approx(np.abs(c.b).sum() + 1e-20, rel=1e-14)
    # constant x: A x = s x, so |Ax - s xbar| = 0 and the factor is sum|b - s xbar|
    x = np.full(m.n_cells, 0.75)
    A = dense(m.lower, m.upper_addr, dg, up)
    s = A.sum(axis=1)
    nf = oracle.norm_factor(m.lower, m.upper_addr, dg, up, x, c.b)
    assert nf == pytest.approx(np.abs(c.b - s * 0.75).sum(), rel=1e-12)


def test_pcg_controls():
    c, up, dg = case(6, jitter=0.2, permute=True, seed=15, lognormal_gamma=True)
    m = c.mesh
    args = (m.lower, m.upper_addr, dg, up, c.b)
    _, p = oracle.pcg(*args, tol=1e-12, max_iter=3)
    assert p["n_iter"] == 3 and p["converged"] == 0
    _, p = oracle.pcg(*args, tol=10.0, min_iter=0)
    assert p["n_iter"] == 0 and p["converged"] == 1
    _, p = oracle.pcg(*args, tol=10.0, min_iter=2)
    assert p["n_iter"] == 2
    _, p = oracle.pcg(*args, tol=0.0, rel_tol=1e-3)
    assert p["converged"] == 1 and p["final_residual"] < 1e-3 * p["initial_residual"]
    # x0 = exact solution: initial residual ~ 0
    xs = np.linalg.solve(dense(m.lower, m.upper_addr, dg, up), c.b)
    _, p = oracle.pcg(*args, x0=xs, tol=1e-10)
    assert p["n_iter"] == 0 and p["initial_residual"] < 1e-12


def test_pcg_diagonal_matrix_one_iteration():
    n = 7
    dg = np.linspace(1, 3, n)
    b = np.arange(1.0, n + 1)
    e = np.zeros(0, np.int32)
    x, p = oracle.pcg(e, e, dg, np.zeros(0), b, precond=1, tol=1e-14)
    assert p["n_iter"] == 1 and np.allclose(x, b / dg, rtol=1e-15)


def test_pcg_singular_detection():
    # zero matrix: sigma = 0 -> singular flag, no NaN propagation into x
    n = 4
    e = np.zeros(0, np.int32)
    x, p = oracle.pcg(e, e, np.zeros(n), np.zeros(0), np.ones(n), precond=0, tol=1e-10)
    assert p["singular"] == 1 and np.all(x == 0)


# ---------------------------------------------------------------- mixed ----
def test_mixed_ir_reaches_fp64_solution():
    c, up, dg = case(10, jitter=0.2, permute=True, seed=16, lognormal_gamma=True)
    m = c.mesh
    A = dense(m.lower, m.upper_addr, dg, up)
    xs = np.linalg.solve(A, c.b)
    x, p = oracle.mixed_ir(m.lower, m.upper_addr, dg, up, c.b, tol=1e-10, inner_rel_tol=1e-4)
    assert p["converged"] == 1 and p["n_outer"] >= 2
    r = c.b - A @ x
    assert np.abs(r).sum() / np.abs(c.b).sum() < 1e-10
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= kappa * 1e-10


def test_mixed_reliable_converges_without_restart_penalty():
    """Reliable updates keep the FP32 Krylov space: the FP64 residual reaches the
    tolerance, the solution is the FP64 system's, and the iteration count stays
    close to the FP64 PCG's (a restarted refinement needs many more)."""
    c, up, dg = case(16, jitter=0.2, permute=True, seed=20, lognormal_gamma=True)
    m = c.mesh
    A = dense(m.lower, m.upper_addr, dg, up)
    xs = np.linalg.solve(A, c.b)
    _, p64 = oracle.pcg(m.lower, m.upper_addr, dg, up, c.b, tol=1e-10)
    x, p = oracle.mixed_reliable(m.lower, m.upper_addr, dg, up, c.b, tol=1e-10, delta=0.1)
    assert p["converged"] == 1 and p["n_outer"] >= 5
    r = c.b - A @ x
    assert np.abs(r).sum() / np.abs(c.b).sum() < 1e-10
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= np.linalg.cond(A) * 1e-10
    assert p["n_iter"] <= 1.15 * p64["n_iter"] + 2
    _, pr = oracle.mixed_ir(m.lower, m.upper_addr, dg, up, c.b, tol=1e-10, inner_rel_tol=1e-4)
    assert pr["n_iter"] > p["n_iter"]
    # a tolerance already met: no iteration, no update
    _, p0 = oracle.mixed_reliable(m.lower, m.upper_addr, dg, up, c.b, x0=xs, tol=1e-6)
    assert p0["n_iter"] == 0 and p0["n_outer"] == 0


# -------------------------------------------------------------- adjoint ----
def test_adjoint_dense_and_identity():
    c = hexmesh.pressure_case(6, jitter=0.2, permute=True, seed=17, lognormal_gamma=True, with_target=True)
    m = c.mesh
    up, dg = oracle.assemble_laplacian(m, c.gamma, c.bgamma, c.btype)
    A = dense(m.lower, m.upper_addr, dg, up)
    x = np.linalg.solve(A, c.b)
    g = x - c.x_t
    lam, du, dd, _ = oracle.adjoint(m.lower, m.upper_addr, dg, up, x, g, tol=1e-15)
    assert np.allclose(lam, np.linalg.solve(A, g), rtol=1e-10, atol=1e-12 * np.abs(lam).max())
    assert np.dot(lam, c.b) == pytest.approx(np.dot(g, x), rel=1e-10)
    # dense gradient of L = 0.5|A^-1 b - x_t|^2 w.r.t. A: -lambda x^T, symmetrised per face
    G = -np.outer(lam, x)
    assert np.allclose(du, G[m.lower, m.upper_addr] + G[m.upper_addr, m.lower], rtol=1e-9, atol=1e-13)
    assert np.allclose(dd, np.diag(G), rtol=1e-9, atol=1e-13)


def test_adjoint_finite_differences():
    c = hexmesh.pressure_case(5, jitter=0.2, permute=True, seed=18, lognormal_gamma=True, with_target=True)
    m = c.mesh
    up, dg = oracle.assemble_laplacian(m, c.gamma, c.bgamma, c.btype)
    args = (m.lower, m.upper_addr)

    def loss(upper, diag, b):
        x, _ = oracle.pcg(*args, diag, upper, b, tol=1e-15, max_iter=5000)
        return 0.5 * np.sum((x - c.x_t) ** 2), x

    L0, x = loss(up, dg, c.b)
    lam, du, dd, _ = oracle.adjoint(*args, dg, up, x, x - c.x_t, tol=1e-15)
    rng = np.random.default_rng(5)
    h = 1e-6
    for _ in range(8):
        vb = rng.standard_normal(m.n_cells)
        vu = rng.standard_normal(m.n_faces) * np.abs(up) * 0.1
        fd_b = (loss(up, dg, c.b + h * vb)[0] - loss(up, dg, c.b - h * vb)[0]) / (2 * h)
        fd_u = (loss(up + h * vu, dg, c.b)[0] - loss(up - h * vu, dg, c.b)[0]) / (2 * h)
        assert fd_b == pytest.approx(np.dot(lam, vb), rel=1e-6)
        assert fd_u == pytest.approx(np.dot(du, vu), rel=1e-6)


# ------------------------------------------------ assembly adjoint (dL/dgamma) ----
def _assembly_grads(c, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(c.mesh.n_faces), rng.standard_normal(c.mesh.n_cells)


def test_assembly_adjoint_homogeneity():
    """upper and diag are homogeneous of degree one in (gamma, bgamma), so
    gamma.dL/dgamma + bgamma.dL/dbgamma = upper.dL/dupper + diag.dL/ddiag."""
    c, up, dg = case(6, jitter=0.2, permute=True, seed=31, lognormal_gamma=True)
    gu, gd = _assembly_grads(c, 32)
    gg, gb = oracle.assembly_adjoint(c.mesh, gu, gd, c.btype)
    lhs = np.dot(gg, c.gamma) + np.dot(gb, c.bgamma)
    assert lhs == pytest.approx(np.dot(gu, up) + np.dot(gd, dg), rel=1e-12)


def test_assembly_adjoint_directional_derivative():
    """The assembly is linear in the diffusivities: a central difference of
    phi = dL/dupper.upper + dL/ddiag.diag along any direction is exact up to
    rounding, and equals the adjoint's directional derivative."""
    c, up, dg = case((5, 4, 3), jitter=0.2, permute=True, seed=33, lognormal_gamma=True)
    m = c.mesh
    gu, gd = _assembly_grads(c, 34)
    gg, gb = oracle.assembly_adjoint(m, gu, gd, c.btype)
    rng = np.random.default_rng(35)
    for _ in range(4):
        vg = rng.standard_normal(m.n_faces) * c.gamma
        vb = rng.standard_normal(m.n_bfaces) * c.bgamma

        def phi(t):
            u1, d1 = oracle.assemble_laplacian(m, c.gamma + t * vg, c.bgamma + t * vb, c.btype)
            return np.dot(gu, u1) + np.dot(gd, d1)

        fd = (phi(0.5) - phi(-0.5)) / 1.0
        assert fd == pytest.approx(np.dot(gg, vg) + np.dot(gb, vb), rel=1e-9)
    # zero-gradient faces get no gradient, Dirichlet faces do
    assert np.all(gb[c.btype != 1] == 0.0) and np.any(gb[c.btype == 1] != 0.0)


def test_assembly_adjoint_uniform_closed_form():
    """Uniform cubes of side h: d a_f / d gamma_f = |S| / |d| = h for internal
    faces and h^2 / (h/2) = 2h for Dirichlet faces."""
    n = 4
    c, up, dg = case(n, seed=36)
    m = c.mesh
    h = 1.0 / n
    gu, gd = _assembly_grads(c, 37)
    gg, gb = oracle.assembly_adjoint(m, gu, gd, c.btype)
    assert np.allclose(gg, ((gd[m.lower] + gd[m.upper_addr]) - gu) * h, rtol=1e-12, atol=0)
    dir_ = c.btype == 1
    assert np.allclose(gb[dir_], gd[m.bface_cell[dir_]] * 2 * h, rtol=1e-12, atol=0)


def test_gamma_gradient_through_solve_finite_differences():
    """L(gamma) = 0.5 |x(gamma) - x_t|^2 with A(gamma) x = b: the solve's
    adjoint followed by the assembly's against central differences."""
    c = hexmesh.pressure_case(4, jitter=0.2, permute=True, seed=38, lognormal_gamma=True, with_target=True)
    m = c.mesh
    args = (m.lower, m.upper_addr)

    def loss(gamma, bgamma):
        up, dg = oracle.assemble_laplacian(m, gamma, bgamma, c.btype)
        x, _ = oracle.pcg(*args, dg, up, c.b, tol=1e-15, max_iter=5000)
        return 0.5 * np.sum((x - c.x_t) ** 2), x, up, dg

    L0, x, up, dg = loss(c.gamma, c.bgamma)
    _, du, dd, _ = oracle.adjoint(*args, dg, up, x, x - c.x_t, tol=1e-15)
    gg, gb = oracle.assembly_adjoint(m, du, dd, c.btype)
    rng = np.random.default_rng(39)
    h = 1e-6
    for _ in range(4):
        vg = rng.standard_normal(m.n_faces) * c.gamma
        vb = rng.standard_normal(m.n_bfaces) * c.bgamma
        fd = (loss(c.gamma + h * vg, c.bgamma + h * vb)[0] - loss(c.gamma - h * vg, c.bgamma - h * vb)[0]) / (2 * h)
        assert fd == pytest.approx(np.dot(gg, vg) + np.dot(gb, vb), rel=1e-6)


def test_pcg_norm_factor_shift_invariance():
    """With zero row sums (all-Neumann boundary) A (x + c) - s (xbar + c) = A x - s xbar
    for every constant c, so the normalisation factor does not depend on the
    level of x.  With any boundary it bounds the initial residual (triangle
    inequality: |b - Ax| <= |b - t| + |Ax - t|) and the PCG's initial residual is
    sum|b - A x0| over it."""
    c = hexmesh.pressure_case(4, jitter=0.2, permute=True, seed=19, lognormal_gamma=True, dirichlet=())
    m = c.mesh
    up, dg = oracle.assemble_laplacian(m, c.gamma, c.bgamma, c.btype)
    x = np.random.default_rng(6).standard_normal(m.n_cells)
    nf = oracle.norm_factor(m.lower, m.upper_addr, dg, up, x, c.b)
    for shift in (3.0, -40.0):
        assert oracle.norm_factor(m.lower, m.upper_addr, dg, up, x + shift, c.b) == pytest.approx(nf, rel=1e-12)
    c, up, dg = case(4, jitter=0.2, permute=True, seed=19, lognormal_gamma=True)
    m = c.mesh
    x = 50.0 * np.random.default_rng(7).standard_normal(m.n_cells)
    nf = oracle.norm_factor(m.lower, m.upper_addr, dg, up, x, c.b)
    r = c.b - oracle.amul(m.lower, m.upper_addr, dg, up, x)
    assert np.abs(r).sum() <= nf
    _, p = oracle.pcg(m.lower, m.upper_addr, dg, up, c.b, x0=x, tol=1e-30, max_iter=1)
    assert p["initial_residual"] == pytest.approx(np.abs(r).sum() / nf, rel=1e-13)
