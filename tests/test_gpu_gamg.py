"""GPU parity of GAMG against the oracle (oracle/gamg.py): the same level
hierarchy (built on the host by the library, independently of the oracle),
the solution at matched iteration counts, and repeated solves on one cached
hierarchy with changing coefficients.  Sizes put every level on the first
block (8^3), split the hierarchy between the grid and the first block
(24^3, ragged), and exercise a 1-D chain."""
import numpy as np
import pytest

import hexmesh
import oracle
from gpu_cases import dev, mesh_of
from oracle import gamg as G

pytestmark = pytest.mark.gpu

CASES = [dict(n=8, seed=101, jitter=0.2, permute=True, lognormal_gamma=True),
         dict(n=24, seed=102, jitter=0.2, permute=True, lognormal_gamma=True),
         dict(n=(37, 19, 11), seed=103, jitter=0.2, permute=True, lognormal_gamma=True),
         dict(n=(60, 1, 1), seed=104)]
IDS = ["8c-first-block", "24c-split", "37x19x11-ragged", "chain60"]


@pytest.fixture(scope="module", params=range(len(CASES)), ids=IDS)
def gc(request):
    from paper_2512_22215_gb300 import GamgSolver
    c = hexmesh.pressure_case(**CASES[request.param])
    m = c.mesh
    M = mesh_of(c, centres=True)
    w = np.linalg.norm(m.sf, axis=1)
    S = GamgSolver(M, dev(w))
    up, dg = oracle.assemble_laplacian(m, c.gamma, c.bgamma, c.btype)
    return c, m, M, S, w, up, dg


def test_same_hierarchy(gc):
    c, m, M, S, w, up, dg = gc
    levels = G.hierarchy(m.n_cells, m.lower, m.upper_addr, w)
    assert S.level_cells == [lv["n"] for lv in levels]


def test_matched_iterations(gc):
    from paper_2512_22215_gb300 import SolverControls
    c, m, M, S, w, up, dg = gc
    x, p = S.solve(dev(dg), dev(up), dev(c.b), None, SolverControls(tolerance=1e-10, max_iter=500))
    assert p["converged"] == 1 and p["status"] == 0
    _, po, _ = G.gamg(m.lower, m.upper_addr, dg, up, c.b, w, tol=1e-10, max_iter=500)
    assert p["initial_residual"] == pytest.approx(po["initial_residual"], rel=1e-12)
    assert abs(p["n_iter"] - po["n_iter"]) <= max(2, po["n_iter"] // 20)
    xo, _, _ = G.gamg(m.lower, m.upper_addr, dg, up, c.b, w, tol=0.0, max_iter=p["n_iter"])
    x = x.cpu().numpy()
    assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)
    r = c.b - oracle.amul(m.lower, m.upper_addr, dg, up, x)
    assert np.abs(r).sum() / np.abs(c.b).sum() < 1e-10


def test_cached_hierarchy_new_coefficients(gc):
    """The hierarchy depends on the mesh only; each solve takes new coefficients
    (as in a SIMPLE loop) and an initial guess."""
    from paper_2512_22215_gb300 import SolverControls
    c, m, M, S, w, up, dg = gc
    rng = np.random.default_rng(105)
    gamma2 = c.gamma * np.exp(0.5 * rng.standard_normal(m.n_faces))
    up2, dg2 = oracle.assemble_laplacian(m, gamma2, c.bgamma, c.btype)
    x0 = rng.standard_normal(m.n_cells)
    x, p = S.solve(dev(dg2), dev(up2), dev(c.b), dev(x0), SolverControls(tolerance=1e-9, max_iter=500))
    xo, po, _ = G.gamg(m.lower, m.upper_addr, dg2, up2, c.b, w, x0=x0, tol=0.0, max_iter=p["n_iter"])
    assert p["converged"] == 1
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-8 * np.linalg.norm(xo)


@pytest.mark.parametrize("smoother,coarsest", [(1, 1), (0, 2), (1, 2)], ids=["gs2-diag", "richardson-dic", "gs2-dic"])
def test_smoother_and_coarsest_options_matched_iterations(gc, smoother, coarsest):
    """The two-stage Gauss-Seidel smoother and the DIC-PCG coarsest level
    (the paper's smoother table) at matched V-cycle counts."""
    from paper_2512_22215_gb300 import GamgSolver, SolverControls
    c, m, M, S, w, up, dg = gc
    S2 = GamgSolver(M, dev(w), smoother=smoother, coarsest_precond=coarsest)
    name = "gs2" if smoother == 1 else "richardson"
    x, p = S2.solve(dev(dg), dev(up), dev(c.b), None, SolverControls(tolerance=1e-10, max_iter=500))
    assert p["converged"] == 1 and p["status"] == 0
    _, po, _ = G.gamg(m.lower, m.upper_addr, dg, up, c.b, w, tol=1e-10, max_iter=500, smoother=name,
                      coarsest_precond=coarsest)
    assert abs(p["n_iter"] - po["n_iter"]) <= max(2, po["n_iter"] // 20)
    xo, _, _ = G.gamg(m.lower, m.upper_addr, dg, up, c.b, w, tol=0.0, max_iter=p["n_iter"], smoother=name,
                      coarsest_precond=coarsest)
    x = x.cpu().numpy()
    assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)
    r = c.b - oracle.amul(m.lower, m.upper_addr, dg, up, x)
    assert np.abs(r).sum() / np.abs(c.b).sum() < 1e-10
    assert p["true_rel_residual_l2"] == pytest.approx(np.linalg.norm(r) / np.linalg.norm(c.b), rel=1e-12)


def test_options_rejected():
    from paper_2512_22215_gb300 import GamgSolver, SpumaError
    c = hexmesh.pressure_case(4, seed=106)
    M = mesh_of(c)
    with pytest.raises(SpumaError):
        GamgSolver(M, dev(np.linalg.norm(c.mesh.sf, axis=1)), smoother=2)
    with pytest.raises(SpumaError):
        GamgSolver(M, dev(np.linalg.norm(c.mesh.sf, axis=1)), coarsest_precond=0)


def test_gamg_then_prepared_matrix_calls(gc):
    """A multi-level GAMG solve gathers its level-0 coefficients into the mesh
    handle's matrix region: a preconditioner prepared before is refused until
    it is prepared again, and PCG solves on the same handle are unaffected."""
    from paper_2512_22215_gb300 import SolverControls, SpumaError
    c, m, M, S, w, up, dg = gc
    r = dev(c.b)
    M.prepare(dev(dg), dev(up), 2)
    w0 = M.precondition(r, 2).cpu().numpy()
    x0, p0 = M.solve(dev(dg), dev(up), dev(c.b), None, SolverControls(precond=2, tolerance=1e-10))
    S.solve(dev(dg * 1.5), dev(up * 1.5), dev(c.b), None, SolverControls(tolerance=1e-8, max_iter=500))
    if len(S.level_cells) >= 2:
        with pytest.raises(SpumaError):
            M.precondition(r, 2)
    M.prepare(dev(dg), dev(up), 2)
    assert np.array_equal(M.precondition(r, 2).cpu().numpy(), w0)
    x1, p1 = M.solve(dev(dg), dev(up), dev(c.b), None, SolverControls(precond=2, tolerance=1e-10))
    assert p1["n_iter"] == p0["n_iter"] and np.array_equal(x1.cpu().numpy(), x0.cpu().numpy())


@pytest.mark.slow
def test_large_mesh_hierarchy_and_vcycles():
    """A mesh large enough (110,592 cells, 324,864 faces) for the hierarchy
    build's multi-threaded passes (face keys, radix sort, row and list
    copies): the same level sizes as the oracle, and x after 10 V-cycles of
    each smoother at 1e-8 of the oracle's."""
    from paper_2512_22215_gb300 import GamgSolver, SolverControls
    c = hexmesh.pressure_case(48, seed=107, jitter=0.2, permute=True, lognormal_gamma=True)
    m = c.mesh
    assert m.n_cells >= 65536 and m.n_faces >= 65536
    M = mesh_of(c, centres=True)
    up, dg = oracle.assemble_laplacian(m, c.gamma, c.bgamma, c.btype)
    w = np.abs(up)
    levels = G.hierarchy(m.n_cells, m.lower, m.upper_addr, w)
    for smoother, name in ((0, "richardson"), (1, "gs2")):
        S = GamgSolver(M, dev(w), smoother=smoother)
        assert S.level_cells == [lv["n"] for lv in levels]
        x, p = S.solve(dev(dg), dev(up), dev(c.b), None, SolverControls(tolerance=0.0, max_iter=10))
        assert p["n_iter"] == 10 and p["status"] == 0
        xo, _, _ = G.gamg(m.lower, m.upper_addr, dg, up, c.b, w, tol=0.0, max_iter=10, smoother=name)
        assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-8 * np.linalg.norm(xo)
