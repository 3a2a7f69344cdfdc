"""GPU parity of PBiCG on asymmetric matrices (seeded convection-diffusion
systems, tests/asym_cases.py) against the oracle: the DILU factor bit for
bit, x at matched iteration counts to 1e-10 relative for each
preconditioner, and PBiCG on a symmetric matrix against the PCG path."""
import numpy as np
import pytest

import oracle
from asym_cases import asym_case
from gpu_cases import bits, dev

pytestmark = pytest.mark.gpu

CASES = [dict(n=(11, 7, 5), seed=81, jitter=0.2, permute=True, lognormal_gamma=True),
         dict(n=12, seed=82, jitter=0.2, permute=True, lognormal_gamma=True, pe=6.0),
         dict(n=(9, 1, 1), seed=83)]
IDS = ["ragged-pe2", "12c-pe6", "chain9"]


@pytest.fixture(scope="module", params=range(len(CASES)), ids=IDS)
def pc(request):
    from paper_2512_22215_gb300 import LduMesh
    kw = dict(CASES[request.param])
    c, lower, upper, diag = asym_case(kw.pop("n"), kw.pop("seed"), **kw)
    m = c.mesh
    M = LduMesh(m.lower, m.upper_addr, m.n_cells, centres=m.c, asymmetric=True)
    return c, lower, upper, diag, M


@pytest.mark.parametrize("precond", [0, 1, 3])
def test_pbicg_matched_iterations(pc, precond):
    from paper_2512_22215_gb300 import SolverControls
    c, lo, up, d, M = pc
    m = c.mesh
    x, p = M.pbicg_solve(dev(d), dev(lo), dev(up), dev(c.b), None,
                         SolverControls(precond=precond, tolerance=1e-10, max_iter=3000))
    _, po = oracle.pbicg(m.lower, m.upper_addr, d, lo, up, c.b, precond=precond, tol=1e-10, max_iter=3000)
    assert p["converged"] == 1 and p["status"] == 0
    assert p["initial_residual"] == pytest.approx(po["initial_residual"], rel=1e-12)
    assert abs(p["n_iter"] - po["n_iter"]) <= max(1, po["n_iter"] // 20)
    xo, _ = oracle.pbicg(m.lower, m.upper_addr, d, lo, up, c.b, precond=precond, tol=0.0, max_iter=p["n_iter"])
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-9 * np.linalg.norm(xo)
    r = c.b - oracle.amul_asym(m.lower, m.upper_addr, d, lo, up, x.cpu().numpy())
    assert np.abs(r).sum() / np.abs(c.b).sum() < 1e-10


def test_dilu_factor_bitwise(pc):
    from paper_2512_22215_gb300 import SolverControls
    c, lo, up, d, M = pc
    m = c.mesh
    M.pbicg_solve(dev(d), dev(lo), dev(up), dev(c.b), None, SolverControls(precond=3, tolerance=1e-6))
    rDo, bad = oracle.dilu_factor(m.lower, m.upper_addr, d, lo, up)
    assert bad == -1
    assert np.array_equal(bits(M.read_rD().cpu().numpy()), bits(rDo))


def test_pbicg_on_symmetric_matrix_matches_pcg(pc):
    """lower == upper: PBiCG with DILU follows PCG with DIC (same recurrences)."""
    from paper_2512_22215_gb300 import SolverControls
    c, lo, up, d, M = pc
    sym = 0.5 * (lo + up)
    x1, p1 = M.pbicg_solve(dev(d), dev(sym), dev(sym), dev(c.b), None, SolverControls(precond=3, tolerance=1e-10))
    x2, p2 = M.solve(dev(d), dev(sym), dev(c.b), None, SolverControls(precond=2, tolerance=1e-10))
    assert abs(p1["n_iter"] - p2["n_iter"]) <= 1
    assert np.linalg.norm((x1 - x2).cpu().numpy()) <= 1e-9 * np.linalg.norm(x2.cpu().numpy())


def test_pbicg_needs_asymmetric_workspace():
    from paper_2512_22215_gb300 import LduMesh, SolverControls, SpumaError
    c, lo, up, d = asym_case(4, 84)
    m = c.mesh
    M = LduMesh(m.lower, m.upper_addr, m.n_cells)
    with pytest.raises(SpumaError):
        M.pbicg_solve(dev(d), dev(lo), dev(up), dev(c.b), None, SolverControls(precond=3))
