"""GPU: the solver report's true residual ||b - A x||_2 / ||b||_2, computed on
the device at the end of every solve kind, against the same quantity on the
host from the returned x with the oracle's face-loop Amul (bit-identical
r = b - A x, only the order of the sums of squares differs: 1e-12 relative)."""
import numpy as np
import pytest

import oracle
from asym_cases import asym_case
from gpu_cases import assemble_oracle, case, dev, mesh_of

pytestmark = pytest.mark.gpu


def host_true(b, r):
    return np.linalg.norm(r) / np.linalg.norm(b)


@pytest.mark.parametrize("precond,precision", [(2, 0), (1, 0), (0, 0), (2, 1), (2, 3)],
                         ids=["dic-f64", "diag-f64", "none-f64", "dic-mixed", "dic-mixed-restart"])
def test_pcg_true_residual(precond, precision):
    from paper_2512_22215_gb300 import SolverControls
    c = case((19, 13, 11), jitter=0.2, permute=True, seed=61, lognormal=True)
    m = c.mesh
    M = mesh_of(c, centres=True)
    uo, do = assemble_oracle(c)
    x, p = M.solve(dev(do), dev(uo), dev(c.b), None,
                   SolverControls(precond=precond, precision=precision, tolerance=1e-9))
    assert p["status"] == 0 and p["converged"] == 1
    r = c.b - oracle.amul(m.lower, m.upper_addr, do, uo, x.cpu().numpy())
    assert p["true_rel_residual_l2"] == pytest.approx(host_true(c.b, r), rel=1e-12)
    # the L1 residual the solver stops on and the L2 report describe the same x
    assert np.abs(r).sum() / np.abs(c.b).sum() < 1e-9


def test_pcg_true_residual_of_a_partial_solve():
    """A solve stopped after 3 iterations: the report describes the x it returns."""
    from paper_2512_22215_gb300 import SolverControls
    c = case(14, jitter=0.2, permute=True, seed=62, lognormal=True)
    m = c.mesh
    M = mesh_of(c)
    uo, do = assemble_oracle(c)
    x, p = M.solve(dev(do), dev(uo), dev(c.b), None, SolverControls(precond=2, tolerance=0.0, max_iter=3))
    r = c.b - oracle.amul(m.lower, m.upper_addr, do, uo, x.cpu().numpy())
    assert p["n_iter"] == 3 and p["converged"] == 0
    assert p["true_rel_residual_l2"] == pytest.approx(host_true(c.b, r), rel=1e-12)
    assert p["true_rel_residual_l2"] > 1e-6


def test_pbicg_true_residual():
    from paper_2512_22215_gb300 import LduMesh, SolverControls
    c, lo, up, d = asym_case((11, 7, 5), 81, jitter=0.2, permute=True, lognormal_gamma=True)
    m = c.mesh
    M = LduMesh(m.lower, m.upper_addr, m.n_cells, centres=m.c, asymmetric=True)
    x, p = M.pbicg_solve(dev(d), dev(lo), dev(up), dev(c.b), None, SolverControls(precond=3, tolerance=1e-10))
    assert p["status"] == 0 and p["converged"] == 1
    r = c.b - oracle.amul_asym(m.lower, m.upper_addr, d, lo, up, x.cpu().numpy())
    assert p["true_rel_residual_l2"] == pytest.approx(host_true(c.b, r), rel=1e-12)


def test_gamg_true_residual():
    from paper_2512_22215_gb300 import GamgSolver, SolverControls
    c = case(24, jitter=0.2, permute=True, seed=102, lognormal=True)
    m = c.mesh
    M = mesh_of(c, centres=True)
    uo, do = assemble_oracle(c)
    S = GamgSolver(M, dev(np.linalg.norm(m.sf, axis=1)))
    x, p = S.solve(dev(do), dev(uo), dev(c.b), None, SolverControls(tolerance=1e-10, max_iter=500))
    assert p["status"] == 0 and p["converged"] == 1
    r = c.b - oracle.amul(m.lower, m.upper_addr, do, uo, x.cpu().numpy())
    assert p["true_rel_residual_l2"] == pytest.approx(host_true(c.b, r), rel=1e-12)


def test_true_residual_with_zero_rhs():
    """b = 0 from a nonzero guess: the report is the absolute ||A x||_2."""
    from paper_2512_22215_gb300 import SolverControls
    c = case(9, jitter=0.2, permute=True, seed=63, lognormal=True)
    m = c.mesh
    M = mesh_of(c)
    uo, do = assemble_oracle(c)
    x0 = np.random.default_rng(64).standard_normal(m.n_cells)
    b = np.zeros(m.n_cells)
    x, p = M.solve(dev(do), dev(uo), dev(b), dev(x0), SolverControls(precond=2, tolerance=0.0, max_iter=2))
    r = -oracle.amul(m.lower, m.upper_addr, do, uo, x.cpu().numpy())
    assert p["true_rel_residual_l2"] == pytest.approx(np.linalg.norm(r), rel=1e-12)
