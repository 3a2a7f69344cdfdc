"""Pins of the oracle's pressure-correction step (the operators around the
solve in the paper's SIMPLE loop: Gauss linear gradient with linear
interpolation, the explicit non-orthogonal correction of the corrected
laplacian, the right-hand side div(phiHbyA) and the flux reconstruction),
against facts that do not come from the oracle: grid geometry, Gauss's
theorem, a dense incidence matrix, and continuity of the corrected flux."""
import numpy as np
import pytest

import hexmesh
import oracle


def test_weights_uniform_and_stretched():
    c = hexmesh.pressure_case(5)
    assert np.allclose(oracle.fv_weights(c.mesh), 0.5, rtol=0, atol=1e-12)
    # stretched in x only: x-faces interpolate between cell centres at the grid midpoints
    xs = np.cumsum(np.r_[0.0, np.linspace(1.0, 3.0, 6)])
    xs /= xs[-1]
    ys = zs = np.linspace(0.0, 1.0, 4)
    c = hexmesh.pressure_case((6, 3, 3), coords=(xs, ys, zs))
    m = c.mesh
    w = oracle.fv_weights(m)
    xf = m.cf[:, 0]
    xl, xu = m.c[m.lower, 0], m.c[m.upper_addr, 0]
    xface = np.abs(m.sf[:, 0]) > 0.5 * np.linalg.norm(m.sf, axis=1)
    expect = np.abs(xu - xf)[xface] / np.abs(xu - xl)[xface]
    assert np.allclose(w[xface], expect, rtol=1e-13, atol=0)
    assert np.allclose(w[~xface], 0.5, atol=1e-12)
    cj = hexmesh.pressure_case(6, jitter=0.2, permute=True, seed=3)
    wj = oracle.fv_weights(cj.mesh)
    assert np.all((wj > 0.0) & (wj < 1.0))


def test_grad_of_constant_is_zero_without_dirichlet_faces():
    c = hexmesh.pressure_case(5, jitter=0.2, permute=True, seed=51, dirichlet=())
    m = c.mesh
    g = oracle.fv_grad(m, oracle.fv_weights(m), c.btype, np.full(m.n_cells, 3.5))
    assert np.abs(g).max() < 1e-12


@pytest.mark.parametrize("stretched", [False, True])
def test_grad_of_linear_field_exact_in_interior_cells(stretched):
    """Gauss's theorem with planar faces and exact linear interpolation."""
    coords = None
    n = (7, 6, 5)
    if stretched:
        xs = np.cumsum(np.r_[0.0, np.linspace(1.0, 2.0, 7)])
        coords = (xs / xs[-1], np.linspace(0, 1, 7) ** 1.3, np.linspace(0, 1, 6))
    c = hexmesh.pressure_case(n, permute=True, seed=52, coords=coords, dirichlet=())
    m = c.mesh
    a = np.array([0.7, -1.3, 2.1])
    p = m.c @ a + 0.25
    g = oracle.fv_grad(m, oracle.fv_weights(m), c.btype, p)
    ijk = m.cell_ijk
    inner = np.all((ijk > 0) & (ijk < np.array(n) - 1), axis=1)
    assert inner.sum() > 0
    assert np.allclose(g[inner], a, rtol=1e-11, atol=1e-11)


def test_grad_boundary_values():
    """p = 1 - x on a uniform block, Dirichlet p = 0 on x-max, zero gradient
    elsewhere: the boundary values the gradient uses are then exact on every
    face except x-min (p_b = p_cell there), so every cell off x-min gets
    grad p = (-1, 0, 0), the x-max cells through their Dirichlet face."""
    n = (6, 4, 3)
    c = hexmesh.pressure_case(n, permute=True, seed=59, dirichlet=("xmax",))
    m = c.mesh
    g = oracle.fv_grad(m, oracle.fv_weights(m), c.btype, 1.0 - m.c[:, 0])
    off = m.cell_ijk[:, 0] > 0
    assert np.allclose(g[off], [-1.0, 0.0, 0.0], rtol=0, atol=1e-11)
    assert not np.allclose(g[~off], [-1.0, 0.0, 0.0], rtol=0, atol=1e-3)


def test_div_matches_incidence_matrix():
    c = hexmesh.pressure_case((5, 4, 3), jitter=0.2, permute=True, seed=53)
    m = c.mesh
    rng = np.random.default_rng(54)
    phi, bphi = rng.standard_normal(m.n_faces), rng.standard_normal(m.n_bfaces)
    D = np.zeros((m.n_cells, m.n_faces + m.n_bfaces))
    D[m.lower, np.arange(m.n_faces)] = 1.0
    D[m.upper_addr, np.arange(m.n_faces)] = -1.0
    D[m.bface_cell, m.n_faces + np.arange(m.n_bfaces)] = 1.0
    assert np.allclose(oracle.fv_div(m, phi, bphi), D @ np.r_[phi, bphi], rtol=1e-13, atol=1e-13)


def _inputs(c, seed):
    m = c.mesh
    rng = np.random.default_rng(seed)
    magS = np.linalg.norm(m.sf, axis=1)
    phi = rng.standard_normal(m.n_faces) * magS
    bphi = rng.standard_normal(m.n_bfaces) * np.linalg.norm(m.bface_sf, axis=1)
    p_old = rng.standard_normal(m.n_cells)
    return phi, bphi, p_old


def test_correction_vanishes_on_orthogonal_meshes():
    c = hexmesh.pressure_case(6, seed=55, lognormal_gamma=True)
    m = c.mesh
    phi, bphi, p_old = _inputs(c, 56)
    w = oracle.fv_weights(m)
    g = oracle.fv_grad(m, w, c.btype, p_old)
    corr, b = oracle.pressure_rhs(m, w, c.gamma, g, phi, bphi)
    scale = np.abs(c.gamma * np.linalg.norm(m.sf, axis=1) * np.linalg.norm(g[m.lower], axis=1)).max()
    assert np.abs(corr).max() <= 1e-13 * scale
    assert np.allclose(b, -oracle.fv_div(m, phi, bphi), rtol=0, atol=1e-12 * np.abs(b).max())


@pytest.mark.parametrize("n,seed", [(6, 57), ((9, 5, 4), 58)])
def test_corrected_flux_is_divergence_free(n, seed):
    """laplacian(gamma, p) = div(phiHbyA) solved, then phi = phiHbyA minus the
    full corrected laplacian flux: div(phi) vanishes to the solver tolerance.
    A wrong sign or a correction used on one side only breaks it."""
    c = hexmesh.pressure_case(n, jitter=0.2, permute=True, seed=seed, lognormal_gamma=True,
                              dirichlet=("xmax", "zmin"))
    m = c.mesh
    phi, bphi, p_old = _inputs(c, seed + 100)
    up, dg = oracle.assemble_laplacian(m, c.gamma, c.bgamma, c.btype)
    w = oracle.fv_weights(m)
    g = oracle.fv_grad(m, w, c.btype, p_old)
    corr, b = oracle.pressure_rhs(m, w, c.gamma, g, phi, bphi)
    assert np.abs(corr).max() > 1e-3 * np.abs(phi).max()       # jittered: the correction is active
    p, perf = oracle.pcg(m.lower, m.upper_addr, dg, up, b, tol=1e-15, max_iter=5000)
    phin, bphin = oracle.pressure_flux(m, up, corr, p, phi, c.bgamma, c.btype, bphi)
    div0 = oracle.fv_div(m, phi, bphi)
    div1 = oracle.fv_div(m, phin, bphin)
    assert np.abs(div1).max() <= 1e-10 * np.abs(div0).max()
    # zero-gradient boundary fluxes are untouched, Dirichlet ones change
    assert np.array_equal(bphin[c.btype == 0], bphi[c.btype == 0])
    assert np.any(bphin[c.btype == 1] != bphi[c.btype == 1])
