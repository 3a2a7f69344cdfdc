"""GPU parity of the pressure-correction step around the solve: interpolation
weights, Gauss linear gradient, the corrected-laplacian right-hand side and
correction flux, the flux reconstruction and the divergence, each bit-exact
against the oracle (same per-cell order, no contraction); then one whole
step whose corrected flux is divergence-free to the solver tolerance."""
import numpy as np
import pytest

import hexmesh
import oracle
from gpu_cases import bits, dev, mesh_of

pytestmark = pytest.mark.gpu

CASES = [
    dict(n=(11, 7, 5), jitter=0.2, permute=True, seed=61, lognormal_gamma=True, dirichlet=("xmax", "zmin")),
    dict(n=6, seed=62, dirichlet=("xmax",)),
    dict(n=(9, 8, 1), jitter=0.2, permute=True, seed=63, lognormal_gamma=True, dirichlet=()),
]
IDS = ["ragged-jittered-2patches", "6c-uniform", "9x8x1-no-dirichlet"]


def _inputs(c, seed):
    m = c.mesh
    rng = np.random.default_rng(seed)
    phi = rng.standard_normal(m.n_faces) * np.linalg.norm(m.sf, axis=1)
    bphi = rng.standard_normal(m.n_bfaces) * np.linalg.norm(m.bface_sf, axis=1)
    return phi, bphi, rng.standard_normal(m.n_cells)


@pytest.fixture(scope="module", params=range(len(CASES)), ids=IDS)
def pc(request):
    c = hexmesh.pressure_case(**CASES[request.param])
    return c, mesh_of(c, centres=True)


def _geom(m):
    return dict(sf=dev(m.sf), cf=dev(m.cf), c=dev(m.c), v=dev(m.v), bcell=dev(m.bface_cell), bsf=dev(m.bface_sf),
                bcf=dev(m.bface_cf))


def test_operators_bitwise(pc):
    c, M = pc
    m = c.mesh
    G = _geom(m)
    bt = dev(c.btype)
    phi, bphi, p_old = _inputs(c, 64)
    w = M.fv_weights(G["sf"], G["cf"], G["c"])
    wo = oracle.fv_weights(m)
    assert np.array_equal(bits(w.cpu().numpy()), bits(wo))
    g = M.fv_grad(G["sf"], w, G["v"], dev(p_old), G["bcell"], G["bsf"], bt)
    go = oracle.fv_grad(m, wo, c.btype, p_old)
    assert np.array_equal(bits(g.cpu().numpy()), bits(go))
    corr, b = M.pressure_rhs(G["sf"], G["c"], w, dev(c.gamma), g, dev(phi), G["bcell"], dev(bphi))
    corro, bo = oracle.pressure_rhs(m, wo, c.gamma, go, phi, bphi)
    assert np.array_equal(bits(corr.cpu().numpy()), bits(corro))
    assert np.array_equal(bits(b.cpu().numpy()), bits(bo))
    up, dg = oracle.assemble_laplacian(m, c.gamma, c.bgamma, c.btype)
    p = np.random.default_rng(65).standard_normal(m.n_cells)
    phin, bphin = M.pressure_flux(dev(up), corr, dev(p), dev(phi), G["c"], G["bcell"], G["bsf"], G["bcf"],
                                  dev(c.bgamma), bt, dev(bphi))
    phio, bphio = oracle.pressure_flux(m, up, corro, p, phi, c.bgamma, c.btype, bphi)
    assert np.array_equal(bits(phin.cpu().numpy()), bits(phio))
    assert np.array_equal(bits(bphin.cpu().numpy()), bits(bphio))
    d = M.fv_div(dev(phi), G["bcell"], dev(bphi))
    assert np.array_equal(bits(d.cpu().numpy()), bits(oracle.fv_div(m, phi, bphi)))


def test_pressure_step_divergence_free(pc):
    from paper_2512_22215_gb300 import SolverControls
    c, M = pc
    m = c.mesh
    if not np.any(c.btype == 1):
        pytest.skip("all-Neumann: A is singular without a reference level")
    G = _geom(m)
    phi, bphi, p_old = _inputs(c, 66)
    geom = (G["sf"], G["cf"], G["c"], G["v"], G["bcell"], G["bsf"], G["bcf"])
    p, phin, bphin, perf = M.pressure_step(geom, dev(c.gamma), dev(c.bgamma), dev(c.btype), dev(phi), dev(bphi),
                                           dev(p_old), SolverControls(precond=2, tolerance=1e-13))
    assert perf["converged"] == 1
    div0 = oracle.fv_div(m, phi, bphi)
    div1 = M.fv_div(phin, G["bcell"], bphin).cpu().numpy()
    assert np.abs(div1).max() <= 1e-9 * np.abs(div0).max()
