"""GPU: reverse mode of the Laplacian assembly with respect to the face
diffusivities (spuma_assemble_laplacian_adjoint) against the oracle, bit for
bit (same operation order), and the gradient of a loss on x with respect to
gamma through assembly + solve (LaplacianAssembly + PressureSolve) against
central differences."""
import numpy as np
import pytest
import torch

import oracle
from gpu_cases import bits, case, dev, mesh_of

pytestmark = pytest.mark.gpu


def _geometry(m):
    return (dev(m.sf), dev(m.c), dev(m.bface_cell), dev(m.bface_sf), dev(m.bface_cf))


@pytest.mark.parametrize("kw", [dict(n=(13, 6, 5), jitter=0.2, permute=True, seed=41, lognormal=True),
                                dict(n=4, seed=42, dirichlet=("xmax", "ymin"))], ids=["ragged-permuted", "4c-uniform"])
def test_assembly_adjoint_bitwise(kw):
    c = case(**kw)
    m = c.mesh
    M = mesh_of(c)
    rng = np.random.default_rng(43)
    gu, gd = rng.standard_normal(m.n_faces), rng.standard_normal(m.n_cells)
    sf, cc, bcell, bsf, bcf = _geometry(m)
    gg, gb = M.assemble_laplacian_adjoint(sf, cc, dev(gu), dev(gd), bcell, bsf, bcf, dev(c.btype))
    ggo, gbo = oracle.assembly_adjoint(m, gu, gd, c.btype)
    assert np.array_equal(bits(gg.cpu().numpy()), bits(ggo))
    assert np.array_equal(bits(gb.cpu().numpy()), bits(gbo))


def test_gamma_gradient_through_solve_finite_differences():
    """L(gamma) = 0.5 |x - x_t|^2, x = A(gamma, bgamma)^-1 b: 16 random
    directions, central differences with step 1e-6 relative, FP64 solves to
    1e-14; agreement to 1e-6 relative."""
    from paper_2512_22215_gb300 import SolverControls, assemble_laplacian, pressure_solve
    c = case(12, jitter=0.2, permute=True, seed=44, lognormal=True, target=True)
    m = c.mesh
    M = mesh_of(c)
    sf, cc, bcell, bsf, bcf = _geometry(m)
    bt, xt, b = dev(c.btype), dev(c.x_t), dev(c.b)
    ctl = SolverControls(precond=2, tolerance=1e-14, max_iter=3000)

    def loss(gamma, bgamma):
        up, dg = assemble_laplacian(M, gamma, bgamma, sf, cc, bcell, bsf, bcf, bt)
        x = pressure_solve(M, up, dg, b, ctl)
        return 0.5 * ((x - xt) ** 2).sum()

    g = dev(c.gamma).requires_grad_(True)
    gbd = dev(c.bgamma).requires_grad_(True)
    loss(g, gbd).backward()
    rng = np.random.default_rng(45)
    h = 1e-6
    with torch.no_grad():
        for _ in range(16):
            vg = dev(rng.standard_normal(m.n_faces) * c.gamma)
            vb = dev(rng.standard_normal(m.n_bfaces) * c.bgamma)
            fd = (float(loss(g + h * vg, gbd + h * vb)) - float(loss(g - h * vg, gbd - h * vb))) / (2 * h)
            an = float((g.grad * vg).sum() + (gbd.grad * vb).sum())
            assert fd == pytest.approx(an, rel=1e-6)
    # zero-gradient boundary faces carry no gradient
    assert torch.all(gbd.grad[dev(c.btype) != 1] == 0)
