"""Seeded asymmetric LDU systems for the PBiCG tests: the laplacian of a
pressure case plus first-order upwind convection of a random face flux, with
the diagonal raised to the row's absolute sum divided by an under-relaxation
factor 0.7 (the paper's U relaxation factor), as in a momentum equation:
  lower_f = -a_f - max(phi_f, 0),  upper_f = -a_f - max(-phi_f, 0),
  diag_i = (sum of |off-diagonal| of row i + Dirichlet boundary a_b) / 0.7.
phi_f = Pe * xi_f * mean(a) with xi ~ N(0, 1): Pe sets how asymmetric A is."""
import numpy as np

import hexmesh
import oracle


def asym_case(n, seed, pe=2.0, **kw):
    c = hexmesh.pressure_case(n, seed=seed, **kw)
    m = c.mesh
    up, dg = oracle.assemble_laplacian(m, c.gamma, c.bgamma, c.btype)
    a = -up
    rng = np.random.default_rng(seed + 1000)
    phi = pe * rng.standard_normal(m.n_faces) * a.mean()
    lower = -a - np.maximum(phi, 0.0)
    upper = -a - np.maximum(-phi, 0.0)
    rowabs = np.zeros(m.n_cells)
    np.add.at(rowabs, m.upper_addr, np.abs(lower))
    np.add.at(rowabs, m.lower, np.abs(upper))
    lap_row = np.zeros(m.n_cells)
    np.add.at(lap_row, m.lower, a)
    np.add.at(lap_row, m.upper_addr, a)
    boundary = dg - lap_row                       # the Dirichlet coefficients the assembly added
    diag = (rowabs + boundary) / 0.7
    return c, lower, upper, diag


def dense_asym(l, u, diag, lower, upper):
    n = len(diag)
    A = np.zeros((n, n))
    A[np.arange(n), np.arange(n)] = diag
    A[u, l] = lower
    A[l, u] = upper
    return A
