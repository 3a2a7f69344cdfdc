"""Shared helpers of the GPU parity tests: seeded cases on the device, the
oracle's answers on the host."""
from functools import lru_cache

import numpy as np
import torch

import hexmesh
import oracle


@lru_cache(maxsize=16)
def case(n, jitter=0.0, permute=False, seed=0, lognormal=False, dirichlet=("xmax",), target=False):
    return hexmesh.pressure_case(n, jitter=jitter, permute=permute, seed=seed, lognormal_gamma=lognormal,
                                 dirichlet=dirichlet, with_target=target)


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def mesh_of(c, centres=False):
    from paper_2512_22215_gb300 import LduMesh
    m = c.mesh
    return LduMesh(m.lower, m.upper_addr, m.n_cells, centres=m.c if centres else None)


def assemble_gpu(M, c):
    m = c.mesh
    return M.assemble_laplacian(dev(m.sf), dev(m.c), dev(c.gamma), dev(m.bface_cell), dev(m.bface_sf),
                                dev(m.bface_cf), dev(c.bgamma), dev(c.btype))


def assemble_oracle(c):
    return oracle.assemble_laplacian(c.mesh, c.gamma, c.bgamma, c.btype)


def levels_bruteforce(m):
    """DIC level of each cell by one sequential pass in face order."""
    lv = np.zeros(m.n_cells, dtype=np.int64)
    for f in range(m.n_faces):
        l, u = m.lower[f], m.upper_addr[f]
        if lv[l] + 1 > lv[u]:
            lv[u] = lv[l] + 1
    return lv


def bits(a):
    a = np.ascontiguousarray(a)
    return a.view(np.uint64) if a.dtype == np.float64 else a.view(np.uint32)
