"""Seeded synthetic hex-block meshes in OpenFOAM's face-addressed (LDU) layout.

This module generates inputs only.  It computes the mesh geometry (face area
vectors, face and cell centres) from jittered points, draws the per-face
diffusivity and the right-hand side, and orders the faces the OpenFOAM way.
It holds none of the pressure-solve arithmetic (coefficient assembly, Amul,
DIC, PCG): both the CPU oracle and the CUDA path take its arrays as inputs.

Recipe (the paper's DrivAer meshes are not available; these blocks stand in
for them, Sec. 4 of the paper uses 8-30M cells per GPU):

* an ``nx x ny x nz`` block of hexahedra on ``[0,1]^3`` (or on given
  graded coordinate lines), spacing ``h = 1/n`` per direction;
* interior points (no coordinate on the box boundary) are moved by
  ``U(-jitter, jitter) * h`` per coordinate;
* cells optionally randomly permuted;
* each internal face gets ``lower = min`` and ``upper = max`` of its two cell
  ids; its area vector is negated when owner and neighbour swap, so that it
  points from ``lower`` to ``upper``; internal faces are sorted by
  ``(lower, upper)`` (OpenFOAM's upper-triangular order);
* boundary faces follow, grouped by patch: x-min, x-max, y-min, y-max, z-min,
  z-max; within a patch in structured order; area vectors point outwards;
* random draws, all from ``numpy.random.default_rng(seed)``, in this order:
  jitter, permutation, face diffusivity (internal faces in sorted order, then
  boundary faces), ``b``, then ``x_t`` (adjoint target).

Geometry (OpenFOAM's primitiveMesh construction, restated): a face's estimated
centre is the mean of its 4 points; it is split into 4 triangles
``(p_k, p_{k+1}, c~)`` with area vectors ``a_t = 1/2 (p_{k+1}-p_k) x (c~-p_k)``;
``S_f = sum a_t`` and ``C_f = sum |a_t| c_t / sum |a_t|``.  A cell's estimated
centre is the mean of its 6 face centres; each face spans a pyramid of volume
``V = 1/3 S_out . (C_f - c~)`` and centroid ``3/4 C_f + 1/4 c~``; the cell centre
is the volume-weighted mean of the pyramid centroids.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

PATCHES = ("xmin", "xmax", "ymin", "ymax", "zmin", "zmax")
ZERO_GRADIENT = 0
DIRICHLET = 1


@dataclass
class Mesh:
    n_cells: int
    n_faces: int
    lower: np.ndarray          # int32 [F]   owner (lowerAddr), l < u
    upper_addr: np.ndarray     # int32 [F]   neighbour (upperAddr)
    sf: np.ndarray             # f64 [F,3]   area vector, points lower -> upper
    cf: np.ndarray             # f64 [F,3]   face centre
    c: np.ndarray              # f64 [N,3]   cell centre
    v: np.ndarray              # f64 [N]     cell volume
    bface_cell: np.ndarray     # int32 [B]
    bface_sf: np.ndarray       # f64 [B,3]   outward area vector
    bface_cf: np.ndarray       # f64 [B,3]
    bface_patch: np.ndarray    # int8 [B]    index into PATCHES
    shape: tuple = (0, 0, 0)
    cell_ijk: Optional[np.ndarray] = None   # int32 [N,3] structured index of each cell
    meta: dict = field(default_factory=dict)

    @property
    def n_bfaces(self) -> int:
        return int(self.bface_cell.shape[0])

    def bface_type(self, dirichlet: Sequence[str] = ("xmax",)) -> np.ndarray:
        t = np.zeros(self.n_bfaces, dtype=np.int8)
        for name in dirichlet:
            t[self.bface_patch == PATCHES.index(name)] = DIRICHLET
        return t


def _tri_geometry(p0, p1, p2, p3):
    """Area vector and centre of quads given as 4 corner arrays [...,3]
    (component-wise arithmetic; returns arrays [...,3])."""
    ctil = 0.25 * (((p0 + p1) + p2) + p3)
    corners = (p0, p1, p2, p3)
    s = np.zeros_like(p0)
    wsum = np.zeros(p0.shape[:-1])
    csum = np.zeros_like(p0)
    for k in range(4):
        a = corners[k]
        b = corners[(k + 1) % 4]
        e = b - a
        q = ctil - a
        at = np.empty_like(e)
        at[..., 0] = 0.5 * (e[..., 1] * q[..., 2] - e[..., 2] * q[..., 1])
        at[..., 1] = 0.5 * (e[..., 2] * q[..., 0] - e[..., 0] * q[..., 2])
        at[..., 2] = 0.5 * (e[..., 0] * q[..., 1] - e[..., 1] * q[..., 0])
        ct = (a + b + ctil) / 3.0
        mag = np.sqrt(at[..., 0] ** 2 + at[..., 1] ** 2 + at[..., 2] ** 2)
        s += at
        wsum += mag
        csum += mag[..., None] * ct
    cf = csum / wsum[..., None]
    return s, cf


def hex_block(n, jitter: float = 0.0, permute: bool = False, seed: int = 0,
              coords: Optional[Sequence[np.ndarray]] = None,
              rng: Optional[np.random.Generator] = None) -> tuple[Mesh, np.random.Generator]:
    """Build a hex block.  Returns the mesh and the generator, positioned after
    the jitter and permutation draws so that the caller draws gamma, b, x_t next."""
    if np.isscalar(n):
        nx = ny = nz = int(n)
    else:
        nx, ny, nz = (int(v) for v in n)
    if rng is None:
        rng = np.random.default_rng(seed)
    if coords is None:
        xs = np.linspace(0.0, 1.0, nx + 1)
        ys = np.linspace(0.0, 1.0, ny + 1)
        zs = np.linspace(0.0, 1.0, nz + 1)
    else:
        xs, ys, zs = (np.asarray(a, dtype=np.float64) for a in coords)
        assert len(xs) == nx + 1 and len(ys) == ny + 1 and len(zs) == nz + 1
    # points P[k, j, i, :]
    P = np.empty((nz + 1, ny + 1, nx + 1, 3))
    P[..., 0] = xs[None, None, :]
    P[..., 1] = ys[None, :, None]
    P[..., 2] = zs[:, None, None]
    if jitter > 0.0 and nx > 1 and ny > 1 and nz > 1:
        hx, hy, hz = 1.0 / nx, 1.0 / ny, 1.0 / nz
        inner = P[1:-1, 1:-1, 1:-1]
        d = rng.uniform(-jitter, jitter, size=inner.shape)
        d[..., 0] *= hx
        d[..., 1] *= hy
        d[..., 2] *= hz
        P[1:-1, 1:-1, 1:-1] = inner + d
    N = nx * ny * nz

    # faces normal to x: at i = 0..nx, (k < nz, j < ny); corners ordered for +x normal
    Sx, Cx = _tri_geometry(P[:-1, :-1, :], P[:-1, 1:, :], P[1:, 1:, :], P[1:, :-1, :])
    # normal to y: at j = 0..ny, (k < nz, i < nx); +y normal
    Sy, Cy = _tri_geometry(P[:-1, :, :-1], P[1:, :, :-1], P[1:, :, 1:], P[:-1, :, 1:])
    # normal to z: at k = 0..nz; +z normal
    Sz, Cz = _tri_geometry(P[:, :-1, :-1], P[:, :-1, 1:], P[:, 1:, 1:], P[:, 1:, :-1])
    del P

    # cell centres and volumes (natural order, index [k, j, i])
    faces_out = [(-Sx[:, :, :-1], Cx[:, :, :-1]), (Sx[:, :, 1:], Cx[:, :, 1:]),
                 (-Sy[:, :-1, :], Cy[:, :-1, :]), (Sy[:, 1:, :], Cy[:, 1:, :]),
                 (-Sz[:-1], Cz[:-1]), (Sz[1:], Cz[1:])]
    ctil = sum(cf for _, cf in faces_out) / 6.0
    vol = np.zeros((nz, ny, nx))
    vc = np.zeros((nz, ny, nx, 3))
    for sfo, cf in faces_out:
        dc = cf - ctil
        pv = (sfo[..., 0] * dc[..., 0] + sfo[..., 1] * dc[..., 1] + sfo[..., 2] * dc[..., 2]) / 3.0
        pc = 0.75 * cf + 0.25 * ctil
        vol += pv
        vc += pv[..., None] * pc
    cc = vc / vol[..., None]
    del faces_out, ctil, vc

    if permute:
        perm = rng.permutation(N).astype(np.int64)   # perm[old] = new id
    else:
        perm = np.arange(N, dtype=np.int64)
    newid = perm.reshape(nz, ny, nx)

    # global face numbering: Sx flattened, then Sy, then Sz
    nfx, nfy = Sx[..., 0].size, Sy[..., 0].size
    fid_x = np.arange(nfx, dtype=np.int64).reshape(nz, ny, nx + 1)
    fid_y = nfx + np.arange(nfy, dtype=np.int64).reshape(nz, ny + 1, nx)
    fid_z = nfx + nfy + np.arange(Sz[..., 0].size, dtype=np.int64).reshape(nz + 1, ny, nx)
    S_all = [np.concatenate([Sx[..., d].ravel(), Sy[..., d].ravel(), Sz[..., d].ravel()]) for d in range(3)]
    C_all = [np.concatenate([Cx[..., d].ravel(), Cy[..., d].ravel(), Cz[..., d].ravel()]) for d in range(3)]

    # per cell (natural index) its 6 neighbours and faces: x-, x+, y-, y+, z-, z+
    BIG = np.int64(np.iinfo(np.int64).max)
    nb = np.full((nz, ny, nx, 6), BIG, dtype=np.int64)
    fc = np.zeros((nz, ny, nx, 6), dtype=np.int64)
    sg = np.zeros((nz, ny, nx, 6), dtype=np.int8)
    nb[:, :, 1:, 0] = newid[:, :, :-1]
    nb[:, :, :-1, 1] = newid[:, :, 1:]
    nb[:, 1:, :, 2] = newid[:, :-1, :]
    nb[:, :-1, :, 3] = newid[:, 1:, :]
    nb[1:, :, :, 4] = newid[:-1]
    nb[:-1, :, :, 5] = newid[1:]
    fc[..., 0] = fid_x[:, :, :-1]
    fc[..., 1] = fid_x[:, :, 1:]
    fc[..., 2] = fid_y[:, :-1, :]
    fc[..., 3] = fid_y[:, 1:, :]
    fc[..., 4] = fid_z[:-1]
    fc[..., 5] = fid_z[1:]
    sg[..., 0::2] = -1      # face on the cell's minus side: stored S points towards the cell
    sg[..., 1::2] = 1
    nb = nb.reshape(N, 6)
    fc = fc.reshape(N, 6)
    sg = sg.reshape(N, 6)
    # rows in new-id order; keep only neighbours with a larger id (this cell is "lower")
    rows = np.empty_like(nb)
    rows[perm] = nb
    fcr = np.empty_like(fc)
    fcr[perm] = fc
    sgr = np.empty_like(sg)
    sgr[perm] = sg
    del nb, fc, sg
    own = np.arange(N, dtype=np.int64)[:, None]
    rows[rows <= own] = BIG
    order = np.argsort(rows, axis=1, kind="stable")
    rows = np.take_along_axis(rows, order, axis=1)
    fcr = np.take_along_axis(fcr, order, axis=1)
    sgr = np.take_along_axis(sgr, order, axis=1)
    valid = rows != BIG
    up = rows[valid].astype(np.int32)
    lo = np.broadcast_to(own, rows.shape)[valid].astype(np.int32)
    fsel = fcr[valid]
    sgn = sgr[valid].astype(np.float64)
    del rows, fcr, sgr, valid, order
    sf = np.empty((lo.shape[0], 3))
    cf = np.empty((lo.shape[0], 3))
    for d in range(3):
        sf[:, d] = S_all[d][fsel] * sgn
        cf[:, d] = C_all[d][fsel]
    del S_all, C_all, fsel, sgn

    # boundary faces, patch order xmin, xmax, ymin, ymax, zmin, zmax
    bcell, bsf, bcf, bpatch = [], [], [], []
    blocks = [
        (newid[:, :, 0], -Sx[:, :, 0], Cx[:, :, 0]),
        (newid[:, :, -1], Sx[:, :, -1], Cx[:, :, -1]),
        (newid[:, 0, :], -Sy[:, 0, :], Cy[:, 0, :]),
        (newid[:, -1, :], Sy[:, -1, :], Cy[:, -1, :]),
        (newid[0], -Sz[0], Cz[0]),
        (newid[-1], Sz[-1], Cz[-1]),
    ]
    for pi, (cid, s, c) in enumerate(blocks):
        bcell.append(cid.ravel())
        bsf.append(s.reshape(-1, 3))
        bcf.append(c.reshape(-1, 3))
        bpatch.append(np.full(cid.size, pi, dtype=np.int8))

    cnew = np.empty((N, 3))
    cnew[perm] = cc.reshape(-1, 3)
    vnew = np.empty(N)
    vnew[perm] = vol.ravel()
    ijk = np.empty((N, 3), dtype=np.int32)
    kk, jj, ii = np.meshgrid(np.arange(nz, dtype=np.int32), np.arange(ny, dtype=np.int32),
                             np.arange(nx, dtype=np.int32), indexing="ij")
    ijk[perm, 0] = ii.ravel()
    ijk[perm, 1] = jj.ravel()
    ijk[perm, 2] = kk.ravel()

    mesh = Mesh(
        n_cells=N, n_faces=int(lo.shape[0]), lower=lo, upper_addr=up, sf=sf, cf=cf,
        c=cnew, v=vnew,
        bface_cell=np.concatenate(bcell).astype(np.int32),
        bface_sf=np.ascontiguousarray(np.concatenate(bsf)),
        bface_cf=np.ascontiguousarray(np.concatenate(bcf)),
        bface_patch=np.concatenate(bpatch),
        shape=(nx, ny, nz), cell_ijk=ijk,
        meta=dict(jitter=jitter, permute=permute, seed=seed),
    )
    return mesh, rng


@dataclass
class PressureCase:
    """A mesh plus the per-solve inputs of the pressure equation."""
    mesh: Mesh
    gamma: np.ndarray        # f64 [F]  face diffusivity
    bgamma: np.ndarray       # f64 [B]
    btype: np.ndarray        # int8 [B] 0 zero-gradient, 1 Dirichlet (value 0)
    b: np.ndarray            # f64 [N]  source
    x_t: Optional[np.ndarray] = None   # f64 [N]  adjoint target


def pressure_case(n, jitter=0.0, permute=False, seed=0, lognormal_gamma=False,
                  dirichlet=("xmax",), with_target=False, coords=None) -> PressureCase:
    """The recipe of the synthetic pressure systems: mesh, then gamma (log-normal
    sigma=1 or unit), then b ~ N(0,1), then optionally x_t ~ N(0,1)."""
    mesh, rng = hex_block(n, jitter=jitter, permute=permute, seed=seed, coords=coords)
    if lognormal_gamma:
        gamma = np.exp(rng.standard_normal(mesh.n_faces))
        bgamma = np.exp(rng.standard_normal(mesh.n_bfaces))
    else:
        gamma = np.ones(mesh.n_faces)
        bgamma = np.ones(mesh.n_bfaces)
    b = rng.standard_normal(mesh.n_cells)
    x_t = rng.standard_normal(mesh.n_cells) if with_target else None
    return PressureCase(mesh=mesh, gamma=gamma, bgamma=bgamma,
                        btype=mesh.bface_type(dirichlet), b=b, x_t=x_t)


def batch_sizes(n_sys: int, seed: int, lo: float = 1e4, hi: float = 5e5) -> list[int]:
    """Side lengths of a batch: cell counts log-uniform in [lo, hi], side = round(N^(1/3))."""
    rng = np.random.default_rng(seed)
    ncell = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_sys))
    return [max(2, int(round(v ** (1.0 / 3.0)))) for v in ncell]
