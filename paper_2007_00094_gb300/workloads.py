"""Seeded synthetic inputs: Q1 hexahedral meshes and initial states.

This module is shared by the CUDA path and by the FP64 oracle, so it holds
none of the method's arithmetic: it only lays out node positions, the
hexahedra that connect them, per-node boundary flags and initial conserved
states.  Finite-element matrices (Sec. 3.1, eq. "matrices"), wavespeeds,
limiters etc. are computed independently on each side.

Conventions (the input format of ``idp_upload_mesh_hex`` in include/idp.h):

* ``cells[c, v]`` lists the 8 node ids of hexahedron ``c`` with local vertex
  ``v = a + 2 b + 4 c`` for reference coordinates ``(a, b, c) in {0,1}^3``.
* ``cell_xyz[c, v, :]`` is the physical position of that vertex as seen from
  the cell.  On periodic axes it is the unwrapped position, so a cell that
  straddles the periodic seam keeps a positive Jacobian even though its node
  ids wrap around.
* ``bc[i]`` is a bit mask: ``BC_SLIP_X|BC_SLIP_Y|BC_SLIP_Z`` name the
  axis-aligned wall normals of the faces node ``i`` lies on (slip walls remove
  those momentum components), ``BC_INFLOW`` fixes the node to the inflow
  state.  Outflow and periodic nodes carry no flag.
* A 2D mesh (Q1 quadrilaterals, 9-point stencil; ``idp_upload_mesh_quad``)
  uses the same container with 4 vertices per cell, ``v = a + 2 b``; node and
  vertex positions keep a zero z coordinate.
* States are conserved variables ``U = (rho, m_x, m_y, m_z, E)`` stored
  struct-of-arrays as a ``(5, N)`` float64 array (Sec. 2).

The workloads follow the paper's setting (3D Q1, 27-point stencil, gamma=7/5,
Sec. 5): a periodic isentropic vortex, a Sod shock tube, a Mach 3
forward-facing step on a jittered (unstructured-like) mesh, batches of random
Riemann problems, and a vortex with seeded Gaussian density bumps.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

GAMMA = 1.4

BC_SLIP_X = 1
BC_SLIP_Y = 2
BC_SLIP_Z = 4
BC_INFLOW = 8


@dataclass
class HexMesh:
    """A Q1 hexahedral mesh in the input format described in the module docstring."""

    x: np.ndarray  # (N, 3) node positions
    cells: np.ndarray  # (C, 8) int64 node ids
    cell_xyz: np.ndarray  # (C, 8, 3) vertex positions seen from the cell
    bc: np.ndarray  # (N,) int32 flags
    volume: float
    name: str = "mesh"
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    periodic: tuple = (False, False, False)
    inflow: np.ndarray | None = None  # (5,) conserved inflow state for BC_INFLOW nodes
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_cells(self) -> int:
        return int(self.cells.shape[0])

    @property
    def dim(self) -> int:
        return 2 if self.cells.shape[1] == 4 else 3


def _axis_nodes(n, lo, hi, periodic):
    """Node coordinates and spacing along one axis."""
    if periodic:
        h = (hi - lo) / n
        return lo + h * np.arange(n), h, n  # n cells
    h = (hi - lo) / (n - 1)
    return lo + h * np.arange(n), h, n - 1


def box_mesh(shape, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), periodic=(True, True, True),
             jitter=0.0, seed=0, walls="slip", name=None) -> HexMesh:
    """Tensor-product box mesh with ``shape = (nx, ny, nz)`` unique nodes per axis.

    On a periodic axis the ``n`` nodes are spaced ``h = L/n`` and the last cell
    wraps to node 0; on a non-periodic axis ``h = L/(n-1)`` and the faces are
    walls (``walls="slip"`` flags them, ``walls=None`` leaves them unflagged,
    which makes them outflow-like).  Nodes that lie on no wall are displaced by
    ``U[-jitter*h, jitter*h]`` per coordinate (seeded).
    """
    nx, ny, nz = (int(s) for s in shape)
    lo = tuple(float(v) for v in lo)
    hi = tuple(float(v) for v in hi)
    coords, hs, ncell = [], [], []
    for n, a, b, p in zip((nx, ny, nz), lo, hi, periodic):
        c, h, nc = _axis_nodes(n, a, b, p)
        coords.append(c)
        hs.append(h)
        ncell.append(nc)
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ii, jj, kk = (a.transpose(2, 1, 0).ravel() for a in (ii, jj, kk))  # x fastest
    x = np.stack([coords[0][ii], coords[1][jj], coords[2][kk]], axis=1)
    N = x.shape[0]

    bc = np.zeros(N, dtype=np.int32)
    on_wall = np.zeros(N, dtype=bool)
    for axis, (idx, n, p) in enumerate(zip((ii, jj, kk), (nx, ny, nz), periodic)):
        if p:
            continue
        w = (idx == 0) | (idx == n - 1)
        on_wall |= w
        if walls == "slip":
            bc[w] |= (BC_SLIP_X, BC_SLIP_Y, BC_SLIP_Z)[axis]

    rng = np.random.default_rng(seed)
    disp = np.zeros_like(x)
    if jitter > 0.0:
        disp = rng.uniform(-1.0, 1.0, size=x.shape) * (jitter * np.asarray(hs))[None, :]
        disp[on_wall] = 0.0
    x = x + disp

    ci, cj, ck = np.meshgrid(np.arange(ncell[0]), np.arange(ncell[1]), np.arange(ncell[2]), indexing="ij")
    ci, cj, ck = (a.transpose(2, 1, 0).ravel() for a in (ci, cj, ck))
    C = ci.shape[0]
    cells = np.empty((C, 8), dtype=np.int64)
    cell_xyz = np.empty((C, 8, 3), dtype=np.float64)
    L = np.asarray(hi) - np.asarray(lo)
    for v in range(8):
        a, b, c = v & 1, (v >> 1) & 1, (v >> 2) & 1
        gi, gj, gk = ci + a, cj + b, ck + c
        wrap = [np.zeros(C, dtype=bool)] * 3
        if periodic[0]:
            wrap[0] = gi == nx
            gi = gi % nx
        if periodic[1]:
            wrap[1] = gj == ny
            gj = gj % ny
        if periodic[2]:
            wrap[2] = gk == nz
            gk = gk % nz
        node = gi + nx * (gj + ny * gk)
        cells[:, v] = node
        pos = x[node].copy()
        for axis in range(3):
            pos[wrap[axis], axis] += L[axis]
        cell_xyz[:, v, :] = pos
    vol = float(np.prod(L))
    return HexMesh(x=x, cells=cells, cell_xyz=cell_xyz, bc=bc, volume=vol,
                   name=name or f"box{nx}x{ny}x{nz}", lo=lo, hi=hi, periodic=tuple(periodic),
                   meta={"shape": (nx, ny, nz), "h": tuple(hs), "jitter": jitter, "seed": seed})


def forward_step_mesh(m=120, jitter=0.2, seed=2007) -> HexMesh:
    """Mach 3 forward-facing step channel [0,3]x[0,1]x[0,0.5], step x>=0.6, y<=0.2.

    Uniform spacing ``h = 1/m`` (``m`` a multiple of 10 so that 0.2, 0.5 and 0.6
    fall on grid lines); nodes strictly inside the step are removed.  Interior
    nodes are jittered by ``U[-jitter*h, jitter*h]`` per coordinate (seeded).
    Flags: x=0 inflow; x=3 outflow (none); y=0, y=1, the step top y=0.2 and the
    step face x=0.6 slip; z=0 and z=0.5 slip.  ``m=120`` gives 2,242,909 nodes.
    """
    if m % 10:
        raise ValueError("m must be a multiple of 10")
    h = 1.0 / m
    nx, ny, nz = 3 * m + 1, m + 1, m // 2 + 1
    sx, sy = (6 * m) // 10, (2 * m) // 10  # step corner indices
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ii, jj, kk = (a.transpose(2, 1, 0).ravel() for a in (ii, jj, kk))
    keep = ~((ii > sx) & (jj < sy))
    gid = -np.ones(ii.shape[0], dtype=np.int64)
    gid[keep] = np.arange(int(keep.sum()))
    ii, jj, kk = ii[keep], jj[keep], kk[keep]
    x = np.stack([ii * h, jj * h, kk * h], axis=1).astype(np.float64)
    N = x.shape[0]

    bc = np.zeros(N, dtype=np.int32)
    wall_y = (jj == 0) | (jj == ny - 1) | ((jj == sy) & (ii >= sx))
    wall_x = (ii == sx) & (jj <= sy)
    wall_z = (kk == 0) | (kk == nz - 1)
    bc[wall_x] |= BC_SLIP_X
    bc[wall_y] |= BC_SLIP_Y
    bc[wall_z] |= BC_SLIP_Z
    inflow = ii == 0
    bc[inflow] = BC_INFLOW
    boundary = wall_x | wall_y | wall_z | inflow | (ii == nx - 1)

    rng = np.random.default_rng(seed)
    if jitter > 0.0:
        disp = rng.uniform(-jitter * h, jitter * h, size=x.shape)
        disp[boundary] = 0.0
        x = x + disp

    ci, cj, ck = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1), np.arange(nz - 1), indexing="ij")
    ci, cj, ck = (a.transpose(2, 1, 0).ravel() for a in (ci, cj, ck))
    ckeep = ~((ci >= sx) & (cj < sy))
    ci, cj, ck = ci[ckeep], cj[ckeep], ck[ckeep]
    C = ci.shape[0]
    cells = np.empty((C, 8), dtype=np.int64)
    for v in range(8):
        a, b, c = v & 1, (v >> 1) & 1, (v >> 2) & 1
        g = (ci + a) + nx * ((cj + b) + ny * (ck + c))
        cells[:, v] = gid[g]
    assert (cells >= 0).all()
    cell_xyz = x[cells]
    vol = 3.0 * 1.0 * 0.5 - (3.0 - 0.6) * 0.2 * 0.5
    U_in = primitive_to_conserved(np.array([1.4]), np.array([[3.0], [0.0], [0.0]]), np.array([1.0]))[:, 0]
    return HexMesh(x=x, cells=cells, cell_xyz=cell_xyz, bc=bc, volume=vol, name=f"ffs_m{m}",
                   lo=(0.0, 0.0, 0.0), hi=(3.0, 1.0, 0.5), periodic=(False, False, False),
                   inflow=U_in, meta={"m": m, "h": h, "jitter": jitter, "seed": seed})


def rect_mesh(shape, lo=(0.0, 0.0), hi=(1.0, 1.0), periodic=(True, True), jitter=0.0, seed=0,
              walls="slip", name=None) -> HexMesh:
    """2D tensor-product mesh of Q1 quadrilaterals with ``shape = (nx, ny)`` unique
    nodes per axis; periodic axes, wall flags and jitter as in ``box_mesh``."""
    nx, ny = (int(v) for v in shape)
    lo = tuple(float(v) for v in lo)
    hi = tuple(float(v) for v in hi)
    coords, hs, ncell = [], [], []
    for n, a, b, p in zip((nx, ny), lo, hi, periodic):
        c, h, nc = _axis_nodes(n, a, b, p)
        coords.append(c)
        hs.append(h)
        ncell.append(nc)
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    ii, jj = ii.ravel(), jj.ravel()  # x fastest
    N = ii.shape[0]
    x = np.zeros((N, 3))
    x[:, 0] = coords[0][ii]
    x[:, 1] = coords[1][jj]

    bc = np.zeros(N, dtype=np.int32)
    on_wall = np.zeros(N, dtype=bool)
    for axis, (idx, n, p) in enumerate(zip((ii, jj), (nx, ny), periodic)):
        if p:
            continue
        w = (idx == 0) | (idx == n - 1)
        on_wall |= w
        if walls == "slip":
            bc[w] |= (BC_SLIP_X, BC_SLIP_Y)[axis]

    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        disp = rng.uniform(-1.0, 1.0, size=(N, 2)) * (jitter * np.asarray(hs))[None, :]
        disp[on_wall] = 0.0
        x[:, :2] += disp

    cj, ci = np.meshgrid(np.arange(ncell[1]), np.arange(ncell[0]), indexing="ij")
    ci, cj = ci.ravel(), cj.ravel()
    C = ci.shape[0]
    cells = np.empty((C, 4), dtype=np.int64)
    cell_xyz = np.zeros((C, 4, 3))
    L = np.asarray(hi) - np.asarray(lo)
    for v in range(4):
        gi, gj = ci + (v & 1), cj + ((v >> 1) & 1)
        wrap = [np.zeros(C, dtype=bool)] * 2
        if periodic[0]:
            wrap[0] = gi == nx
            gi = gi % nx
        if periodic[1]:
            wrap[1] = gj == ny
            gj = gj % ny
        node = gi + nx * gj
        cells[:, v] = node
        pos = x[node].copy()
        for axis in range(2):
            pos[wrap[axis], axis] += L[axis]
        cell_xyz[:, v, :] = pos
    return HexMesh(x=x, cells=cells, cell_xyz=cell_xyz, bc=bc, volume=float(np.prod(L)),
                   name=name or f"rect{nx}x{ny}", lo=lo + (0.0,), hi=hi + (0.0,), periodic=tuple(periodic) + (False,),
                   meta={"shape": (nx, ny), "h": tuple(hs), "jitter": jitter, "seed": seed})


def forward_step_mesh_2d(m=1000, jitter=0.2, seed=2007) -> HexMesh:
    """2D Mach 3 forward-facing step (Woodward-Colella) [0,3]x[0,1], step x>=0.6, y<=0.2.

    Q1 quadrilaterals of spacing ``h = 1/m`` (``m`` a multiple of 5); nodes
    strictly inside the step removed, interior nodes jittered by
    ``U[-jitter*h, jitter*h]`` per coordinate (seeded).  Flags: x=0 inflow,
    x=3 outflow, y=0, y=1, the step top and the step face slip.  ``m=1000``
    gives 2,524,001 nodes.
    """
    if m % 5:
        raise ValueError("m must be a multiple of 5")
    h = 1.0 / m
    nx, ny = 3 * m + 1, m + 1
    sx, sy = (3 * m) // 5, m // 5
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    ii, jj = ii.ravel(), jj.ravel()
    keep = ~((ii > sx) & (jj < sy))
    gid = -np.ones(ii.shape[0], dtype=np.int64)
    gid[keep] = np.arange(int(keep.sum()))
    ii, jj = ii[keep], jj[keep]
    N = ii.shape[0]
    x = np.zeros((N, 3))
    x[:, 0] = ii * h
    x[:, 1] = jj * h

    bc = np.zeros(N, dtype=np.int32)
    wall_y = (jj == 0) | (jj == ny - 1) | ((jj == sy) & (ii >= sx))
    wall_x = (ii == sx) & (jj <= sy)
    bc[wall_x] |= BC_SLIP_X
    bc[wall_y] |= BC_SLIP_Y
    inflow = ii == 0
    bc[inflow] = BC_INFLOW
    boundary = wall_x | wall_y | inflow | (ii == nx - 1)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        disp = rng.uniform(-jitter * h, jitter * h, size=(N, 2))
        disp[boundary] = 0.0
        x[:, :2] += disp

    cj, ci = np.meshgrid(np.arange(ny - 1), np.arange(nx - 1), indexing="ij")
    ci, cj = ci.ravel(), cj.ravel()
    ckeep = ~((ci >= sx) & (cj < sy))
    ci, cj = ci[ckeep], cj[ckeep]
    cells = np.empty((ci.shape[0], 4), dtype=np.int64)
    for v in range(4):
        cells[:, v] = gid[(ci + (v & 1)) + nx * (cj + ((v >> 1) & 1))]
    assert (cells >= 0).all()
    U_in = primitive_to_conserved(np.array([1.4]), np.array([[3.0], [0.0], [0.0]]), np.array([1.0]))[:, 0]
    return HexMesh(x=x, cells=cells, cell_xyz=x[cells], bc=bc, volume=3.0 - 2.4 * 0.2, name=f"ffs2d_m{m}",
                   lo=(0.0, 0.0, 0.0), hi=(3.0, 1.0, 0.0), periodic=(False, False, False),
                   inflow=U_in, meta={"m": m, "h": h, "jitter": jitter, "seed": seed})


def vortex_mesh_2d(n, jitter=0.0, seed=0):
    """Periodic unit square with ``n`` nodes along x and y (Q1 quadrilaterals)."""
    return rect_mesh((n, n), periodic=(True, True), jitter=jitter, seed=seed, name=f"vortex2d_{n}")


def sod_mesh_2d(nx, ny=4):
    """2D shock tube [0,1]x[0,1], slip walls along x, periodic in y."""
    return rect_mesh((nx, ny), periodic=(False, True), walls="slip", name=f"sod2d_{nx}")


# ---------------------------------------------------------------------------
# Initial states (conserved variables, gamma = 7/5 polytropic gas, Sec. 2)
# ---------------------------------------------------------------------------

def primitive_to_conserved(rho, u, p, gamma=GAMMA):
    """(rho, u[3,N], p) -> U[5,N] with E = p/(gamma-1) + rho |u|^2 / 2."""
    rho = np.asarray(rho, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    U = np.empty((5,) + rho.shape, dtype=np.float64)
    U[0] = rho
    U[1:4] = rho[None] * u
    U[4] = p / (gamma - 1.0) + 0.5 * rho * (u * u).sum(axis=0)
    return U


def uniform_state(mesh: HexMesh, rho=1.0, u=(0.0, 0.0, 0.0), p=1.0):
    N = mesh.n_nodes
    return primitive_to_conserved(np.full(N, rho), np.tile(np.asarray(u, float)[:, None], (1, N)), np.full(N, p))


def vortex_primitive(x, t=0.0, beta=5.0, u_inf=(1.0, 1.0, 0.0), center=(0.5, 0.5), scale=10.0,
                     period=(1.0, 1.0), gamma=GAMMA):
    """Isentropic vortex extruded in z, translated by ``u_inf * t`` on a periodic unit square.

    Coordinates are mapped by ``x' = scale * (x - x_c)`` (minimum image on the
    periodic square); ``du = beta/(2 pi) exp((1-r'^2)/2) (-y', x')``,
    ``T = 1 - (gamma-1) beta^2/(8 gamma pi^2) exp(1-r'^2)``, ``rho = T^(1/(gamma-1))``,
    ``p = rho T``.  This is an exact solution of the Euler equations for any
    ``scale`` (radial balance dp/dr = rho u_theta^2 / r holds in r').
    """
    x = np.asarray(x, dtype=np.float64)
    dx = x[:, 0] - center[0] - u_inf[0] * t
    dy = x[:, 1] - center[1] - u_inf[1] * t
    dx = dx - period[0] * np.round(dx / period[0])
    dy = dy - period[1] * np.round(dy / period[1])
    xs, ys = scale * dx, scale * dy
    r2 = xs * xs + ys * ys
    f = beta / (2.0 * np.pi) * np.exp(0.5 * (1.0 - r2))
    T = 1.0 - (gamma - 1.0) * beta * beta / (8.0 * gamma * np.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho * T
    u = np.stack([u_inf[0] - f * ys, u_inf[1] + f * xs, np.full_like(xs, u_inf[2])])
    return rho, u, p


def vortex_state(mesh: HexMesh, t=0.0, beta=5.0):
    rho, u, p = vortex_primitive(mesh.x, t=t, beta=beta)
    return primitive_to_conserved(rho, u, p)


def riemann_state(x, left, right, normal=(1.0, 0.0, 0.0), point=(0.5, 0.5, 0.5)):
    """Piecewise-constant Riemann data across the plane through ``point`` with ``normal``.

    ``left``/``right`` are ``(rho, (ux, uy, uz), p)``; left is the side with
    ``(x - point) . normal < 0``.
    """
    x = np.asarray(x, dtype=np.float64)
    nrm = np.asarray(normal, dtype=np.float64)
    s = (x - np.asarray(point)[None, :]) @ nrm
    is_left = s < 0.0
    N = x.shape[0]
    rho = np.where(is_left, left[0], right[0])
    u = np.where(is_left[None, :], np.asarray(left[1], float)[:, None], np.asarray(right[1], float)[:, None])
    p = np.where(is_left, left[2], right[2])
    return primitive_to_conserved(rho.astype(np.float64), u.reshape(3, N), p.astype(np.float64))


def sod_state(mesh: HexMesh, x0=0.5):
    return riemann_state(mesh.x, (1.0, (0.0, 0.0, 0.0), 1.0), (0.125, (0.0, 0.0, 0.0), 0.1),
                         normal=(1.0, 0.0, 0.0), point=(x0, 0.0, 0.0))


def forward_step_state(mesh: HexMesh):
    """Uniform Mach 3 inflow state rho=1.4, p=1, u=(3,0,0) everywhere."""
    return uniform_state(mesh, rho=1.4, u=(3.0, 0.0, 0.0), p=1.0)


def bumpy_vortex_state(mesh: HexMesh, n_bumps=8, amplitude=1e-2, width=0.1, seed=5):
    """Vortex plus seeded Gaussian density bumps (velocity and pressure kept)."""
    rho, u, p = vortex_primitive(mesh.x)
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, 1.0, size=(n_bumps, 3))
    for c in centres:
        d = mesh.x - c[None, :]
        d = d - np.round(d)
        rho = rho + amplitude * np.exp(-(d * d).sum(axis=1) / (2.0 * width * width))
    return primitive_to_conserved(rho, u, p)


def perturbation_directions(U, count, seed=16):
    """Seeded directions v_k = xi_k |U| (xi_k standard normal, element-wise)
    in the space of states, for directional-derivative checks."""
    rng = np.random.default_rng(seed)
    return [rng.standard_normal(U.shape) * np.abs(U) for _ in range(count)]


def random_riemann_batch(n_instances=256, side_range=(8, 48), seed=4):
    """Independent 3D Riemann problems on slip-walled unit cubes of random size.

    Side lengths ~ U{side_range}; left/right states rho ~ U[0.1,2], p ~ U[0.1,10],
    each velocity component ~ U[-2,2]; the interface passes through the cube
    centre with a uniformly random unit normal.  Returns ``[(mesh, U0), ...]``.
    """
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_instances):
        n = int(rng.integers(side_range[0], side_range[1] + 1))
        mesh = box_mesh((n, n, n), periodic=(False, False, False), walls="slip", name=f"riemann{k}_{n}")
        states = []
        for _ in range(2):
            rho = rng.uniform(0.1, 2.0)
            u = tuple(rng.uniform(-2.0, 2.0, size=3))
            p = rng.uniform(0.1, 10.0)
            states.append((rho, u, p))
        nrm = rng.normal(size=3)
        nrm /= np.linalg.norm(nrm)
        out.append((mesh, riemann_state(mesh.x, states[0], states[1], normal=tuple(nrm))))
    return out


def random_riemann_batch_2d(n_instances=256, side_range=(16, 160), seed=6):
    """Independent 2D Riemann problems on slip-walled unit squares of random size
    (Q1 quadrilaterals); states drawn as in ``random_riemann_batch`` with u_z = 0
    and a uniformly random in-plane interface normal."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_instances):
        n = int(rng.integers(side_range[0], side_range[1] + 1))
        mesh = rect_mesh((n, n), periodic=(False, False), walls="slip", name=f"riemann2d{k}_{n}")
        states = []
        for _ in range(2):
            rho = rng.uniform(0.1, 2.0)
            u = tuple(rng.uniform(-2.0, 2.0, size=2)) + (0.0,)
            p = rng.uniform(0.1, 10.0)
            states.append((rho, u, p))
        a = rng.uniform(0.0, 2.0 * np.pi)
        out.append((mesh, riemann_state(mesh.x, states[0], states[1], normal=(np.cos(a), np.sin(a), 0.0),
                                        point=(0.5, 0.5, 0.0))))
    return out


def vortex_mesh(n, nz=None, jitter=0.0, seed=0):
    """Periodic unit cube with ``n`` nodes along x and y (``nz`` along z, default ``n``)."""
    return box_mesh((n, n, nz or n), periodic=(True, True, True), jitter=jitter, seed=seed,
                    name=f"vortex{n}x{n}x{nz or n}")


def sod_mesh(nx, ny=4, nz=4):
    """Shock tube [0,1]x[0,1]x[0,1] with slip walls along x, periodic in y and z."""
    return box_mesh((nx, ny, nz), periodic=(False, True, True), walls="slip", name=f"sod{nx}")


def sod_cube_mesh(n=128):
    """128^3-node slip-walled unit cube for the 3D Sod precision workload."""
    return box_mesh((n, n, n), periodic=(False, False, False), walls="slip", name=f"sodcube{n}")


def concat_meshes(meshes, states=None):
    """Union of independent meshes in one HexMesh.

    Node ids of mesh k are shifted by the node count of meshes 0..k-1, so the
    instances occupy contiguous node ranges and share no cell.  Returns
    ``(mesh, node_offsets, U)`` with ``node_offsets`` of length len(meshes)+1
    and ``U`` the concatenated states (None if ``states`` is None).
    """
    offsets = [0]
    for m in meshes:
        offsets.append(offsets[-1] + m.n_nodes)
    cells = np.concatenate([m.cells + off for m, off in zip(meshes, offsets[:-1])])
    x = np.concatenate([m.x for m in meshes])
    cell_xyz = np.concatenate([m.cell_xyz for m in meshes])
    bc = np.concatenate([m.bc for m in meshes]).astype(np.int32)
    U = None if states is None else np.concatenate([np.asarray(u) for u in states], axis=1)
    mesh = HexMesh(x=x, cells=cells, cell_xyz=cell_xyz, bc=bc, volume=float(sum(m.volume for m in meshes)),
                   name=f"batch{len(meshes)}", meta={"instances": len(meshes)})
    return mesh, np.asarray(offsets, dtype=np.int64), U
