"""Seeded synthetic inputs for the coarse-grid-projection (CGP) step.

This module is shared by the CUDA path's tests/bench and by the CPU oracle. It
holds only problem *data*: coarse meshes drawn from a counter-based generator,
boundary classification, boundary values and initial fields. None of the
method's arithmetic (refinement, element matrices, solves, mapping) is here.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used in counter form: draw ``k``
of stream ``seed`` is ``mix(seed + (k + 1) * 0x9E3779B97F4A7C15)``.

Workloads (the paper's Sect. 3 flows, reshaped to seeded synthetic meshes):

* lid-driven cavity on the unit square (jittered random-diagonal grid);
* backward-facing-step channel [0,30]x[0,2] minus the step [0,1]x[0,1]
  (the paper's Sect. 3.2 geometry scaled by 2, parabolic inflow, open outflow);
* Taylor-Green vortex on the unit square with exact Dirichlet data
  (the paper's Eqs. 34-36; the paper's holed square is replaced by the plain
  square so the jittered-grid generator can be reused).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """SplitMix64 output number ``idx`` (0-based) of the stream started at ``seed``."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (idx + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, idx: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, idx) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# --------------------------------------------------------------------------------------
# Coarse meshes
# --------------------------------------------------------------------------------------

@dataclass
class CoarseMesh:
    """A coarse P1 triangle mesh: node coordinates and counter-clockwise triangles."""
    xy: np.ndarray          # float64 [n_nodes, 2]
    tri: np.ndarray         # int32   [n_tris, 3], counter-clockwise
    name: str = ""

    @property
    def n_nodes(self) -> int:
        return int(self.xy.shape[0])

    @property
    def n_tris(self) -> int:
        return int(self.tri.shape[0])


def jittered_grid(x0: float, x1: float, y0: float, y1: float, nx: int, ny: int, seed: int,
                  removed_cell: Callable[[np.ndarray, np.ndarray], np.ndarray] | None = None,
                  jitter: float = 0.2) -> CoarseMesh:
    """Grid of ``nx`` x ``ny`` cells, each split by a seed-random diagonal, interior nodes jittered.

    Draw layout of the SplitMix64 stream ``seed``: draw ``c`` (cell ``c = j*nx + i`` of the full
    bounding grid) picks the diagonal by its top bit; draws ``nx*ny + 2k`` and ``nx*ny + 2k + 1``
    jitter node ``k = j*(nx+1) + i`` in x and y by ``U[-jitter*h, +jitter*h]``. Nodes on the
    domain boundary (the boundary of the kept cells) are not moved. Cells for which
    ``removed_cell(i, j)`` is true are cut out; nodes that no kept cell touches are dropped and the
    rest renumbered in row-major order.
    """
    hx = (x1 - x0) / nx
    hy = (y1 - y0) / ny
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")  # [ny, nx]
    keep = np.ones((ny, nx), dtype=bool)
    if removed_cell is not None:
        keep = ~removed_cell(ii, jj)
    n_cells = nx * ny
    diag = (splitmix64(seed, np.arange(n_cells)) >> np.uint64(63)).astype(np.int64).reshape(ny, nx)

    # node usage and boundary detection: a node is on the boundary if its 4 surrounding cells are
    # not all kept (cells outside the bounding box count as removed)
    kp = np.zeros((ny + 2, nx + 2), dtype=bool)
    kp[1:-1, 1:-1] = keep
    # node (i, j) touches cells (i-1..i, j-1..j) -> padded indices (i..i+1, j..j+1)
    c00 = kp[0:ny + 1, 0:nx + 1]
    c10 = kp[0:ny + 1, 1:nx + 2]
    c01 = kp[1:ny + 2, 0:nx + 1]
    c11 = kp[1:ny + 2, 1:nx + 2]
    used = c00 | c10 | c01 | c11
    interior = c00 & c10 & c01 & c11

    nI, nJ = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
    # (x1-x0)*i/nx rather than i*hx so that grid lines such as x = 1 land exactly
    x = x0 + (x1 - x0) * nI / nx
    y = y0 + (y1 - y0) * nJ / ny
    k = (nJ * (nx + 1) + nI).astype(np.int64)
    jx = (2.0 * uniform01(seed, n_cells + 2 * k) - 1.0) * jitter * hx
    jy = (2.0 * uniform01(seed, n_cells + 2 * k + 1) - 1.0) * jitter * hy
    x = np.where(interior, x + jx, x)
    y = np.where(interior, y + jy, y)

    new_id = -np.ones((ny + 1) * (nx + 1), dtype=np.int64)
    used_flat = used.ravel()
    new_id[used_flat] = np.arange(int(used_flat.sum()))
    xy = np.stack([x.ravel()[used_flat], y.ravel()[used_flat]], axis=1)

    tris = []
    cj, ci = np.nonzero(keep)
    a = cj * (nx + 1) + ci
    b = a + 1
    c = a + (nx + 1) + 1
    d = a + (nx + 1)
    dg = diag[cj, ci]
    # diagonal a-c: (a,b,c), (a,c,d); diagonal b-d: (a,b,d), (b,c,d); both counter-clockwise
    t1 = np.where(dg[:, None] == 0, np.stack([a, b, c], 1), np.stack([a, b, d], 1))
    t2 = np.where(dg[:, None] == 0, np.stack([a, c, d], 1), np.stack([b, c, d], 1))
    tri = np.empty((2 * len(a), 3), dtype=np.int64)
    tri[0::2] = t1
    tri[1::2] = t2
    tris = new_id[tri]
    assert (tris >= 0).all()
    return CoarseMesh(xy=np.ascontiguousarray(xy, dtype=np.float64),
                      tri=np.ascontiguousarray(tris, dtype=np.int32))


def cavity_mesh(n_side: int = 33, seed: int = 1000) -> CoarseMesh:
    """Unit-square cavity mesh with ``n_side`` x ``n_side`` grid nodes."""
    m = jittered_grid(0.0, 1.0, 0.0, 1.0, n_side - 1, n_side - 1, seed)
    m.name = f"cavity{n_side}"
    return m


def bfs_mesh(cells_per_unit: int = 33, seed: int = 1001) -> CoarseMesh:
    """Backward-facing-step channel [0,30]x[0,2] minus the step [0,1]x[0,1]."""
    n = cells_per_unit
    nx, ny = 30 * n, 2 * n
    m = jittered_grid(0.0, 30.0, 0.0, 2.0, nx, ny, seed,
                      removed_cell=lambda i, j: (i < n) & (j < n))
    m.name = f"bfs{n}"
    return m


def centroid_split(m: CoarseMesh, n_split: int) -> CoarseMesh:
    """``m`` with its first ``n_split`` even-numbered triangles each divided at its centroid into
    three counter-clockwise triangles: one node and two triangles more per split, the boundary
    unchanged. Reaches a prescribed node and triangle count (a jittered grid fixes the boundary
    node count, the splits the rest)."""
    tri = np.asarray(m.tri, dtype=np.int64)
    sel = np.arange(0, 2 * n_split, 2)
    if n_split < 0 or (n_split > 0 and sel[-1] >= len(tri)):
        raise ValueError("not enough triangles to split")
    g = m.xy[tri[sel]].mean(axis=1)
    gi = m.n_nodes + np.arange(n_split)
    a, b, c = tri[sel, 0], tri[sel, 1], tri[sel, 2]
    keep = np.ones(len(tri), dtype=bool)
    keep[sel] = False
    new = np.concatenate([tri[keep], np.stack([a, b, gi], 1), np.stack([b, c, gi], 1), np.stack([c, a, gi], 1)])
    return CoarseMesh(xy=np.ascontiguousarray(np.concatenate([m.xy, g]), dtype=np.float64),
                      tri=np.ascontiguousarray(new.astype(np.int32)), name=f"{m.name}+{n_split}split")


# --------------------------------------------------------------------------------------
# Boundary conditions and problem definitions
# --------------------------------------------------------------------------------------

BC_U = 1   # bit 0: x-velocity Dirichlet
BC_V = 2   # bit 1: y-velocity Dirichlet


@dataclass
class Problem:
    """A flow problem: physical constants and boundary data as functions of node positions.

    ``vel_bc(xy, on_boundary, t)`` returns ``(mask uint8[N], g float64[N,2])``: bit 0 / bit 1 of
    ``mask`` mark nodes where u / v is prescribed, ``g`` holds the prescribed values (zero where
    not prescribed). ``p_bc(xy, on_boundary)`` returns a uint8[N] mask of pressure nodes held at
    p = 0 (the open boundary of the paper's Eq. 14, plus one pinned node for enclosed flows).
    ``u0(xy, mask, g)`` is the initial velocity.
    """
    name: str
    rho: float
    mu: float
    dt: float
    levels: int
    vel_bc: Callable
    p_bc: Callable
    u0: Callable
    time_dependent_bc: bool = False
    extra: dict = field(default_factory=dict)


def _zero_u0(xy, mask, g):
    u = np.zeros((xy.shape[0], 2))
    u[mask & BC_U != 0, 0] = g[mask & BC_U != 0, 0]
    u[mask & BC_V != 0, 1] = g[mask & BC_V != 0, 1]
    return u


def cavity_problem(re: float = 100.0, dt: float = 0.01, levels: int = 1) -> Problem:
    """Lid-driven cavity: lid y=1 moves with u=1, other walls no-slip; corners take u=0.

    The enclosed pressure problem is pinned at the node nearest (0, 0)."""

    def vel_bc(xy, onb, t):
        mask = np.where(onb, BC_U | BC_V, 0).astype(np.uint8)
        g = np.zeros((xy.shape[0], 2))
        lid = onb & (xy[:, 1] == 1.0) & (xy[:, 0] > 0.0) & (xy[:, 0] < 1.0)
        g[lid, 0] = 1.0
        return mask, g

    def p_bc(xy, onb):
        m = np.zeros(xy.shape[0], dtype=np.uint8)
        m[int(np.argmin(xy[:, 0] ** 2 + xy[:, 1] ** 2))] = 1
        return m

    return Problem("cavity", 1.0, 1.0 / re, dt, levels, vel_bc, p_bc, _zero_u0)


def bfs_problem(re: float = 400.0, dt: float = 0.005, levels: int = 1) -> Problem:
    """Backward-facing step (the paper's Sect. 3.2 geometry scaled by 2).

    Inflow on x=0, 1<=y<=2: u = 6(y-1)(2-y) (mean 1), v = 0. Walls no-slip. Outflow x=30 natural
    for the velocity and p = 0 for the pressure (Eq. 14). Re = rho*H*mean/mu with H = 2.
    """

    def vel_bc(xy, onb, t):
        x, y = xy[:, 0], xy[:, 1]
        outflow = onb & (x == 30.0) & (y > 0.0) & (y < 2.0)
        dir_ = onb & ~outflow
        mask = np.where(dir_, BC_U | BC_V, 0).astype(np.uint8)
        g = np.zeros((xy.shape[0], 2))
        inflow = onb & (x == 0.0) & (y > 1.0) & (y < 2.0)
        g[inflow, 0] = 6.0 * (y[inflow] - 1.0) * (2.0 - y[inflow])
        return mask, g

    def p_bc(xy, onb):
        return (onb & (xy[:, 0] == 30.0)).astype(np.uint8)

    return Problem("bfs", 1.0, 2.0 / re, dt, levels, vel_bc, p_bc, _zero_u0)


def taylor_green_velocity(xy: np.ndarray, t: float, mu: float) -> np.ndarray:
    """Taylor-Green velocity of the paper's Eqs. 34-35 (rho = 1)."""
    x, y = xy[:, 0], xy[:, 1]
    d = math.exp(-8.0 * math.pi ** 2 * mu * t)
    return np.stack([-np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y) * d,
                     np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) * d], axis=1)


def taylor_green_pressure(xy: np.ndarray, t: float, mu: float) -> np.ndarray:
    """Taylor-Green pressure of the paper's Eq. 36 (rho = 1)."""
    x, y = xy[:, 0], xy[:, 1]
    return -(np.cos(4 * np.pi * x) + np.cos(4 * np.pi * y)) / 4.0 * math.exp(-16.0 * math.pi ** 2 * mu * t)


def taylor_green_problem(mu: float = 0.01, dt: float = 0.01, levels: int = 1) -> Problem:
    """Taylor-Green vortex on the unit square with exact Dirichlet velocity on the whole boundary.

    All-Dirichlet velocity gives a pure-Neumann pressure problem (Eq. 13), pinned at the node
    nearest (0, 0); pressures are compared modulo a constant."""

    def vel_bc(xy, onb, t):
        mask = np.where(onb, BC_U | BC_V, 0).astype(np.uint8)
        g = np.where(onb[:, None], taylor_green_velocity(xy, t, mu), 0.0)
        return mask, g

    def p_bc(xy, onb):
        m = np.zeros(xy.shape[0], dtype=np.uint8)
        m[int(np.argmin(xy[:, 0] ** 2 + xy[:, 1] ** 2))] = 1
        return m

    def u0(xy, mask, g):
        return taylor_green_velocity(xy, 0.0, mu)

    return Problem("taylor_green", 1.0, mu, dt, levels, vel_bc, p_bc, u0, time_dependent_bc=True)


def batch_cavities(n_inst: int = 64, seed: int = 1003, n_min: int = 2000, n_max: int = 50000,
                   re_min: float = 100.0, re_max: float = 1000.0, dt: float = 0.005):
    """Independent lid-driven cavities of uneven size: a list of ``(CoarseMesh, Problem)``.

    Instance i uses the SplitMix64 stream ``seed * 1000 + i``: draw 0 gives the coarse node
    count N_i = exp(U[ln n_min, ln n_max]) (log-uniform, grid side round(sqrt(N_i))), draw 1 the
    Reynolds number U[re_min, re_max]; the mesh itself is drawn by ``jittered_grid`` from the
    stream ``seed * 1000 + i + 7919``."""
    out = []
    for i in range(n_inst):
        s = seed * 1000 + i
        u = uniform01(s, np.arange(2))
        n_c = math.exp(math.log(n_min) + u[0] * (math.log(n_max) - math.log(n_min)))
        side = max(3, int(round(math.sqrt(n_c))))
        re = re_min + u[1] * (re_max - re_min)
        mesh = jittered_grid(0.0, 1.0, 0.0, 1.0, side - 1, side - 1, s + 7919)
        mesh.name = f"cavity{side}"
        out.append((mesh, cavity_problem(re, dt, 1)))
    return out


def cylinder_mesh(h_min: float = 0.0297, seed: int = 1002, length: float = 30.0, height: float = 10.0,
                  centre=(5.0, 5.0), radius: float = 0.5, grading: float = 5.0) -> CoarseMesh:
    """Flow past a cylinder: [0,length]x[0,height] minus a disc, Poisson-disk points, Delaunay.

    The target spacing is h(d) = h_min (1 + min(1, d / grading)) with d the distance to the
    cylinder surface (twice as fine, four times as dense, near the cylinder). Boundary points are
    placed on the rectangle and the circle at that spacing; interior points come from dart
    throwing (Cook 1986): candidates drawn from SplitMix64 stream ``seed`` are accepted when no
    accepted point lies closer than the local spacing. The points are Delaunay-triangulated
    (scipy.spatial, Qhull), triangles inside the disc removed and all triangles made
    counter-clockwise."""
    from scipy.spatial import Delaunay

    cx, cy = centre

    def spacing(x, y):
        d = np.sqrt((x - cx) ** 2 + (y - cy) ** 2) - radius
        return h_min * (1.0 + np.minimum(1.0, np.maximum(d, 0.0) / grading))

    pts = []
    # rectangle edges, walked with the local spacing (corners included once)
    for (x0, y0, x1, y1) in ((0, 0, length, 0), (length, 0, length, height), (length, height, 0, height),
                             (0, height, 0, 0)):
        t = 0.0
        L = math.hypot(x1 - x0, y1 - y0)
        while t < L - 1e-12:
            x = x0 + (x1 - x0) * t / L
            y = y0 + (y1 - y0) * t / L
            pts.append((float(x), float(y)))
            t += float(spacing(np.array(x), np.array(y)))
    for (x, y) in list(pts):
        pass
    # snap the walked coordinates onto the exact edge lines
    fixed = []
    for (x, y) in pts:
        if abs(y) < 1e-9:
            y = 0.0
        if abs(y - height) < 1e-9:
            y = height
        if abs(x) < 1e-9:
            x = 0.0
        if abs(x - length) < 1e-9:
            x = length
        fixed.append((x, y))
    pts = fixed
    nc = max(12, int(round(2.0 * math.pi * radius / h_min)))
    for k in range(nc):
        a = 2.0 * math.pi * k / nc
        pts.append((cx + radius * math.cos(a), cy + radius * math.sin(a)))
    # dart throwing on a background grid of cell h_min / sqrt(2) (at most one point per cell)
    cell = h_min / math.sqrt(2.0)
    gx, gy = int(math.ceil(length / cell)) + 1, int(math.ceil(height / cell)) + 1
    grid = -np.ones((gy, gx), dtype=np.int64)
    P = [np.array(p) for p in pts]
    for i, (x, y) in enumerate(pts):
        grid[min(gy - 1, int(y / cell)), min(gx - 1, int(x / cell))] = i
    reach = int(math.ceil(2.0 * h_min / cell))
    n_cand = int(6.0 * length * height / (h_min * h_min))
    u = uniform01(seed, np.arange(2 * n_cand, dtype=np.uint64)).reshape(-1, 2)
    cand = np.stack([u[:, 0] * length, u[:, 1] * height], axis=1)
    r_c = spacing(cand[:, 0], cand[:, 1])
    dc = np.sqrt((cand[:, 0] - cx) ** 2 + (cand[:, 1] - cy) ** 2)
    margin_ok = (cand[:, 0] > 0.5 * r_c) & (cand[:, 0] < length - 0.5 * r_c) & (cand[:, 1] > 0.5 * r_c) & \
        (cand[:, 1] < height - 0.5 * r_c) & (dc > radius + 0.5 * r_c)
    for k in np.flatnonzero(margin_ok):
        x, y = cand[k]
        r = r_c[k]
        i0, j0 = int(y / cell), int(x / cell)
        ok = True
        for i in range(max(0, i0 - reach), min(gy, i0 + reach + 1)):
            row = grid[i]
            for j in range(max(0, j0 - reach), min(gx, j0 + reach + 1)):
                q = row[j]
                if q >= 0:
                    dx, dy = P[q][0] - x, P[q][1] - y
                    if dx * dx + dy * dy < r * r:
                        ok = False
                        break
            if not ok:
                break
        if ok and grid[i0, j0] < 0:
            grid[i0, j0] = len(P)
            P.append(np.array((x, y)))
    xy = np.array(P, dtype=np.float64)
    tri = Delaunay(xy).simplices.astype(np.int64)
    c = xy[tri].mean(axis=1)
    tri = tri[(c[:, 0] - cx) ** 2 + (c[:, 1] - cy) ** 2 > radius ** 2]
    p = xy[tri]
    area2 = (p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1])
    tri[area2 < 0] = tri[area2 < 0][:, [0, 2, 1]]
    tri = tri[np.abs(area2) > 1e-14]
    used = np.zeros(len(xy), dtype=bool)
    used[tri.ravel()] = True
    remap = -np.ones(len(xy), dtype=np.int64)
    remap[used] = np.arange(int(used.sum()))
    m = CoarseMesh(xy=np.ascontiguousarray(xy[used]), tri=np.ascontiguousarray(remap[tri].astype(np.int32)))
    m.name = f"cylinder{m.n_nodes}"
    return m


def cylinder_problem(re: float = 100.0, dt: float = 0.002, levels: int = 2, length: float = 30.0,
                     height: float = 10.0) -> Problem:
    """Cylinder of diameter 1 in a channel (the paper's Sect. 3.3 set-up, shortened domain).

    Inflow x = 0: (u, v) = (1, 0). Top and bottom: slip walls, v = 0 prescribed and u natural
    (per-component masks). Cylinder: no-slip. Outflow x = length: natural, p = 0. Re = rho d u /
    mu with d = u = rho = 1, so mu = 1/Re."""

    def vel_bc(xy, onb, t):
        x, y = xy[:, 0], xy[:, 1]
        mask = np.zeros(xy.shape[0], dtype=np.uint8)
        g = np.zeros((xy.shape[0], 2))
        inflow = onb & (x == 0.0)
        wall = onb & ~inflow & ((y == 0.0) | (y == height))
        outflow = onb & (x == length) & ~wall
        cyl = onb & ~inflow & ~wall & ~outflow
        mask[inflow] = BC_U | BC_V
        g[inflow, 0] = 1.0
        mask[wall] = BC_V
        mask[cyl] = BC_U | BC_V
        return mask, g

    def p_bc(xy, onb):
        return (onb & (xy[:, 0] == length)).astype(np.uint8)

    return Problem("cylinder", 1.0, 1.0 / re, dt, levels, vel_bc, p_bc, _zero_u0)


def mlp_init_params(n: int, hidden: int, seed: int):
    """Initial weights of the warm-start network n -> hidden -> hidden -> n (float32 arrays).

    Uniform in +-0.5 sqrt(6 / fan_in) from SplitMix64 stream ``seed`` (W1, W2, W3 drawn in that
    order, row-major [out, in]); biases zero. Returned as [W1, b1, W2, b2, W3, b3]."""
    shapes = [(hidden, n), (hidden, hidden), (n, hidden)]
    out, off = [], 0
    for o, i in shapes:
        cnt = o * i
        u = uniform01(seed, np.arange(off, off + cnt, dtype=np.uint64))
        off += cnt
        bound = 0.5 * math.sqrt(6.0 / i)
        out.append(((2.0 * u - 1.0) * bound).astype(np.float32).reshape(o, i))
        out.append(np.zeros(o, dtype=np.float32))
    return out


# --------------------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------------------

def workload(name: str):
    """Return ``(CoarseMesh, Problem, n_steps)`` for a named workload.

    ``cavity33``: 33x33-node cavity, Re=100, dt=0.01, one refinement, 100 steps (seed 1000).
    ``bfs33``: backward-facing step, h=1/33 (65,308 coarse nodes), Re=400, dt=0.005, one
    refinement, 500 steps (seed 1001).
    ``cavity129``: 129x129-node cavity, Re=100, dt=0.005, one refinement (seed 1004).
    ``cylinder``: cylinder in [0,30]x[0,10], ~64k graded Poisson-disk coarse nodes, two
    refinements (~1M fine nodes), Re=100, dt=0.002, 2,000 steps (seed 1002).
    ``cylinder_small``: the same geometry at h_min = 0.25 (988 coarse nodes).
    ``cavityN`` for other N: an N x N-node cavity (seed 1000), Re=100, dt=0.01.
    """
    if name == "cavity33":
        return cavity_mesh(33, 1000), cavity_problem(100.0, 0.01, 1), 100
    if name == "bfs33":
        return bfs_mesh(33, 1001), bfs_problem(400.0, 0.005, 1), 500
    if name == "cylinder":
        return cylinder_mesh(), cylinder_problem(100.0, 0.002, 2), 2000
    if name == "cylinder_small":
        return cylinder_mesh(h_min=0.25), cylinder_problem(100.0, 0.002, 2), 2000
    if name == "cavity129":
        return cavity_mesh(129, 1004), cavity_problem(100.0, 0.005, 1), 200
    if name.startswith("bfs"):
        n = int(name[3:])
        return bfs_mesh(n, 1001), bfs_problem(400.0, 0.005, 1), 500
    if name.startswith("cavity"):
        n = int(name[6:])
        return cavity_mesh(n, 1000), cavity_problem(100.0, 0.01, 1), 100
    raise KeyError(name)
