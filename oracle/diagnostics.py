"""Flow diagnostics of the paper's benchmark flows (test infrastructure, see ``oracle``).

Sect. 3.3 reports the drag and lift of the cylinder (and their viscous and pressure parts) and the
Strouhal number St = f_s d / u_inf of the shedding (Eq. 42); Sect. 3.2 the reattachment length of
the backward-facing step. The paper prints no formula for the forces; this module takes the
standard definitions, written out here:

* force on a body, F = sum over its boundary edges of the traction sigma n_b integrated along the
  edge, sigma = -p I + mu (grad u + grad u^T), n_b the unit normal pointing from the body into
  the fluid; p is P1 on the edge (the trapezoid rule is exact), grad u is the constant P1
  gradient of the fluid triangle that owns the edge. Pressure part: -int p n_b; viscous part:
  int mu (grad u + grad u^T) n_b. C_D = 2 F_x / (rho u_inf^2 d), C_L = 2 F_y / (rho u_inf^2 d);
* wall shear along a wall, tau = mu t . (grad u) n_f per wall edge (t the unit tangent along
  increasing x, n_f the unit normal into the fluid); the reattachment point is the first x past
  x_start where tau changes from negative to non-negative, interpolated linearly between the edge
  midpoints (None if there is none);
* the Strouhal number from a lift series: the mean period between upward zero crossings of
  C_L - mean(C_L) over the series' second half.
"""
from __future__ import annotations

import numpy as np


def boundary_edges(tri: np.ndarray, n_nodes: int):
    """Edges that belong to one triangle: ``(a, b, t)`` with (a, b) in the triangle's CCW order, so
    the fluid lies to the left of a -> b and the outward normal of the fluid domain to the right."""
    tri = np.asarray(tri, dtype=np.int64)
    loc = np.stack([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]], axis=1).reshape(-1, 2)
    owner = np.repeat(np.arange(tri.shape[0]), 3)
    key = np.minimum(loc[:, 0], loc[:, 1]) * n_nodes + np.maximum(loc[:, 0], loc[:, 1])
    uniq, inv, cnt = np.unique(key, return_inverse=True, return_counts=True)
    single = cnt[inv] == 1
    return loc[single, 0], loc[single, 1], owner[single]


def _grad_u(xy, tri, u, t):
    """Constant P1 velocity gradient G[c, d] = d u_c / d x_d on triangle t."""
    p = xy[tri[t]]
    V = np.column_stack([np.ones(3), p[:, 0], p[:, 1]])
    C = np.linalg.inv(V)               # [1, x, y] @ C[:, i] = phi_i
    gphi = C[1:, :]                    # [2 (d/dx, d/dy), 3]
    return u[tri[t]].T @ gphi.T        # [2 (u, v), 2 (x, y)]


def body_force(xy, tri, u, p, mu, body_nodes):
    """(pressure force [2], viscous force [2]) on the body whose boundary edges have both ends in
    ``body_nodes`` (bool per node); u [n, 2] and p [n] nodal fields of the fine mesh."""
    a, b, t = boundary_edges(tri, xy.shape[0])
    sel = body_nodes[a] & body_nodes[b]
    fp, fv = np.zeros(2), np.zeros(2)
    for ea, eb, et in zip(a[sel], b[sel], t[sel]):
        d = xy[eb] - xy[ea]
        length = float(np.hypot(d[0], d[1]))
        n_out = np.array([d[1], -d[0]]) / length     # right of a -> b: out of the fluid
        n_b = -n_out                                  # from the body into the fluid
        fp += -0.5 * (p[ea] + p[eb]) * length * n_b
        G = _grad_u(xy, tri, u, et)
        fv += mu * length * ((G + G.T) @ n_b)
    return fp, fv


def wall_shear(xy, tri, u, mu, wall_nodes):
    """(x of each wall edge midpoint, tau per edge), edges sorted by x."""
    a, b, t = boundary_edges(tri, xy.shape[0])
    sel = wall_nodes[a] & wall_nodes[b]
    xs, taus = [], []
    for ea, eb, et in zip(a[sel], b[sel], t[sel]):
        d = xy[eb] - xy[ea]
        length = float(np.hypot(d[0], d[1]))
        tvec = d / length
        if tvec[0] < 0:
            tvec = -tvec
        n_out = np.array([d[1], -d[0]]) / length
        n_f = -n_out
        G = _grad_u(xy, tri, u, et)
        xs.append(0.5 * (xy[ea, 0] + xy[eb, 0]))
        taus.append(mu * float(tvec @ G @ n_f))
    order = np.argsort(xs, kind="stable")
    return np.asarray(xs)[order], np.asarray(taus)[order]


def reattachment(xs, taus, x_start):
    """First x >= x_start where tau goes from negative to non-negative (linear interpolation
    between edge midpoints), or None."""
    for k in range(len(xs) - 1):
        if xs[k] < x_start:
            continue
        if taus[k] < 0.0 <= taus[k + 1]:
            return float(xs[k] - taus[k] * (xs[k + 1] - xs[k]) / (taus[k + 1] - taus[k]))
    return None


def strouhal(t, cl, d=1.0, u_inf=1.0):
    """St = f_s d / u_inf from the mean period of upward zero crossings of cl - mean over the
    series' second half; None with fewer than two crossings."""
    t, cl = np.asarray(t, dtype=np.float64), np.asarray(cl, dtype=np.float64)
    h = len(t) // 2
    t, c = t[h:], cl[h:] - cl[h:].mean()
    up = np.nonzero((c[:-1] < 0.0) & (c[1:] >= 0.0))[0]
    if len(up) < 2:
        return None
    tc = t[up] - c[up] * (t[up + 1] - t[up]) / (c[up + 1] - c[up])
    return d / (u_inf * float(np.mean(np.diff(tc))))
