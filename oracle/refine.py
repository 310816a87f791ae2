"""Nested 1:4 refinement and the CGP mapping tables (test infrastructure, see ``oracle``).

The paper's Sect. 2.2 builds the mesh hierarchy by splitting every coarse triangle conformingly
into four, and Remark 2.2 replaces the prolongation and restriction matrices by two index tables:

* s^p (Eq. 29): for each node alpha of the finer mesh a pair (beta, gamma) of coarser nodes with
  P_f(alpha) = (P_c(beta) + P_c(gamma)) / 2;
* s^u (Eq. 30): for each node eta of the coarser mesh the index xi of the same point on the finer
  mesh, with U_c(eta) = U_f(xi).

Besides the injection R of Eq. 30 this module gives the transpose P^T of the prolongation, which
the Galerkin reading of the restriction uses (b_c = P^T applied to a fine-mesh load vector).

Numbering convention (shared with the CUDA library by specification, not by code): the parent
nodes keep their indices 0..N_k-1; every edge gets one midpoint, appended in order of first visit
(triangles in order, local edges (a,b), (b,c), (c,a)); triangle (a,b,c) becomes the four children
(a, m_ab, m_ca), (m_ab, b, m_bc), (m_ca, m_bc, c), (m_ab, m_bc, m_ca), stored at 4t..4t+3.
Midpoints on curved boundaries are not moved onto the curve, so the spaces stay nested.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def edges_first_visit(tri: np.ndarray, n_nodes: int):
    """Unique undirected edges of a triangle mesh in order of first visit.

    Returns ``(edges int64[E,2] as (min,max), edge_of int64[T,3])`` where ``edge_of[t, e]`` is the
    index of local edge e (0: a-b, 1: b-c, 2: c-a) of triangle t.
    """
    tri = np.asarray(tri, dtype=np.int64)
    loc = np.stack([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]], axis=1).reshape(-1, 2)
    lo = loc.min(axis=1)
    hi = loc.max(axis=1)
    key = lo * n_nodes + hi
    uniq, first, inv = np.unique(key, return_index=True, return_inverse=True)
    order = np.argsort(first, kind="stable")          # unique keys sorted by first visit
    rank = np.empty_like(order)
    rank[order] = np.arange(len(order))
    edge_of = rank[inv].reshape(-1, 3)
    edges = np.stack([lo[first[order]], hi[first[order]]], axis=1)
    return edges, edge_of


def boundary_nodes(tri: np.ndarray, n_nodes: int) -> np.ndarray:
    """Nodes lying on an edge that belongs to exactly one triangle."""
    edges, edge_of = edges_first_visit(tri, n_nodes)
    count = np.bincount(edge_of.ravel(), minlength=len(edges))
    onb = np.zeros(n_nodes, dtype=bool)
    be = edges[count == 1]
    onb[be[:, 0]] = True
    onb[be[:, 1]] = True
    return onb


@dataclass
class Level:
    """One mesh of the hierarchy."""
    xy: np.ndarray        # [N, 2]
    tri: np.ndarray       # [T, 3] int64, counter-clockwise


@dataclass
class Hierarchy:
    """Meshes V_c = levels[0] (coarse, pressure) ... levels[-1] = V_f (fine, velocity).

    ``sp[k]`` is the s^p table (int64[N_{k+1}, 2]) from level k to level k+1; ``su`` is the s^u
    table (int64[N_c]) from the coarse mesh straight to the fine mesh (Eq. 30 may skip levels).
    """
    levels: list
    sp: list
    su: np.ndarray

    @property
    def coarse(self) -> Level:
        return self.levels[0]

    @property
    def fine(self) -> Level:
        return self.levels[-1]


def refine_once(xy: np.ndarray, tri: np.ndarray):
    """One conforming 1:4 split (Sect. 2.2). Returns ``(xy_f, tri_f, sp, su)``.

    ``sp`` is the s^p table of Eq. 29 for the new mesh, ``su`` the s^u table of Eq. 30 for the
    old mesh.
    """
    n = xy.shape[0]
    tri = np.asarray(tri, dtype=np.int64)
    edges, edge_of = edges_first_visit(tri, n)
    mid = n + edge_of                                   # midpoint node of each local edge
    xy_f = np.concatenate([xy, 0.5 * (xy[edges[:, 0]] + xy[edges[:, 1]])], axis=0)
    a, b, c = tri[:, 0], tri[:, 1], tri[:, 2]
    mab, mbc, mca = mid[:, 0], mid[:, 1], mid[:, 2]
    kids = np.stack([
        np.stack([a, mab, mca], 1),
        np.stack([mab, b, mbc], 1),
        np.stack([mca, mbc, c], 1),
        np.stack([mab, mbc, mca], 1),
    ], axis=1).reshape(-1, 3)
    sp = np.concatenate([np.stack([np.arange(n), np.arange(n)], 1), edges], axis=0)
    su = np.arange(n, dtype=np.int64)
    return xy_f, kids, sp, su


def build_hierarchy(xy: np.ndarray, tri: np.ndarray, levels: int) -> Hierarchy:
    """Refine the coarse mesh ``levels`` times and collect the mapping tables."""
    lv = [Level(np.asarray(xy, dtype=np.float64), np.asarray(tri, dtype=np.int64))]
    sps = []
    su = np.arange(xy.shape[0], dtype=np.int64)
    for _ in range(levels):
        xf, tf, sp, su_k = refine_once(lv[-1].xy, lv[-1].tri)
        sps.append(sp)
        su = su_k[su]           # compose: the coarse node's index on the newest level
        lv.append(Level(xf, tf))
    return Hierarchy(lv, sps, su)


def prolong(h: Hierarchy, p_c: np.ndarray) -> np.ndarray:
    """P_k^{k+1} applied level by level (Eq. 22 through the table of Eq. 29)."""
    p = np.asarray(p_c, dtype=np.float64)
    for sp in h.sp:
        p = 0.5 * (p[sp[:, 0]] + p[sp[:, 1]])
    return p


def restrict(h: Hierarchy, u_f: np.ndarray) -> np.ndarray:
    """Injection R (Eq. 20 through the table of Eq. 30)."""
    return np.asarray(u_f)[h.su]


def restrict_transpose(h: Hierarchy, r_f: np.ndarray) -> np.ndarray:
    """P^T applied level by level, from the fine mesh down to the coarse mesh.

    Row alpha of P_k^{k+1} (Eq. 29) holds the weight 1/2 at columns beta_alpha and gamma_alpha
    (a single weight 1 when beta = gamma = alpha), so P^T r gives every coarser node beta half of
    r[alpha] for each finer node alpha whose pair contains beta, plus r[beta] itself from its
    parent-coincident row. For a fine-mesh load vector r_i = int phi_i f, (P^T r)_j = int psi_j f
    with psi_j the coarse shape function, since psi_j = sum_i P_ij phi_i on nested meshes.
    """
    r = np.asarray(r_f, dtype=np.float64)
    for k in range(len(h.sp) - 1, -1, -1):
        sp = h.sp[k]
        out = np.zeros(h.levels[k].xy.shape[0])
        np.add.at(out, sp[:, 0], 0.5 * r)
        np.add.at(out, sp[:, 1], 0.5 * r)
        r = out
    return r
