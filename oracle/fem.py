"""P1 element matrices and global assembly (test infrastructure, see ``oracle``).

The paper's Eqs. 16-18 use the velocity mass matrix M_v, the convection matrix N, the velocity and
pressure Laplacians L_v, L_p, the divergence D and the gradient G, all with piecewise-linear
(P1) shape functions. On a triangle T of area |T| with shape functions phi_1..phi_3 the gradients
are constant, and the exact integrals are

    int_T phi_i phi_j            = |T| (1 + delta_ij) / 12                    (mass)
    int_T grad phi_i . grad phi_j = |T| grad phi_i . grad phi_j               (stiffness)
    int_T phi_i d_x phi_j        = |T| / 3 * d_x phi_j                        (divergence, gradient)
    int_T phi_i (u . grad phi_j)  = |T| / 12 * (sum_k u_k + u_i) . grad phi_j   (convection, u in P1)

with grad phi_i = (y_j - y_k, x_k - x_j) / (2|T|) for (i, j, k) a cyclic permutation of (1, 2, 3).
The stiffness matrix K is +(-Laplacian), so it is positive semi-definite; the divergence D is not
integrated by parts. On the fine mesh G = D because pressure and velocity share the P1 space.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def triangle_geometry(xy: np.ndarray, tri: np.ndarray):
    """Areas |T| and shape-function gradients (int64 tri). Returns ``(area[T], gx[T,3], gy[T,3])``."""
    p = xy[tri]                                     # [T, 3, 2]
    x, y = p[..., 0], p[..., 1]
    area = 0.5 * ((x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0]))
    j = [1, 2, 0]
    k = [2, 0, 1]
    gx = (y[:, j] - y[:, k]) / (2.0 * area[:, None])
    gy = (x[:, k] - x[:, j]) / (2.0 * area[:, None])
    return area, gx, gy


def element_mass(area):
    """[T,3,3] element mass matrices."""
    base = (np.ones((3, 3)) + np.eye(3)) / 12.0
    return area[:, None, None] * base[None]


def element_stiffness(area, gx, gy):
    """[T,3,3] element stiffness matrices int grad phi_i . grad phi_j."""
    return area[:, None, None] * (gx[:, :, None] * gx[:, None, :] + gy[:, :, None] * gy[:, None, :])


def element_div(area, g):
    """[T,3,3] element matrices int phi_i d phi_j (g = gx or gy)."""
    return np.broadcast_to((area / 3.0)[:, None, None] * g[:, None, :], (area.shape[0], 3, 3)).copy()


def element_convection(area, gx, gy, u_el):
    """[T,3,3] element convection matrices int phi_i (u . grad phi_j), u_el = [T,3,2] nodal u."""
    s = u_el.sum(axis=1, keepdims=True)             # [T,1,2]
    c = (area[:, None, None] / 12.0) * (s + u_el)   # [T,3,2] coefficient vector per test function
    return c[:, :, 0:1] * gx[:, None, :] + c[:, :, 1:2] * gy[:, None, :]


def assemble(tri: np.ndarray, ke: np.ndarray, n: int) -> sp.csr_matrix:
    """Sum element matrices ``ke[T,3,3]`` into an ``n`` x ``n`` CSR matrix."""
    rows = np.repeat(tri, 3, axis=1).ravel()
    cols = np.tile(tri, (1, 3)).ravel()
    return sp.coo_matrix((ke.ravel(), (rows, cols)), shape=(n, n)).tocsr()


class P1Operators:
    """Constant P1 matrices of one mesh: M, K, Dx, Dy (and the geometry for N(u))."""

    def __init__(self, xy: np.ndarray, tri: np.ndarray):
        self.xy = np.asarray(xy, dtype=np.float64)
        self.tri = np.asarray(tri, dtype=np.int64)
        self.n = self.xy.shape[0]
        self.area, self.gx, self.gy = triangle_geometry(self.xy, self.tri)
        self.M = assemble(self.tri, element_mass(self.area), self.n)
        self.K = assemble(self.tri, element_stiffness(self.area, self.gx, self.gy), self.n)
        self.Dx = assemble(self.tri, element_div(self.area, self.gx), self.n)
        self.Dy = assemble(self.tri, element_div(self.area, self.gy), self.n)

    def convection(self, u: np.ndarray) -> sp.csr_matrix:
        """N(u) with N_ij = int phi_i (u . grad phi_j), u given at the nodes [n, 2]."""
        return assemble(self.tri, element_convection(self.area, self.gx, self.gy, u[self.tri]), self.n)
