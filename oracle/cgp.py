"""The IFE-CGP time step in plain FP64 (test infrastructure, see ``oracle``).

One time step follows the paper's five steps, Eqs. 19-23, with the density carried explicitly
(Eqs. 9, 12 and 15 contain rho; Eqs. 16-19 and 23 drop it, which is the same for rho = 1):

1. momentum, Eq. 19:   (rho M + dt rho N(u^n) + dt mu K) u~ = rho M u^n + dt M f^{n+1},
   with the rows of velocity-Dirichlet nodes replaced, per component, by identity rows whose
   right-hand side is the boundary value at t^{n+1} (Eqs. 10-11; natural outflow adds nothing);
2. restriction, Eq. 20: u~_c = u~_f[xi] (the s^u table of Eq. 30);
3. coarse Poisson, Eq. 21: K_c p_c = -(rho/dt) (Dx_c u~_c,x + Dy_c u~_c,y); K_c is the coarse
   stiffness (+(-Laplacian)), hence the minus sign against the paper's L_p; pressure-Dirichlet
   nodes (Eq. 14, plus a pin for enclosed flows) are eliminated symmetrically with p = 0;
4. prolongation, Eq. 22: p_f = P p_c through the s^p tables of Eq. 29, level by level;
5. correction, Eq. 23:  M w = G p_f,  u^{n+1} = u~ - (dt/rho) w, then Dirichlet nodes are reset
   to their boundary values (Eq. 3).

f = 0 in every workload here. All systems are solved by sparse LU.

Options beyond the paper's scheme (the paper's Sect. 4 and its comparison of restriction forms
leave these open; each is defined here in plain terms and checked by the pins in ``tests/``):

* ``restrict_mode = "galerkin"``: the coarse right-hand side restricts the fine divergence instead
  of injecting the velocity, b_c = -(rho/dt) P^T (Dx_f u~_x + Dy_f u~_y), i.e. the coarse test
  functions integrated against the divergence of the fine intermediate velocity;
* ``projection = "incremental"``: the momentum right-hand side carries the previous pressure,
  rho M u^n - dt G_f P p_c^n, the coarse Poisson solve gives the increment phi (same matrix and
  right-hand side as Eq. 21), the correction applies phi, and p_c^{n+1} = p_c^n + phi;
* ``projection = "rotational"``: as incremental, with p_c^{n+1} = p_c^n + phi - mu chi, where
  chi = -(dt/rho) M_L^-1 b_c is the discrete divergence the coarse right-hand side was built
  from (D_c u~_c with injection, P^T D_f u~_f with the Galerkin restriction) divided by the
  lumped coarse mass M_L (chi = 0 where the pressure is held, as b_c is).

Test device, not a scheme of the paper: ``exact_projection=True`` (levels = 0 only) keeps steps
1-5 and their code but solves Eq. 23 with the lumped mass M_L and replaces K_c in Eq. 21 by
E = -(Dx P_x M_L^-1 P_x Dx + Dy P_y M_L^-1 P_y Dy), where Dx, Dy give the correction's gradient
G p = (Dx p, Dy p) and P_x, P_y keep the velocity components that are not Dirichlet. E p =
-(rho/dt) D u~ is then exactly the condition D u^{n+1} = 0 on every row whose pressure is free,
so the discrete divergence of the corrected velocity vanishes there up to rounding: an invariant
against which the signs, factors and operator pairings of steps 2-5 are checked. Pressure nodes
none of whose velocity neighbours is free (no row of D P) are held at 0 as well. The paper's own
scheme (K_c, consistent M) does not have this property; equal-order P1 pairs can make E singular
on some meshes (spurious pressure modes), which the sparse LU then reports.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, refine


def _bc_rows(A: sp.csr_matrix, dirichlet: np.ndarray) -> sp.csc_matrix:
    """A with the rows of ``dirichlet`` nodes replaced by identity rows (non-symmetric)."""
    free = (~dirichlet).astype(np.float64)
    return (sp.diags(free) @ A + sp.diags(dirichlet.astype(np.float64))).tocsc()


def _bc_sym(A: sp.csr_matrix, dirichlet: np.ndarray) -> sp.csc_matrix:
    """A with rows and columns of ``dirichlet`` nodes zeroed and a unit diagonal (symmetric)."""
    free = sp.diags((~dirichlet).astype(np.float64))
    return (free @ A @ free + sp.diags(dirichlet.astype(np.float64))).tocsc()


@dataclass
class StepResult:
    u: np.ndarray        # end-of-step velocity u^{n+1}  [N_f, 2]
    ut: np.ndarray       # intermediate velocity u~      [N_f, 2]
    b_c: np.ndarray      # coarse Poisson right-hand side [N_c]
    p_c: np.ndarray      # coarse pressure               [N_c]
    p_f: np.ndarray      # prolonged pressure            [N_f]
    gp: np.ndarray       # M^{-1} G p_f                  [N_f, 2]


class _LumpedMass:
    """M_L^-1 applied by a division (the exact-projection test device)."""

    def __init__(self, ml: np.ndarray):
        self.ml = ml

    def solve(self, v: np.ndarray) -> np.ndarray:
        return v / self.ml


class CGPOracle:
    """The CGP method on one coarse mesh refined ``levels`` times (``levels = 0``: standard scheme)."""

    def __init__(self, coarse_xy, coarse_tri, rho, mu, dt, levels, vel_bc, p_bc, restrict_mode="injection",
                 projection="standard", exact_projection=False):
        if restrict_mode not in ("injection", "galerkin"):
            raise ValueError(restrict_mode)
        if projection not in ("standard", "incremental", "rotational"):
            raise ValueError(projection)
        self.restrict_mode, self.projection = restrict_mode, projection
        self.rho, self.mu, self.dt = float(rho), float(mu), float(dt)
        self.h = refine.build_hierarchy(coarse_xy, coarse_tri, levels)
        fine, coarse = self.h.fine, self.h.coarse
        self.fine = fem.P1Operators(fine.xy, fine.tri)
        self.coarse = fem.P1Operators(coarse.xy, coarse.tri)
        self.onb_f = refine.boundary_nodes(fine.tri, fine.xy.shape[0])
        self.onb_c = refine.boundary_nodes(coarse.tri, coarse.xy.shape[0])
        self.vel_bc = vel_bc
        self.p_mask = np.asarray(p_bc(coarse.xy, self.onb_c)).astype(bool)
        self.A0 = self.rho * self.fine.M + self.dt * self.mu * self.fine.K
        if exact_projection:
            if levels != 0:
                raise ValueError("the exact projection is defined for levels = 0")
            mask, _ = self.dirichlet(0.0)
            ml = np.asarray(self.fine.M.sum(axis=1)).ravel()
            E = sp.csr_matrix((self.fine.n, self.fine.n))
            reach = np.zeros(self.fine.n)
            for c, Dc in enumerate((self.fine.Dx, self.fine.Dy)):
                free = ((mask & (1 << c)) == 0).astype(np.float64)
                E = E - Dc @ sp.diags(free / ml) @ Dc
                reach += abs(Dc) @ free
            self.p_mask = self.p_mask | (reach == 0)
            self.Kc_lu = spla.splu(_bc_sym(E.tocsr(), self.p_mask))
            self.M_lu = _LumpedMass(ml)
            return
        self.Kc_lu = spla.splu(_bc_sym(self.coarse.K, self.p_mask))
        self.M_lu = spla.splu(self.fine.M.tocsc())

    @property
    def n_fine(self) -> int:
        return self.fine.n

    @property
    def n_coarse(self) -> int:
        return self.coarse.n

    def dirichlet(self, t):
        mask, g = self.vel_bc(self.fine.xy, self.onb_f, t)
        return np.asarray(mask, dtype=np.uint8), np.asarray(g, dtype=np.float64)

    # --- the five steps ------------------------------------------------------------------
    def pressure_gradient(self, p_c: np.ndarray) -> np.ndarray:
        """G_f P p_c: the fine gradient (G = D on V_f) of the prolonged coarse pressure, [N_f, 2]."""
        p_f = refine.prolong(self.h, p_c)
        return np.stack([self.fine.Dx @ p_f, self.fine.Dy @ p_f], axis=1)

    def momentum(self, u_n: np.ndarray, t_next: float, p_c_n: np.ndarray | None = None) -> np.ndarray:
        """Step 1, Eq. 19: the intermediate velocity u~^{n+1}. With ``p_c_n`` (incremental forms)
        the right-hand side also carries -dt G_f P p_c^n."""
        mask, g = self.dirichlet(t_next)
        A = self.A0 + (self.dt * self.rho) * self.fine.convection(u_n)
        rhs = self.rho * (self.fine.M @ u_n)
        if p_c_n is not None:
            rhs = rhs - self.dt * self.pressure_gradient(p_c_n)
        ut = np.empty_like(u_n)
        for c in range(2):
            d = (mask & (1 << c)) != 0
            b = np.where(d, g[:, c], rhs[:, c])
            ut[:, c] = spla.spsolve(_bc_rows(A, d), b)
        return ut

    def restrict_rhs(self, ut: np.ndarray) -> np.ndarray:
        """Steps 2-3 right-hand side: Eq. 20 then -(rho/dt) D_c u~_c with pressure BC rows zeroed;
        with restrict_mode "galerkin", -(rho/dt) P^T D_f u~_f instead."""
        if self.restrict_mode == "galerkin":
            div_f = self.fine.Dx @ ut[:, 0] + self.fine.Dy @ ut[:, 1]
            b = -(self.rho / self.dt) * refine.restrict_transpose(self.h, div_f)
        else:
            uc = refine.restrict(self.h, ut)
            b = -(self.rho / self.dt) * (self.coarse.Dx @ uc[:, 0] + self.coarse.Dy @ uc[:, 1])
        b[self.p_mask] = 0.0
        return b

    def pressure_update(self, p_c_n: np.ndarray, phi: np.ndarray, b_c: np.ndarray) -> np.ndarray:
        """Incremental forms: p^{n+1} = p^n + phi, and for the rotational form also - mu chi with
        chi = -(dt/rho) b_c / (lumped coarse mass): the restricted divergence of u~ that b_c was
        built from, as a nodal field (zero where the pressure is held)."""
        p = p_c_n + phi
        if self.projection == "rotational":
            chi = -(self.dt / self.rho) * b_c / np.asarray(self.coarse.M.sum(axis=1)).ravel()
            chi[self.p_mask] = 0.0
            p = p - self.mu * chi
        return p

    def poisson(self, b_c: np.ndarray) -> np.ndarray:
        """Step 3, Eq. 21 (exact solve)."""
        return self.Kc_lu.solve(b_c)

    def prolong_correct(self, p_c: np.ndarray, ut: np.ndarray, t_next: float):
        """Steps 4-5, Eqs. 22-23. Returns ``(u^{n+1}, p_f, gp)``."""
        p_f = refine.prolong(self.h, p_c)
        g = np.stack([self.fine.Dx @ p_f, self.fine.Dy @ p_f], axis=1)     # G p_f (G = D on V_f)
        w = np.stack([self.M_lu.solve(g[:, 0]), self.M_lu.solve(g[:, 1])], axis=1)
        u = ut - (self.dt / self.rho) * w
        mask, gd = self.dirichlet(t_next)
        for c in range(2):
            d = (mask & (1 << c)) != 0
            u[d, c] = gd[d, c]
        return u, p_f, w

    def step(self, u_n: np.ndarray, t_next: float, p_c_n: np.ndarray | None = None) -> StepResult:
        """One step. The incremental forms need the previous coarse pressure ``p_c_n`` (zero if
        omitted); StepResult.p_c is then the new pressure and p_f, gp belong to the increment."""
        if self.projection == "standard":
            ut = self.momentum(u_n, t_next)
            b_c = self.restrict_rhs(ut)
            p_c = self.poisson(b_c)
            u, p_f, gp = self.prolong_correct(p_c, ut, t_next)
            return StepResult(u, ut, b_c, p_c, p_f, gp)
        p_n = np.zeros(self.n_coarse) if p_c_n is None else np.asarray(p_c_n, dtype=np.float64)
        ut = self.momentum(u_n, t_next, p_n)
        b_c = self.restrict_rhs(ut)
        phi = self.poisson(b_c)
        u, p_f, gp = self.prolong_correct(phi, ut, t_next)
        return StepResult(u, ut, b_c, self.pressure_update(p_n, phi, b_c), p_f, gp)


def run(coarse, problem, n_steps: int, levels: int | None = None, u0=None, t0: float = 0.0,
        return_oracle: bool = False, restrict_mode: str = "injection", projection: str = "standard",
        p0=None):
    """Advance ``problem`` on the coarse mesh ``coarse`` (a ``cgp_inputs.CoarseMesh``) by ``n_steps``.

    Returns the last :class:`StepResult` (and the :class:`CGPOracle` if asked). The incremental
    forms start from the coarse pressure ``p0`` (zero if omitted).
    """
    lv = problem.levels if levels is None else levels
    orc = CGPOracle(coarse.xy, coarse.tri, problem.rho, problem.mu, problem.dt, lv,
                    problem.vel_bc, problem.p_bc, restrict_mode=restrict_mode, projection=projection)
    if u0 is None:
        mask, g = orc.dirichlet(t0)
        u = problem.u0(orc.fine.xy, mask, g)
    else:
        u = np.array(u0, dtype=np.float64)
    p = None if p0 is None else np.array(p0, dtype=np.float64)
    res = None
    for n in range(n_steps):
        res = orc.step(u, t0 + (n + 1) * problem.dt, p)
        u, p = res.u, res.p_c
    return (res, orc) if return_oracle else res
