"""Convenience wrapper: one CGP context plus its device state, driven through the C ABI.

``Flow`` only marshals: it hands the coarse mesh to ``cgp_mesh_create``, evaluates the problem's
boundary description on the fine nodes the library returns, uploads it with ``cgp_set_bc`` and
keeps the velocity and coarse pressure as torch device tensors. Every arithmetic step of the
method runs in the CUDA library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import cgp as L


class Flow:
    """A problem on a coarse mesh (``coarse.xy``, ``coarse.tri``), advanced by ``cgp_step``.

    ``problem`` provides ``rho, mu, dt, levels, vel_bc(xy, onb, t), p_bc(xy, onb), u0(xy, mask, g)``.
    """

    def __init__(self, coarse, problem, precision: int = L.CGP_FP64, rtol: float = 1e-8, levels=None,
                 device: str = "cuda:0", autotune: bool = False, **params):
        self.problem = problem
        self.device = torch.device(device)
        torch.cuda.set_device(self.device)
        lv = problem.levels if levels is None else levels
        prm = L.default_params(rho=problem.rho, mu=problem.mu, dt=problem.dt, levels=lv, precision=precision,
                               rtol=rtol, **params)
        self.params = prm
        self.ctx = L.cgp_mesh_create(coarse.xy, coarse.tri, prm)
        self.info = L.cgp_mesh_info(self.ctx)
        self.fine_xy, self.fine_tri, self.onb_f = L.cgp_fine_mesh(self.ctx)
        self.coarse_xy = np.asarray(coarse.xy, dtype=np.float64)
        self.onb_c = self.onb_f[: self.info.n_coarse]      # parents keep their numbers (Eq. 30)
        self.t = 0.0
        mask, g = problem.vel_bc(self.fine_xy, self.onb_f, 0.0)
        self.vel_mask = np.asarray(mask, dtype=np.uint8)
        self.p_mask = np.asarray(problem.p_bc(self.coarse_xy, self.onb_c), dtype=np.uint8)
        L.cgp_set_bc(self.ctx, self.vel_mask, self.p_mask, np.asarray(g, dtype=np.float64))
        self.g_dev = torch.tensor(np.asarray(g), dtype=torch.float64, device=self.device)
        u0 = problem.u0(self.fine_xy, self.vel_mask, g)
        self.u = torch.tensor(np.ascontiguousarray(u0), dtype=torch.float64, device=self.device)
        self.pc = torch.zeros(self.info.n_coarse, dtype=torch.float64, device=self.device)
        if autotune:
            L.cgp_autotune(self.ctx)
        self.info = L.cgp_mesh_info(self.ctx)

    def set_time(self, t_next: float, stream=None) -> None:
        """Upload boundary values at ``t_next`` (only for time-dependent boundary data)."""
        if getattr(self.problem, "time_dependent_bc", False):
            _, g = self.problem.vel_bc(self.fine_xy, self.onb_f, t_next)
            self.g_dev.copy_(torch.from_numpy(np.ascontiguousarray(g)))
            L.cgp_set_dirichlet_values(self.ctx, self.g_dev, stream)

    def step(self, n: int = 1, stream=None) -> None:
        for _ in range(n):
            self.set_time(self.t + self.problem.dt, stream)
            L.cgp_step(self.ctx, self.u, self.pc, stream)
            self.t += self.problem.dt

    def stats(self, check: bool = True):
        return L.cgp_get_stats(self.ctx, None, check=check)

    def close(self) -> None:
        if self.ctx:
            L.cgp_mesh_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several ``Flow`` instances advanced together by ``cgp_batch_step`` / ``cgp_batch_run``.

    The flows keep their own state tensors; the batch only records their pointers, so the flows
    must outlive it."""

    def __init__(self, flows):
        self.flows = list(flows)
        self.handle = L.cgp_batch_create([f.ctx for f in self.flows], [f.u for f in self.flows],
                                         [f.pc for f in self.flows])
        self.blocks, self.group_fine, self.group_coarse = L.cgp_batch_info(self.handle, len(self.flows))

    def step(self, n: int = 1, stream=None) -> None:
        for _ in range(n):
            L.cgp_batch_step(self.handle, stream)
        for f in self.flows:
            f.t += n * f.problem.dt

    def run(self, n: int, stream=None) -> None:
        """``n`` steps by replaying the captured CUDA graph of one step."""
        L.cgp_batch_run(self.handle, n, stream)
        for f in self.flows:
            f.t += n * f.problem.dt

    def stats(self, check: bool = True):
        return L.cgp_batch_get_stats(self.handle, len(self.flows), None, check=check)[0]

    def close(self) -> None:
        if self.handle:
            L.cgp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
