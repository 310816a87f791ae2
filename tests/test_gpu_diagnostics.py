"""GPU diagnostics against the oracle's (Sect. 3.2 reattachment length, Sect. 3.3 drag and lift),
through the C ABI, on states the GPU path produced: the same u and p_c go to both sides.

* Cylinder (l = 2, graded Delaunay mesh): pressure and viscous force on the cylinder after 40
  steps, relative error 1e-12; the drag coefficient of the impulsively started flow is positive.
* Backward-facing step (small mesh): wall shear of every bottom-wall edge and the reattachment
  point after 100 steps, 1e-12.
"""
import os

import numpy as np
import pytest
import torch

import cgp_inputs as ci
from oracle import diagnostics as dg, refine

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_06993_gb300 import cgp
    if not os.path.exists(cgp.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    cgp.load()
    return cgp


def test_body_force_matches_oracle(L):
    from paper_1610_06993_gb300.flow import Flow
    coarse, prob, _ = ci.workload("cylinder_small")
    f = Flow(coarse, prob, rtol=1e-10)
    r = np.hypot(f.fine_xy[:, 0] - 5.0, f.fine_xy[:, 1] - 5.0)
    body = f.onb_f & (r < 0.5 + 1e-9)
    assert L.cgp_set_surface(f.ctx, 0, body) > 20
    f.step(40)
    f.stats(check=True)
    force = torch.zeros(4, dtype=torch.float64, device="cuda")
    L.cgp_body_force(f.ctx, f.u, f.pc, force)
    got = force.cpu().numpy()
    u, pc = f.u.cpu().numpy(), f.pc.cpu().numpy()
    h = refine.build_hierarchy(coarse.xy, coarse.tri, prob.levels)
    fp, fv = dg.body_force(f.fine_xy, f.fine_tri.astype(np.int64), u, refine.prolong(h, pc), prob.mu, body)
    ref = np.concatenate([fp, fv])
    f.close()
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref), (got, ref)
    assert got[0] + got[2] > 0.0     # drag along the inflow


def test_reattachment_matches_oracle(L):
    from paper_1610_06993_gb300.flow import Flow
    coarse, prob = ci.bfs_mesh(4, 1001), ci.bfs_problem(400.0, 0.005, 1)
    f = Flow(coarse, prob, rtol=1e-10)
    xy = f.fine_xy
    wall = f.onb_f & (np.abs(xy[:, 1]) < 1e-12) & (xy[:, 0] >= 1.0 - 1e-12)
    ne = L.cgp_set_surface(f.ctx, 1, wall)
    f.step(100)
    f.stats(check=True)
    xr = torch.zeros(1, dtype=torch.float64, device="cuda")
    xs = torch.empty(ne, dtype=torch.float64, device="cuda")
    tau = torch.empty(ne, dtype=torch.float64, device="cuda")
    L.cgp_reattachment(f.ctx, f.u, 1.0, xr, xs, tau)
    u = f.u.cpu().numpy()
    rx, rt = dg.wall_shear(xy, f.fine_tri.astype(np.int64), u, prob.mu, wall)
    f.close()
    assert np.array_equal(xs.cpu().numpy(), rx)
    assert np.linalg.norm(tau.cpu().numpy() - rt) <= 1e-12 * np.linalg.norm(rt)
    ref = dg.reattachment(rx, rt, 1.0)
    assert ref is not None and abs(float(xr.item()) - ref) <= 1e-12 * abs(ref), (float(xr.item()), ref)
