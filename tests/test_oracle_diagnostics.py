"""Pins of the oracle's flow diagnostics (Sect. 3.2 reattachment length, Sect. 3.3 drag, lift and
Strouhal number), on the CPU.

* Pressure force of a linear pressure a + b x + c y on the closed cylinder body: by the divergence
  theorem over the body, -int p n_b = -(b, c) |body| (|body| from the mesh's missing area).
* Forces of constant fields on the open upper half of the body: a constant stress sigma gives
  sigma times the integrated normal of the polyline, (-(Q_y - P_y), Q_x - P_x) from its end points
  P (left) to Q (right); a linear velocity has a constant P1 gradient.
* Wall shear and reattachment on the backward-facing step's bottom wall for u = (y (x - 3.7), 0):
  the shear of every wall triangle is mu (x_top - 3.7), so the sign change lies at x = 3.7 to
  within a mesh width.
* Strouhal number of a sampled sine of known frequency.
"""
import math

import numpy as np

import cgp_inputs as ci
from oracle import cgp, diagnostics as dg


def _cylinder_oracle():
    coarse, prob = ci.cylinder_mesh(h_min=0.6), ci.cylinder_problem(100.0, 0.002, 1)
    orc = cgp.CGPOracle(coarse.xy, coarse.tri, prob.rho, prob.mu, prob.dt, 1, prob.vel_bc, prob.p_bc)
    xy = orc.fine.xy
    r = np.hypot(xy[:, 0] - 5.0, xy[:, 1] - 5.0)
    body = orc.onb_f & (r < 0.5 + 1e-9)
    return orc, body


def test_pressure_force_of_linear_pressure_on_closed_body():
    orc, body = _cylinder_oracle()
    xy = orc.fine.xy
    b, c = 0.7, -1.3
    p = 2.0 + b * xy[:, 0] + c * xy[:, 1]
    fp, fv = dg.body_force(xy, orc.fine.tri, np.zeros((orc.n_fine, 2)), p, 0.01, body)
    hole = 30.0 * 10.0 - orc.fine.area.sum()
    np.testing.assert_allclose(fp, [-b * hole, -c * hole], rtol=1e-11, atol=1e-13)
    assert np.all(fv == 0.0)


def test_constant_stress_on_open_half_body():
    orc, body = _cylinder_oracle()
    xy = orc.fine.xy
    half = body & (xy[:, 1] >= 5.0 - 1e-12)
    idx = np.nonzero(half)[0]
    P, Q = xy[idx[np.argmin(xy[idx, 0])]], xy[idx[np.argmax(xy[idx, 0])]]
    nsum = np.array([-(Q[1] - P[1]), Q[0] - P[0]])
    G = np.array([[0.3, -1.1], [0.8, 0.25]])           # u = G x + const, a linear field
    u = xy @ G.T + np.array([1.0, -2.0])
    mu, p0 = 0.01, 1.7
    fp, fv = dg.body_force(xy, orc.fine.tri, u, np.full(orc.n_fine, p0), mu, half)
    np.testing.assert_allclose(fp, -p0 * nsum, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(fv, mu * (G + G.T) @ nsum, rtol=1e-11, atol=1e-14)
    assert nsum[1] > 0.9    # the upper half's net normal points up, into the fluid


def test_reattachment_of_a_linear_shear():
    coarse, prob = ci.bfs_mesh(4, 1001), ci.bfs_problem(400.0, 0.005, 1)
    orc = cgp.CGPOracle(coarse.xy, coarse.tri, prob.rho, prob.mu, prob.dt, 1, prob.vel_bc, prob.p_bc)
    xy = orc.fine.xy
    wall = orc.onb_f & (np.abs(xy[:, 1]) < 1e-12) & (xy[:, 0] >= 1.0 - 1e-12)
    u = np.stack([xy[:, 1] * (xy[:, 0] - 3.7), np.zeros(orc.n_fine)], axis=1)
    xs, taus = dg.wall_shear(xy, orc.fine.tri, u, prob.mu, wall)
    assert np.all(np.diff(xs) > 0) and taus[0] < 0 < taus[-1]
    xr = dg.reattachment(xs, taus, 1.0)
    h = 1.0 / 8.0
    assert abs(xr - 3.7) < h, xr
    assert dg.reattachment(xs, -np.abs(taus), 1.0) is None


def test_strouhal_of_a_sine():
    t = np.arange(0.0, 200.0, 0.01)
    cl = 0.3 * np.sin(2.0 * math.pi * 0.21 * t + 0.4) + 0.05
    assert abs(dg.strouhal(t, cl) - 0.21) < 1e-5
