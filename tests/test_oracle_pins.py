"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these tests compares the oracle with itself: each checks a hand-integrated value, a
closed-form solution, an invariant of the continuous operators, a brute-force recomputation by
quadrature and point location on a tiny mesh, or a convergence rate the paper states.
"""
import math
import os

import numpy as np
import pytest

import cgp_inputs as ci
from oracle import cgp, fem, refine

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------------------
# Element matrices (Eqs. 16-18)
# ----------------------------------------------------------------------------------------

def _load_reference_triangle():
    mats = {}
    with open(os.path.join(GOLDEN, "p1_reference_triangle.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, i, j, num, den = line.split()
            mats.setdefault(name, np.zeros((3, 3)))[int(i), int(j)] = int(num) / int(den)
    return mats


def test_element_matrices_reference_triangle():
    """Hand-integrated element matrices on the right triangle (0,0),(1,0),(0,1)."""
    gold = _load_reference_triangle()
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    tri = np.array([[0, 1, 2]])
    area, gx, gy = fem.triangle_geometry(xy, tri)
    assert area[0] == 0.5
    np.testing.assert_allclose(fem.element_mass(area)[0], gold["M"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(fem.element_stiffness(area, gx, gy)[0], gold["K"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(fem.element_div(area, gx)[0], gold["Dx"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(fem.element_div(area, gy)[0], gold["Dy"], rtol=0, atol=1e-15)
    u_el = np.array([[[0.0, 0.0], [1.0, 0.0], [0.0, 0.0]]])          # u = (x, 0)
    np.testing.assert_allclose(fem.element_convection(area, gx, gy, u_el)[0], gold["Nx"], rtol=0, atol=1e-15)


@pytest.fixture(scope="module")
def jmesh():
    m = ci.cavity_mesh(17, 77)
    return fem.P1Operators(m.xy, m.tri), refine.boundary_nodes(m.tri.astype(np.int64), m.n_nodes)


def test_mass_sums_to_area(jmesh):
    ops, _ = jmesh
    assert abs(ops.M.sum() - 1.0) < 1e-13           # sum phi_i = 1 on the unit square


@pytest.mark.parametrize("mesh", [ci.cavity_mesh(17, 77), ci.bfs_mesh(5, 3), ci.cylinder_mesh(h_min=0.6)],
                         ids=["cavity", "bfs", "cylinder"])
def test_jacobi_scaled_mass_spectrum(mesh):
    """The spectrum of D^-1 M (D = diag M) lies in [1/2, 2] for P1 triangles on any mesh: every
    element matrix D_e^-1 M_e has the eigenvalues 1/2, 1/2, 2, and assembly keeps the Rayleigh
    quotient between the elementwise extremes. The mass-solve polynomial preconditioner is built
    on exactly these bounds, so they are checked here by a dense eigensolve, on a jittered
    uniform, a structured and a graded mesh."""
    ops = fem.P1Operators(mesh.xy, mesh.tri)
    M = ops.M.toarray()
    d = 1.0 / np.sqrt(np.diag(M))
    lam = np.linalg.eigvalsh(d[:, None] * M * d[None, :])
    assert lam.min() >= 0.5 - 1e-12 and lam.max() <= 2.0 + 1e-12, (lam.min(), lam.max())
    area = fem.triangle_geometry(mesh.xy, mesh.tri)[0]
    me = fem.element_mass(area)[0]
    de = np.diag(1.0 / np.diag(me))
    np.testing.assert_allclose(np.sort(np.linalg.eigvals(de @ me).real), [0.5, 0.5, 2.0], rtol=0, atol=1e-14)


def _kovasznay(xy, re):
    """Kovasznay's closed-form steady Navier-Stokes flow (rho = 1, mu = 1/Re): u = 1 - e^(lx)
    cos(2 pi y), v = l/(2 pi) e^(lx) sin(2 pi y), p = (1 - e^(2lx))/2, l = Re/2 - sqrt(Re^2/4 + 4 pi^2)."""
    lam = re / 2 - math.sqrt(re * re / 4 + 4 * math.pi ** 2)
    x, y = xy[:, 0], xy[:, 1]
    e = np.exp(lam * x)
    u = np.stack([1 - e * np.cos(2 * np.pi * y), lam / (2 * np.pi) * e * np.sin(2 * np.pi * y)], axis=1)
    return u, 0.5 * (1 - np.exp(2 * lam * x))


def test_kovasznay_steady_residual_converges():
    """The nodal interpolants of Kovasznay's exact steady flow (Re = 40 on [-1/2, 1] x [-1/2, 3/2],
    jittered meshes, h = 1/8, 1/16, 1/32) nearly satisfy the discrete steady momentum equations
    N(u) u + mu K u + G p = 0 at interior nodes (the convection, stiffness and gradient matrices of
    Eqs. 16-18 and 23): the residual in the discrete H^-1 norm (R^T K_0^-1 R, K_0 the interior
    stiffness) falls at better than first order, and the weak divergence D u at first order. A
    wrong sign or factor in N, a missing viscous term or swapped gradient components leave an O(1)
    residual that does not fall."""
    import scipy.sparse.linalg as spla
    re = 40.0
    res, div = [], []
    for k in (4, 8, 16):
        m = ci.jittered_grid(-0.5, 1.0, -0.5, 1.5, 3 * k, 4 * k, 50 + k)
        ops = fem.P1Operators(m.xy, m.tri)
        onb = refine.boundary_nodes(m.tri.astype(np.int64), m.n_nodes)
        u, p = _kovasznay(ops.xy, re)
        R = ops.convection(u) @ u + (1.0 / re) * (ops.K @ u) + np.stack([ops.Dx @ p, ops.Dy @ p], axis=1)
        inner = ~onb
        z = spla.spsolve(ops.K[inner][:, inner].tocsc(), R[inner])
        res.append(math.sqrt(float(np.sum(R[inner] * z))))
        d = ops.Dx @ u[:, 0] + ops.Dy @ u[:, 1]
        lumped = np.asarray(ops.M.sum(axis=1)).ravel()
        div.append(math.sqrt(float(np.sum(d * d / lumped))))
    rate_res = [math.log2(res[i] / res[i + 1]) for i in range(2)]
    rate_div = [math.log2(div[i] / div[i + 1]) for i in range(2)]
    assert min(rate_res) > 1.3 and res[-1] < 1e-2, (res, rate_res)
    assert min(rate_div) > 0.8, (div, rate_div)


def test_stiffness_annihilates_linear_fields(jmesh):
    ops, onb = jmesh
    x, y = ops.xy[:, 0], ops.xy[:, 1]
    assert np.abs(ops.K @ np.ones(ops.n)).max() < 1e-12
    r = ops.K @ (2.0 * x - 3.0 * y + 1.0)
    assert np.abs(r[~onb]).max() < 1e-12            # -Laplacian of a linear field vanishes inside


def test_divergence_of_coordinate_fields(jmesh):
    """int phi_i d_x x = int phi_i = lumped mass; d_x y = 0."""
    ops, _ = jmesh
    x, y = ops.xy[:, 0], ops.xy[:, 1]
    lumped = np.asarray(ops.M.sum(axis=1)).ravel()
    np.testing.assert_allclose(ops.Dx @ x, lumped, rtol=0, atol=1e-15)
    np.testing.assert_allclose(ops.Dy @ y, lumped, rtol=0, atol=1e-15)
    assert np.abs(ops.Dx @ y).max() < 1e-15 and np.abs(ops.Dy @ x).max() < 1e-15


def test_convection_constant_velocity(jmesh):
    """N(c) f = (c . grad f) int phi_i for constant c and linear f; N annihilates constants."""
    ops, _ = jmesh
    x, y = ops.xy[:, 0], ops.xy[:, 1]
    c = np.array([0.7, -1.3])
    N = ops.convection(np.tile(c, (ops.n, 1)))
    lumped = np.asarray(ops.M.sum(axis=1)).ravel()
    f = 2.0 * x + 5.0 * y
    np.testing.assert_allclose(N @ f, (c[0] * 2.0 + c[1] * 5.0) * lumped, rtol=0, atol=1e-14)
    assert np.abs(N @ np.ones(ops.n)).max() < 1e-14


def test_convection_skew_for_divergence_free_velocity(jmesh):
    """For div u = 0: N_ij + N_ji = boundary integral only, so it vanishes if i or j is interior."""
    ops, onb = jmesh
    x, y = ops.xy[:, 0], ops.xy[:, 1]
    u = np.stack([0.3 + 2.0 * y, 1.1 - 0.5 * x], axis=1)             # linear, divergence-free
    N = ops.convection(u).toarray()
    S = N + N.T
    inner = ~onb
    assert np.abs(S[inner, :]).max() < 1e-14
    assert np.abs(S[:, inner]).max() < 1e-14
    assert np.abs(N[inner][:, inner]).max() > 1e-3                  # N itself is not zero


def test_poisson_second_order_convergence():
    """-Lap p = f with p = cos(pi x) cos(pi y), natural BC, P1 error O(h^2) (slope >= 1.85)."""
    errs, hs = [], []
    for n in (9, 17, 33, 65):
        m = ci.cavity_mesh(n, 5)
        ops = fem.P1Operators(m.xy, m.tri)
        x, y = ops.xy[:, 0], ops.xy[:, 1]
        pe = np.cos(np.pi * x) * np.cos(np.pi * y)
        f = 2.0 * np.pi ** 2 * pe
        K = ops.K.tolil()
        b = ops.M @ f
        b -= K[:, 0].toarray().ravel() * pe[0]
        K[0, :] = 0.0
        K[:, 0] = 0.0
        K[0, 0] = 1.0
        b[0] = pe[0]
        import scipy.sparse.linalg as spla
        p = spla.spsolve(K.tocsc(), b)
        e = p - pe
        e -= (ops.M @ e).sum() / ops.M.sum()                         # compare modulo a constant
        errs.append(math.sqrt(e @ (ops.M @ e)))
        hs.append(1.0 / (n - 1))
    slopes = np.diff(np.log(errs)) / np.diff(np.log(hs))
    assert (slopes > 1.85).all(), slopes


def test_poisson_patch_test():
    """A linear pressure with Dirichlet data on the whole boundary is reproduced exactly."""
    m = ci.cavity_mesh(9, 3)
    ops = fem.P1Operators(m.xy, m.tri)
    onb = refine.boundary_nodes(m.tri.astype(np.int64), m.n_nodes)
    pl = 1.5 * ops.xy[:, 0] - 0.25 * ops.xy[:, 1] + 3.0
    K = ops.K.toarray()
    free = ~onb
    p = pl.copy()
    p[free] = np.linalg.solve(K[np.ix_(free, free)], -K[np.ix_(free, onb)] @ pl[onb])
    np.testing.assert_allclose(p, pl, rtol=0, atol=1e-13)


# ----------------------------------------------------------------------------------------
# Refinement and mapping (Sect. 2.2, Remark 2.2, Eqs. 29-30)
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("mesh", [ci.cavity_mesh(9, 11), ci.bfs_mesh(3, 12)], ids=["cavity", "bfs"])
@pytest.mark.parametrize("levels", [1, 2, 3])
def test_refinement_topology(mesh, levels):
    h = refine.build_hierarchy(mesh.xy, mesh.tri, levels)
    for k in range(levels):
        c, f = h.levels[k], h.levels[k + 1]
        ec, _ = refine.edges_first_visit(c.tri, c.xy.shape[0])
        ef, eof = refine.edges_first_visit(f.tri, f.xy.shape[0])
        assert f.tri.shape[0] == 4 * c.tri.shape[0]                   # N = 4^{-l} M (Sect. 2.2)
        assert f.xy.shape[0] == c.xy.shape[0] + ec.shape[0]
        assert f.xy.shape[0] - ef.shape[0] + f.tri.shape[0] == 1      # Euler, simply connected
        cnt = np.bincount(eof.ravel())
        assert cnt.max() == 2                                         # conforming
        area_c, _, _ = fem.triangle_geometry(c.xy, c.tri)
        area_f, _, _ = fem.triangle_geometry(f.xy, f.tri)
        assert area_f.min() > 0                                       # children counter-clockwise
        assert abs(area_f.sum() - area_c.sum()) < 1e-12 * area_c.sum()
        np.testing.assert_allclose(area_f.reshape(-1, 4).sum(1), area_c, rtol=1e-13)


def load_mapping_loop_counts():
    """The mapping-operator loop counts the paper gives for l = 3 (tests/golden)."""
    with open(os.path.join(GOLDEN, "mapping_loop_counts_bfs_l3.txt")) as f:
        return {k: int(v) for k, v in (ln.split() for ln in f if ln.strip() and not ln.startswith("#"))}


def mapping_loop_mesh():
    """A simply connected coarse mesh of the quoted size: a 100 x 4-cell jittered channel (505
    nodes, 800 triangles, 208 boundary nodes) with 400 triangles split at their centroids, 905
    nodes and 1,600 triangles. The paper's grid is not available; the counts do not depend on it."""
    return ci.centroid_split(ci.jittered_grid(0.0, 25.0, 0.0, 1.0, 100, 4, 1005), 400)


def test_mapping_loop_counts_of_the_paper():
    """Sect. 3.2, with Table 5: for l = 3 on a simply connected grid of 1,600 coarse and 102,400
    fine elements the injection (Eqs. 20, 30) runs over the 905 coarse pressure nodes and the
    prolongation (Eqs. 22, 29) over the 68,659 nodes of levels 1-3. A refinement that created a
    midpoint per triangle side instead of per edge, or lost one, would miss both fine counts."""
    g = load_mapping_loop_counts()
    m = mapping_loop_mesh()
    assert m.n_nodes == g["restriction_loops"] and m.n_tris == g["coarse_elements"]
    h = refine.build_hierarchy(m.xy, m.tri, g["levels"])
    assert len(h.fine.tri) == g["fine_elements"]
    assert len(h.su) == g["restriction_loops"]
    assert sum(len(sp) for sp in h.sp) == g["prolongation_loops"]
    assert [len(lv.xy) for lv in h.levels[1:]] == [3409, 13217, 52033]


def load_nested_mesh_counts():
    """Per case, the (nodes, elements) of each level the paper gives (tests/golden)."""
    out = {}
    with open(os.path.join(GOLDEN, "nested_mesh_counts.txt")) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                case, level, nodes, elems = ln.split()
                out.setdefault(case, []).append((int(nodes), int(elems)))
    return out


def holed_mesh_of_size(n_nodes, n_tris, n, k):
    """A mesh with one hole and the given counts: an n x n-cell jittered square with a centred
    k x k-cell hole (boundary nodes 4 n + 4 k = 2 n_nodes - n_tris by Euler's formula) and as many
    centroid splits as the remaining nodes. The paper's meshes are not available; the counts of the
    refined levels depend only on these."""
    c0 = (n - k) // 2
    m = ci.jittered_grid(0.0, 1.0, 0.0, 1.0, n, n, 1006,
                         removed_cell=lambda i, j: (i >= c0) & (i < c0 + k) & (j >= c0) & (j < c0 + k))
    assert 4 * n + 4 * k == 2 * n_nodes - n_tris
    return ci.centroid_split(m, n_nodes - m.n_nodes)


NESTED_GRIDS = {"taylor_green": (40, 16), "cylinder": (30, 2)}


@pytest.mark.parametrize("case", sorted(NESTED_GRIDS))
def test_nested_mesh_counts_of_the_paper(case):
    """The node and element counts the paper prints for its nested Taylor-Green (Sect. 3.1, Fig. 2,
    Table 1) and cylinder (Sect. 3.3) meshes follow from the coarsest level by the refinement of
    Sect. 2.2 on a domain with one hole: the oracle reproduces each level from a mesh of the
    coarsest level's size."""
    levels = load_nested_mesh_counts()[case]
    m = holed_mesh_of_size(*levels[0], *NESTED_GRIDS[case])
    assert (m.n_nodes, m.n_tris) == levels[0]
    h = refine.build_hierarchy(m.xy, m.tri, len(levels) - 1)
    for lv, (nodes, elems) in zip(h.levels, levels):
        assert len(lv.tri) == elems
        assert nodes < 0 or len(lv.xy) == nodes


def test_restrict_prolong_identity_and_linear_exactness():
    m = ci.cavity_mesh(9, 13)
    h = refine.build_hierarchy(m.xy, m.tri, 3)
    rng = np.random.default_rng(0)
    pc = rng.standard_normal(m.n_nodes)
    assert np.array_equal(refine.restrict(h, refine.prolong(h, pc)), pc)      # R P = I bitwise
    lin = lambda xy: 3.0 * xy[:, 0] - 2.0 * xy[:, 1] + 0.5
    np.testing.assert_allclose(refine.prolong(h, lin(h.coarse.xy)), lin(h.fine.xy), rtol=0, atol=1e-14)
    # work counts of Remark 2.2: O(N_c) for R, sum of N_{k+1} for P
    assert h.su.shape[0] == m.n_nodes
    assert sum(s.shape[0] for s in h.sp) == sum(l.xy.shape[0] for l in h.levels[1:])


def _shape_coeffs(p):
    """Coefficients C so that [1, x, y] @ C[:, i] = phi_i, by inverting the vertex system."""
    V = np.column_stack([np.ones(3), p[:, 0], p[:, 1]])
    return np.linalg.inv(V), 0.5 * np.linalg.det(V)


def _interp_matrix(coarse_xy, coarse_tri, pts):
    """Dense P1 interpolation from the coarse mesh to ``pts`` by brute-force point location."""
    P = np.zeros((pts.shape[0], coarse_xy.shape[0]))
    for a, q in enumerate(pts):
        for t in coarse_tri:
            C, _ = _shape_coeffs(coarse_xy[t])
            lam = np.array([1.0, q[0], q[1]]) @ C
            if lam.min() > -1e-12:
                P[a, t] = lam
                break
        else:
            raise AssertionError("point outside mesh")
    return P


def test_prolongation_table_equals_coarse_interpolation():
    """Eq. 29's midpoint average equals evaluating the coarse shape functions psi (nested spaces)."""
    m = ci.cavity_mesh(5, 21)
    h = refine.build_hierarchy(m.xy, m.tri, 2)
    P = _interp_matrix(m.xy, m.tri.astype(np.int64), h.fine.xy)
    pc = np.random.default_rng(1).standard_normal(m.n_nodes)
    np.testing.assert_allclose(refine.prolong(h, pc), P @ pc, rtol=0, atol=1e-13)


# ----------------------------------------------------------------------------------------
# The whole step against a brute-force dense recomputation (Eqs. 19-23)
# ----------------------------------------------------------------------------------------

def _dense_ops(xy, tri, u=None):
    """Dense M, K, Dx, Dy (and N(u)) by 3-point edge-midpoint quadrature (exact to degree 2)."""
    n = xy.shape[0]
    M, K, Dx, Dy, N = (np.zeros((n, n)) for _ in range(5))
    for t in tri:
        p = xy[t]
        C, area = _shape_coeffs(p)
        grad = C[1:, :]                                              # [2, 3]: d/dx, d/dy of phi_i
        qs = 0.5 * (p + p[[1, 2, 0]])
        for q in qs:
            phi = np.array([1.0, q[0], q[1]]) @ C
            w = area / 3.0
            M[np.ix_(t, t)] += w * np.outer(phi, phi)
            Dx[np.ix_(t, t)] += w * np.outer(phi, grad[0])
            Dy[np.ix_(t, t)] += w * np.outer(phi, grad[1])
            if u is not None:
                uq = phi @ u[t]
                N[np.ix_(t, t)] += w * np.outer(phi, uq @ grad)
        K[np.ix_(t, t)] += area * grad.T @ grad
    return M, K, Dx, Dy, N


def _dense_cgp_step(prob, coarse, fine_xy, fine_tri, onb_f, onb_c, u_n, t_next):
    rho, mu, dt = prob.rho, prob.mu, prob.dt
    M, K, Dx, Dy, N = _dense_ops(fine_xy, fine_tri, u_n)
    _, Kc, Dxc, Dyc, _ = _dense_ops(coarse.xy, coarse.tri.astype(np.int64))
    # restriction by matching coordinates, prolongation by coarse interpolation
    R = np.zeros((coarse.n_nodes, fine_xy.shape[0]))
    for eta, q in enumerate(coarse.xy):
        R[eta, np.flatnonzero((fine_xy == q).all(axis=1))[0]] = 1.0
    P = _interp_matrix(coarse.xy, coarse.tri.astype(np.int64), fine_xy)
    mask, g = prob.vel_bc(fine_xy, onb_f, t_next)
    A = rho * M + dt * (rho * N + mu * K)
    b = rho * M @ u_n
    ut = np.zeros_like(u_n)
    for c in range(2):
        d = (mask & (1 << c)) != 0
        Ac, bc = A.copy(), b[:, c].copy()
        Ac[d, :] = 0.0
        Ac[d, d] = 1.0
        bc[d] = g[d, c]
        ut[:, c] = np.linalg.solve(Ac, bc)
    uc = R @ ut
    bcoarse = -(rho / dt) * (Dxc @ uc[:, 0] + Dyc @ uc[:, 1])
    pm = prob.p_bc(coarse.xy, onb_c).astype(bool)
    Kb = Kc.copy()
    Kb[pm, :] = 0.0
    Kb[:, pm] = 0.0
    Kb[pm, pm] = 1.0
    bcoarse[pm] = 0.0
    pc = np.linalg.solve(Kb, bcoarse)
    pf = P @ pc
    w = np.linalg.solve(M, np.stack([Dx @ pf, Dy @ pf], 1))
    u = ut - dt / rho * w
    for c in range(2):
        d = (mask & (1 << c)) != 0
        u[d, c] = g[d, c]
    return dict(ut=ut, b_c=bcoarse, p_c=pc, p_f=pf, gp=w, u=u)


EXACT_CASES = {
    # seeded meshes on which the exact-projection matrix E has no spurious pressure mode
    "cavity17": lambda: (ci.cavity_mesh(17, 3), ci.cavity_problem(100.0, 0.01, 0)),
    "taylor_green9": lambda: (ci.cavity_mesh(9, 3), ci.taylor_green_problem(0.01, 0.01, 0)),
    "bfs4": lambda: (ci.bfs_mesh(4, 1001), ci.bfs_problem(400.0, 0.005, 0)),
}


def exact_projection_divergence(case, exact, rho=2.5):
    """||D u^{n+1}|| / ||D u~|| on the rows of free pressure after one oracle step at l = 0 from
    a perturbed initial field, with or without the exact-projection test device."""
    coarse, prob = EXACT_CASES[case]()
    kw = dict(exact_projection=True) if exact else {}
    orc = cgp.CGPOracle(coarse.xy, coarse.tri, rho, prob.mu, prob.dt, 0, prob.vel_bc, prob.p_bc, **kw)
    mask, g = orc.dirichlet(prob.dt)
    u_n = prob.u0(orc.fine.xy, mask, g) + 0.1 * np.random.default_rng(7).standard_normal((orc.n_fine, 2))
    r = orc.step(u_n, prob.dt)
    free = ~orc.p_mask

    def div(v):
        return orc.fine.Dx @ v[:, 0] + orc.fine.Dy @ v[:, 1]
    return np.linalg.norm(div(r.u)[free]) / np.linalg.norm(div(r.ut)[free])


@pytest.mark.parametrize("case", sorted(EXACT_CASES))
def test_exact_projection_leaves_no_discrete_divergence(case):
    """Steps 2-5 (Eqs. 20-23) run with the exact-projection test device at l = 0 (lumped mass in
    the correction, and as Poisson matrix E = -D P M_L^-1 P G from the correction's own gradient)
    leave a velocity that is discretely divergence-free on every row of free pressure:
    ||D u^{n+1}|| <= 1e-10 ||D u~||. A wrong sign or factor (rho/dt) in the coarse right-hand side
    or the correction, swapped gradient components, or a Dirichlet reset at other nodes than the
    ones E leaves out would keep a divergence of the order of D u~. The paper's scheme itself
    (stiffness K_c, consistent M) keeps a large part of it."""
    assert exact_projection_divergence(case, True) <= 1e-10
    assert exact_projection_divergence(case, False) > 1e-3


def test_exact_projection_needs_levels_zero():
    coarse, prob = EXACT_CASES["cavity17"]()
    with pytest.raises(ValueError):
        cgp.CGPOracle(coarse.xy, coarse.tri, 1.0, prob.mu, prob.dt, 1, prob.vel_bc, prob.p_bc, exact_projection=True)


@pytest.mark.parametrize("case,levels", [("cavity", 1), ("cavity", 0), ("tg", 2), ("bfs", 1)])
def test_step_matches_bruteforce_dense(case, levels):
    if case == "cavity":
        coarse, prob = ci.cavity_mesh(5, 31), ci.cavity_problem(100.0, 0.01, levels)
    elif case == "tg":
        coarse, prob = ci.cavity_mesh(4, 32), ci.taylor_green_problem(0.01, 0.01, levels)
    else:
        coarse, prob = ci.bfs_mesh(2, 33), ci.bfs_problem(400.0, 0.005, levels)
    orc = cgp.CGPOracle(coarse.xy, coarse.tri, prob.rho, prob.mu, prob.dt, levels, prob.vel_bc, prob.p_bc)
    rng = np.random.default_rng(7)
    u_n = 0.5 * rng.standard_normal((orc.n_fine, 2))                # exercise N with a rough field
    t_next = 0.37
    got = orc.step(u_n, t_next)
    ref = _dense_cgp_step(prob, coarse, orc.fine.xy, orc.fine.tri, orc.onb_f, orc.onb_c, u_n, t_next)
    for k, v in ref.items():
        a = getattr(got, k)
        err = np.linalg.norm(a - v) / max(np.linalg.norm(v), 1e-300)
        assert err < 1e-11, (k, err)


def test_enclosed_flow_rhs_is_compatible():
    """sum_i (D u~)_i = closed-contour integral of u~ . n = 0 for the cavity (tangential lid)."""
    coarse, prob = ci.workload("cavity33")[:2]
    res, orc = cgp.run(coarse, prob, 3, return_oracle=True)
    uc = refine.restrict(orc.h, res.ut)
    d = orc.coarse.Dx @ uc[:, 0] + orc.coarse.Dy @ uc[:, 1]
    assert abs(d.sum()) < 1e-13 * np.abs(d).sum()


# ----------------------------------------------------------------------------------------
# Taylor-Green (Eqs. 34-36): first order in time, and CGP close to the standard scheme
# ----------------------------------------------------------------------------------------

def _tg_error(coarse, dt, t_end, levels):
    prob = ci.taylor_green_problem(0.01, dt, levels)
    n = int(round(t_end / dt))
    res, orc = cgp.run(coarse, prob, n, return_oracle=True)
    ue = ci.taylor_green_velocity(orc.fine.xy, n * dt, 0.01)
    return np.linalg.norm(res.u - ue) / np.linalg.norm(ue), res, orc


@pytest.mark.parametrize("levels", [1, 2])
def test_projection_removes_gradient_fields(levels):
    """Steps 2-5 (Eqs. 20-23) applied to a pure gradient field u~ = grad(cos(pi x) cos(pi y)) on the
    unit square (zero normal flux): the continuous projection returns u = 0. The method's discrete
    projection - injection, coarse Poisson with the Laplacian, prolongation, gradient and mass
    solve - leaves a remainder at interior nodes that falls at first order in h (the coarse P1
    pressure gradient). This is the property the approximate projection does have; its discrete
    divergence is not zero, since Eq. 21 solves with the Laplacian rather than D M^-1 G."""
    out = []
    for n in (9, 17, 33):
        coarse = ci.cavity_mesh(n, 7)
        prob = ci.cavity_problem(100.0, 0.01, levels)
        orc = cgp.CGPOracle(coarse.xy, coarse.tri, prob.rho, prob.mu, prob.dt, levels, prob.vel_bc, prob.p_bc)
        x, y = orc.fine.xy[:, 0], orc.fine.xy[:, 1]
        ut = np.stack([-math.pi * np.sin(math.pi * x) * np.cos(math.pi * y),
                       -math.pi * np.cos(math.pi * x) * np.sin(math.pi * y)], axis=1)
        pc = orc.poisson(orc.restrict_rhs(ut))
        u, _, _ = orc.prolong_correct(pc, ut, 0.01)
        inner = ~orc.onb_f
        out.append(np.linalg.norm(u[inner]) / np.linalg.norm(ut[inner]))
    rates = [math.log2(out[i] / out[i + 1]) for i in range(2)]
    assert min(rates) > 0.85 and out[-1] < 0.06, (out, rates)


def test_taylor_green_first_order_in_time():
    """Non-incremental pressure correction is first order in time (Sect. 1, ref. [1]; Remark 3.1)."""
    coarse = ci.cavity_mesh(33, 41)
    e = [_tg_error(coarse, dt, 0.2, 1)[0] for dt in (0.04, 0.02, 0.01)]
    rates = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert ((rates > 0.75) & (rates < 1.25)).all(), (e, rates)


@pytest.mark.parametrize("levels", [0, 1])
def test_taylor_green_second_order_in_space(levels):
    """Taylor-Green velocity (Eqs. 34-35) over 10 steps of dt = 1e-4, where the first-order
    splitting error is small: the nodal velocity error falls at second order in h, the P1 rate, for
    the standard scheme (l = 0) and for CGP (l = 1), on 9-, 17- and 33-node coarse grids."""
    es = [_tg_error(ci.cavity_mesh(n, 43), 1e-4, 1e-3, levels)[0] for n in (9, 17, 33)]
    rates = np.log2(np.array(es[:-1]) / np.array(es[1:]))
    assert ((rates > 1.7) & (rates < 2.5)).all(), (es, rates)


def test_taylor_green_cgp_close_to_standard():
    """One level of CGP on a 65x65-node fine mesh stays within 15 % of the standard scheme's
    velocity error (Table 1: the l = 1 velocity error grows only mildly over l = 0)."""
    e0, _, _ = _tg_error(ci.cavity_mesh(65, 42), 0.01, 0.1, 0)
    e1, _, _ = _tg_error(ci.cavity_mesh(33, 42), 0.01, 0.1, 1)
    assert e1 < 1.15 * e0, (e0, e1)
