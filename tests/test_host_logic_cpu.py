"""CPU checks of the library's host-side preprocessing, through a small g++ driver
(tests/host_checks.cpp) linked against the library's own host sources: the fine CSR pattern and its
diagonal slots, the element -> CSR slot maps of the assembly, the s^u table, the sliced-ELL
layouts of the SpMV kernels and the two-level Schwarz coarse space (linear coarse functions and the
inverse Galerkin matrix of the coarse Poisson preconditioner). Each is checked against its
definition, computed here with numpy / scipy from the mesh alone. No GPU is used."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

import cgp_inputs as ci
from oracle import refine

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1610_06993_gb300", "csrc")
OUT = os.path.join(ROOT, "paper_1610_06993_gb300", "_build", "host_checks")


@pytest.fixture(scope="module")
def driver():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    os.makedirs(OUT, exist_ok=True)
    exe = os.path.join(OUT, "host_checks")
    cmd = [gxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
           os.path.join(ROOT, "tests", "host_checks.cpp"), os.path.join(CSRC, "host_mesh.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def run(exe, mesh, levels, renumber, S=64):
    """The driver's arrays for ``mesh`` refined ``levels`` times."""
    head = f"{levels} {int(renumber)} {S} {mesh.n_nodes} {mesh.n_tris}\n"
    body = " ".join(repr(float(v)) for v in np.asarray(mesh.xy).ravel()) + "\n" + \
        " ".join(str(int(v)) for v in np.asarray(mesh.tri).ravel()) + "\n"
    r = subprocess.run([exe], input=head + body, capture_output=True, text=True, check=True)
    out = {}
    for ln in r.stdout.splitlines():
        name, count, *vals = ln.split()
        arr = np.array([float(v) for v in vals]) if "xy" in name or "fxy" in name or "Ai" in name else \
            np.array([int(v) for v in vals], dtype=np.int64)
        assert len(arr) == int(count), name
        out[name] = arr
    assert out["status"][0] == 0
    return out


MESHES = {
    "cavity": lambda: ci.cavity_mesh(9, 3),
    "bfs": lambda: ci.bfs_mesh(3, 1001),
    "cylinder_small": lambda: ci.workload("cylinder_small")[0],
}


@pytest.mark.parametrize("renumber", [False, True], ids=["refinement", "hilbert"])
@pytest.mark.parametrize("levels", [1, 2])
@pytest.mark.parametrize("name", sorted(MESHES))
def test_fine_pattern_slots_and_tables(driver, name, levels, renumber):
    """The fine CSR holds exactly the pairs of nodes that share a triangle (the P1 pattern of
    Eqs. 16-18), with sorted columns and the diagonal slot of every row; every element's nine slots
    point at (row tri[a], column tri[b]); s^u (Eq. 30) maps each coarse node to the stored fine node
    at the same point; the stored fine mesh is the refinement's mesh relabelled by the storage
    order."""
    mesh = MESHES[name]()
    o = run(driver, mesh, levels, renumber)
    h = refine.build_hierarchy(mesh.xy, mesh.tri, levels)
    n, t = len(h.fine.xy), len(h.fine.tri)
    perm = o["fperm"] if renumber else np.arange(n)
    assert np.array_equal(np.sort(perm), np.arange(n))
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    xy = o["fine_xy"].reshape(n, 2)
    tri = o["fine_tri"].reshape(t, 3)
    assert np.array_equal(xy, h.fine.xy[perm])
    # the same triangles, relabelled (the stored order may sort them)
    ref = np.sort(inv[h.fine.tri], axis=1)
    got = np.sort(tri, axis=1)
    assert np.array_equal(np.unique(ref, axis=0), np.unique(got, axis=0)) and len(np.unique(got, axis=0)) == t
    # CSR pattern = node pairs of a common triangle, columns sorted, diagonal slot
    rp, cols, diag = o["fine_rp"], o["fine_ci"], o["fine_diag"]
    rows = np.repeat(np.arange(n), np.diff(rp))
    pat = sp.coo_matrix((np.ones(9 * t), (np.repeat(tri, 3, axis=1).ravel(), np.tile(tri, (1, 3)).ravel())),
                        shape=(n, n)).tocsr()
    pat.sum_duplicates()
    pat.sort_indices()
    assert np.array_equal(rp, pat.indptr) and np.array_equal(cols, pat.indices)
    assert np.all(np.diff(cols)[np.diff(rows) == 0] > 0)
    assert np.array_equal(cols[diag], np.arange(n)) and np.all((diag >= rp[:-1]) & (diag < rp[1:]))
    # element slots: slot[e][a*3+b] is the CSR entry (tri[e][a], tri[e][b])
    slot = o["fine_slot"].reshape(t, 9)
    for a in range(3):
        for b in range(3):
            s = slot[:, 3 * a + b]
            assert np.array_equal(rows[s], tri[:, a]) and np.array_equal(cols[s], tri[:, b])
    # s^u: the stored fine node at each coarse node's point
    assert np.array_equal(xy[o["su"]], np.asarray(mesh.xy, dtype=np.float64))


@pytest.mark.parametrize("sigma", [32, 1])
@pytest.mark.parametrize("name", sorted(MESHES))
def test_sliced_ell_layout(driver, name, sigma):
    """The sliced-ELL copy of the fine pattern (32-row slices; rows sorted by decreasing length
    inside windows of sigma rows, sigma = 1: the natural order): every CSR entry sits in exactly one
    slot, at slot k of its row's lane, with its column; padding slots carry the row itself as
    column and no entry; each slice is as wide as its longest row."""
    mesh = MESHES[name]()
    o = run(driver, mesh, 2, True)
    rp, cols = o["fine_rp"], o["fine_ci"]
    n, nnz = len(rp) - 1, len(cols)
    tag = f"sell{sigma}_"
    ptr, width, col, src, perm = (o[tag + k] for k in ("ptr", "width", "col", "src", "perm"))
    C = 32
    ns = (n + C - 1) // C
    assert len(width) == ns and np.array_equal(np.diff(ptr), width * C)
    real = perm[perm >= 0]
    assert np.array_equal(np.sort(real), np.arange(n)) and np.all(perm[n:] == -1)
    if sigma == 1:
        assert np.array_equal(real, np.arange(n))
    length = np.diff(rp)
    for w0 in range(0, n, sigma):
        assert np.all(np.diff(length[perm[w0:min(n, w0 + sigma)]]) <= 0)
    hit = np.zeros(nnz, dtype=np.int64)
    for s in range(ns):
        lanes = perm[s * C:(s + 1) * C]
        assert width[s] == max(length[r] for r in lanes if r >= 0)
        for k in range(width[s]):
            p = ptr[s] + k * C + np.arange(C)
            for l, r in enumerate(lanes):
                if r >= 0 and k < length[r]:
                    assert src[p[l]] == rp[r] + k and col[p[l]] == cols[rp[r] + k]
                    hit[src[p[l]]] += 1
                else:
                    assert src[p[l]] == -1 and col[p[l]] == (r if r >= 0 else 0)
    assert np.all(hit == 1)


@pytest.mark.parametrize("name,S", [("bfs", 64), ("cylinder_small", 48), ("cavity", 16)])
def test_schwarz_coarse_space(driver, name, S):
    """The two-level Schwarz preconditioner's coarse space on a Hilbert renumbering of the coarse
    nodes cut into S-row subdomains: the linear functions are (x - xbar) / H and (y - ybar) / H
    with the centroid and RMS radius of each subdomain's nodes, and the library's inverse Galerkin
    matrix inverts A_0 = R_0 A R_0^T (three functions 1, fx, fy per subdomain; a function that
    vanishes on its subdomain, as the linear ones of a one-node subdomain do, gets a unit diagonal)
    for the SPD test matrix A = I + graph Laplacian of the coarse pattern."""
    mesh = MESHES[name]()
    o = run(driver, mesh, 1, True, S)
    assert o["galerkin_status"][0] == 0
    n = mesh.n_nodes
    perm, sub = o["schwarz_perm"], o["schwarz_sub"]
    assert np.array_equal(sub, np.arange(n) // S)
    nsub = int(sub.max()) + 1
    xy = np.asarray(mesh.xy, dtype=np.float64)[perm]
    f = np.empty((n, 2))
    for a in range(nsub):
        m = sub == a
        c = xy[m].mean(axis=0)
        H = np.sqrt(np.mean(np.sum((xy[m] - c) ** 2, axis=1)))
        f[m] = (xy[m] - c) / H if H > 0 else 0.0     # a one-node subdomain has no linear functions
    np.testing.assert_allclose(o["schwarz_fxy"].reshape(n, 2), f, rtol=0, atol=1e-12)
    # A in the renumbered order, from the coarse pattern
    rp, cols = o["coarse_rp"], o["coarse_ci"]
    rows = np.repeat(np.arange(n), np.diff(rp))
    deg = np.diff(rp) - 1
    vals = np.where(rows == cols, 1.0 + deg[rows], -1.0)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))[perm][:, perm].toarray()
    R0 = np.zeros((3 * nsub, n))
    for fi, phi in enumerate((np.ones(n), f[:, 0], f[:, 1])):
        R0[fi * nsub + sub, np.arange(n)] = phi
    A0 = R0 @ A @ R0.T
    idle = np.diag(A0) == 0.0                       # functions vanishing on their subdomain
    A0[idle, idle] = 1.0
    Ai = o["schwarz_Ai"].reshape(3 * nsub, 3 * nsub)
    assert np.allclose(Ai, Ai.T, rtol=0, atol=1e-12 * np.abs(Ai).max())
    err = np.abs(Ai @ A0 - np.eye(3 * nsub)).max()
    assert err < 1e-9, err
