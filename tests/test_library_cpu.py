"""CPU checks of the C ABI library: it loads, exports every declared symbol, and its host-side
preprocessing (refinement numbering, s^p table, colouring, mesh validation) agrees with the oracle."""
import os
import re

import numpy as np
import pytest

import cgp_inputs as ci
from oracle import refine

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1610_06993_gb300 import cgp
    if not os.path.exists(cgp.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    cgp.load()
    return cgp


def test_exports_every_declared_symbol(L):
    decl = open(os.path.join(ROOT, "include", "cgp.h")).read()
    names = re.findall(r"^\s*(?:int|void|const char\*)\s+(cgp_\w+)\(", decl, re.M)
    assert len(names) >= 15
    lib = L.load()
    for n in names:
        assert hasattr(lib, n), n
    for n in ("cgp_mesh_create", "cgp_assemble", "cgp_momentum_solve", "cgp_restrict", "cgp_poisson_solve",
              "cgp_prolong_correct", "cgp_step"):
        assert n in names


def test_binding_declares_every_entry_point(L):
    """Every entry point of the header has explicit ctypes argument types in the binding: without
    them ctypes passes Python integers as 32-bit C ints, which truncates device pointers."""
    decl = open(os.path.join(ROOT, "include", "cgp.h")).read()
    names = re.findall(r"^\s*(?:int|void|const char\*)\s+(cgp_\w+)\(", decl, re.M)
    missing = [n for n in names if n not in L._SIGNATURES]
    assert not missing, missing


def test_every_entry_point_documents_its_errors():
    """Each declaration of the boundary header carries a comment that states what it does and how
    it fails (its CGP_ERR_* codes, or what it returns when it cannot fail)."""
    decl = open(os.path.join(ROOT, "include", "cgp.h")).read()
    names = re.findall(r"^\s*(?:int|void|const char\*)\s+(cgp_\w+)\(", decl, re.M)
    documented = {m.group(2): m.group(1) for m in
                  re.finditer(r"/\*((?:(?!\*/).)*)\*/\s*(?:int|void|const char\*)\s+(cgp_\w+)\(", decl, re.S)}
    missing = [n for n in names if n not in documented]
    assert not missing, missing
    silent = [n for n, doc in documented.items()
              if not re.search(r"Errors|CGP_ERR_|Returns|returns|nothing is written|never NULL", doc)]
    assert not silent, silent


def _header_structs():
    """Field lists (C type, name) of the header's typedef structs, comments removed."""
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "cgp.h")).read(), flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct \{(.*?)\}\s*(\w+);", text, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.match(r"((?:const )?\w+\s*\**)\s*(.*)", decl)
            ctype = m.group(1).replace(" ", "")
            for nm in m.group(2).split(","):
                nm = nm.strip()
                stars = len(nm) - len(nm.lstrip("*"))
                fields.append((ctype + "*" * stars, nm.lstrip("*")))
        out[name] = fields
    return out


def test_binding_structs_match_header(L):
    """The ctypes mirrors of the header's structs list the same fields, in the same order, with the
    same C types: a field added to one side only would shift every later field across the ABI."""
    import ctypes as C
    ctype_of = {"double": C.c_double, "int": C.c_int, "constdouble*": C.POINTER(C.c_double),
                "constint*": C.POINTER(C.c_int)}
    structs = _header_structs()
    for name in ("cgp_params", "cgp_mesh_desc", "cgp_info", "cgp_stats"):
        hdr = structs[name]
        py = getattr(L, name)._fields_
        assert [n for _, n in hdr] == [n for n, _ in py], name
        for (ct, n), (_, pt) in zip(hdr, py):
            assert ctype_of[ct] == pt, (name, n, ct, pt)


@pytest.mark.parametrize("mesh", [ci.cavity_mesh(9, 3), ci.bfs_mesh(2, 4)], ids=["cavity", "bfs"])
@pytest.mark.parametrize("levels", [0, 1, 2])
def test_native_refinement_matches_oracle(L, mesh, levels):
    xf, tf, sp, col = L.cgp_refine(mesh.xy, mesh.tri, levels)
    h = refine.build_hierarchy(mesh.xy, mesh.tri, levels)
    assert np.array_equal(xf, h.fine.xy)            # same numbering, same midpoint bits
    assert np.array_equal(tf, h.fine.tri)
    if levels > 0:
        assert np.array_equal(sp, h.sp[-1])
    # colouring: no two elements of one colour share a node
    for c in np.unique(col):
        nodes = tf[col == c].ravel()
        assert len(np.unique(nodes)) == len(nodes)
    assert col.max() < 32


def test_refinement_at_workload_size(L):
    m = ci.bfs_mesh(33, 1001)
    xf, tf, sp, col = L.cgp_refine(m.xy, m.tri, 1)
    assert xf.shape == (259117, 2) and tf.shape == (514008, 3)
    h = refine.build_hierarchy(m.xy, m.tri, 1)
    assert np.array_equal(xf, h.fine.xy) and np.array_equal(tf, h.fine.tri)


def _hilbert_position(x, y, bits):
    """Position of the integer cells (x, y), 0 <= x, y < 2^bits, along the Hilbert curve, from its
    recursive construction: at each scale, coarsest first, the quadrant (rx, ry) gives the base-4
    digit (3 rx) xor ry, and the coordinates are mapped into that quadrant's sub-curve (the lower
    quadrants are transposed, the lower-right one also reflected)."""
    n = 1 << bits
    x, y = np.asarray(x, dtype=np.int64).copy(), np.asarray(y, dtype=np.int64).copy()
    d = np.zeros_like(x)
    s = n // 2
    while s > 0:
        rx, ry = (x & s) > 0, (y & s) > 0
        d += s * s * ((3 * rx.astype(np.int64)) ^ ry.astype(np.int64))
        flip = ~ry & rx
        x, y = np.where(flip, n - 1 - x, x), np.where(flip, n - 1 - y, y)
        x, y = np.where(~ry, y, x), np.where(~ry, x, y)
        s //= 2
    return d


@pytest.mark.parametrize("bits", [1, 2, 3, 5])
def test_hilbert_position_visits_every_cell_by_unit_steps(bits):
    """The test's curve is a Hilbert curve: a bijection onto 0..4^bits - 1 starting at (0, 0) and
    ending at (2^bits - 1, 0), whose consecutive cells are edge neighbours."""
    n = 1 << bits
    gx, gy = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    d = _hilbert_position(gx.ravel(), gy.ravel(), bits)
    assert np.array_equal(np.sort(d), np.arange(n * n))
    order = np.argsort(d)
    px, py = gx.ravel()[order], gy.ravel()[order]
    assert (px[0], py[0]) == (0, 0) and (px[-1], py[-1]) == (n - 1, 0)
    assert np.all(np.abs(np.diff(px)) + np.abs(np.diff(py)) == 1)
    if bits == 1:
        assert [(a, b) for a, b in zip(px, py)] == [(0, 0), (0, 1), (1, 1), (1, 0)]


@pytest.mark.parametrize("name", ["cavity", "bfs", "cylinder_small"])
@pytest.mark.parametrize("levels", [0, 1, 2])
def test_stored_fine_order_is_the_hilbert_order(L, name, levels):
    """The fine-node storage order (fine_order = 0) is the refinement-order nodes sorted by their
    Hilbert position on 2^16 x 2^16 cells over the larger side of the bounding box, ties kept in
    refinement order; the identity at levels = 0. It makes the matrix graph local: the median index
    distance of the fine edges falls to a few rows (observed 3, against 168-3,237 in the refinement
    order on these meshes)."""
    mesh = {"cavity": lambda: ci.cavity_mesh(17, 3), "bfs": lambda: ci.bfs_mesh(4, 1001),
            "cylinder_small": lambda: ci.workload("cylinder_small")[0]}[name]()
    xf, tf, _, _ = L.cgp_refine(mesh.xy, mesh.tri, levels)
    perm = L.cgp_refine_order(mesh.xy, mesh.tri, levels)
    assert np.array_equal(perm, L.cgp_refine_order(mesh.xy, mesh.tri, levels))
    if levels == 0:
        assert np.array_equal(perm, np.arange(len(xf)))
        return
    lo = xf.min(axis=0)
    ext = float((xf.max(axis=0) - lo).max())
    cells = np.minimum(65535.0, np.maximum(0.0, (xf - lo) * (65535.0 / ext))).astype(np.int64)
    key = _hilbert_position(cells[:, 0], cells[:, 1], 16)
    assert np.array_equal(perm, np.argsort(key, kind="stable"))
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    e = np.concatenate([tf[:, [0, 1]], tf[:, [1, 2]], tf[:, [2, 0]]])
    stored = np.median(np.abs(inv[e[:, 0]] - inv[e[:, 1]]))
    natural = np.median(np.abs(e[:, 0] - e[:, 1]))
    assert stored <= 8 and stored * 8 < natural, (stored, natural)


def test_native_mapping_loop_counts_of_the_paper(L):
    """The native refinement on the mesh of the paper's mapping count (Sect. 3.2, Table 5; l = 3,
    1,600 coarse and 102,400 fine elements): the prolongation's levels 1-3 hold 68,659 nodes."""
    from test_oracle_pins import load_mapping_loop_counts, mapping_loop_mesh
    g = load_mapping_loop_counts()
    m = mapping_loop_mesh()
    sizes = []
    for lv in range(1, g["levels"] + 1):
        xf, tf, sp, _ = L.cgp_refine(m.xy, m.tri, lv)
        sizes.append(len(xf))
        assert len(sp) == len(xf)
    assert len(tf) == g["fine_elements"]
    assert sum(sizes) == g["prolongation_loops"]


@pytest.mark.parametrize("case", ["taylor_green", "cylinder"])
def test_native_nested_mesh_counts_of_the_paper(L, case):
    """The native refinement reproduces the nested-mesh counts of the paper's Taylor-Green and
    cylinder meshes (Sects. 3.1, 3.3) from a mesh of the coarsest level's size."""
    from test_oracle_pins import NESTED_GRIDS, holed_mesh_of_size, load_nested_mesh_counts
    levels = load_nested_mesh_counts()[case]
    m = holed_mesh_of_size(*levels[0], *NESTED_GRIDS[case])
    for lv, (nodes, elems) in enumerate(levels[1:], start=1):
        xf, tf, _, _ = L.cgp_refine(m.xy, m.tri, lv)
        assert len(tf) == elems and (nodes < 0 or len(xf) == nodes)


def test_mesh_validation_errors(L):
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    good = np.array([[0, 1, 2], [1, 3, 2]])
    L.cgp_refine(xy, good, 1)
    with pytest.raises(L.CGPError) as e:
        L.cgp_refine(xy, np.array([[0, 2, 1], [1, 3, 2]]), 1)      # clockwise
    assert e.value.code == L.CGP_ERR_MESH
    with pytest.raises(L.CGPError) as e:
        L.cgp_refine(xy, np.array([[0, 1, 7]]), 1)                  # index out of range
    assert e.value.code == L.CGP_ERR_MESH
    with pytest.raises(L.CGPError) as e:                             # three triangles on one edge
        xy5 = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, 1.0], [0.5, 2.0], [0.5, 3.0]])
        L.cgp_refine(xy5, np.array([[0, 1, 2], [0, 1, 3], [0, 1, 4]]), 0)
    assert e.value.code == L.CGP_ERR_MESH
    with pytest.raises(L.CGPError) as e:
        L.cgp_refine(xy, good, 7)
    assert e.value.code == L.CGP_ERR_ARG
    with pytest.raises(L.CGPError) as e:
        L.cgp_refine_order(xy, np.array([[0, 2, 1], [1, 3, 2]]), 1)
    assert e.value.code == L.CGP_ERR_MESH


def test_status_strings(L):
    assert L.cgp_status_str(0) == "CGP_OK"
    assert L.cgp_status_str(L.CGP_ERR_TIMEOUT) == "CGP_ERR_TIMEOUT"
