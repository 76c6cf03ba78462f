"""The C ABI library loads without a GPU, exports every symbol the header
declares, and its host-side analysis (numbering, pattern, symbolic
factorisation) is consistent with the oracle's unknowns and Jacobian."""
import os
import re

import numpy as np
import pytest

from paper_2609_31477_b300 import build, inputs as I, viv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return viv.load()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "viv.h")).read()
    declared = set(re.findall(r"\b(viv_[a-z0-9_]+)\s*\(", hdr))
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(viv.SIGNATURES), declared ^ set(viv.SIGNATURES)
    assert b"sm_103a" in lib.viv_version()


def test_bad_mesh_is_rejected(lib):
    m = I.viv_cylinder_mesh(4)
    bad = dict(m)
    bad["conn"] = m["conn"].copy()
    bad["conn"][3, 2] = len(m["X"]) + 5
    with pytest.raises(viv.VivError) as e:
        viv.Mesh(bad, device=False)
    assert e.value.status == 1 and "range" in str(e.value)


def _labels_oracle(c):
    lab = {}
    D = c.dof_u.shape[1]
    for a in range(c.n):
        for i, f in enumerate(("ux", "uy", "uz")[:D]):
            if c.dof_u[a, i] >= 0:
                lab[c.dof_u[a, i]] = (a, f)
        if c.dof_p[a] >= 0:
            lab[c.dof_p[a]] = (a, "p")
        for i, f in enumerate(("xx", "xy", "xz")[:D]):
            if c.dof_x[a, i] >= 0:
                lab[c.dof_x[a, i]] = (a, f)
        for i, f in enumerate(("lx", "ly", "lz")[:D]):
            if c.dof_l[a, i] >= 0:
                lab[c.dof_l[a, i]] = (a, f)
    if c.has_body:
        lab[c.dof_d[0]] = (c.n, "dx")
        lab[c.dof_d[1]] = (c.n, "dy")
    return lab


def test_host_analysis_matches_oracle_unknowns_and_pattern(lib):
    from oracle.solver import viv_oracle_case
    m = I.viv_cylinder_mesh(4)
    M = viv.Mesh(m, device=False)
    node, field = M.dof_labels()
    oc = viv_oracle_case(m, 100.0, 8.0, 0.1, I.viv_initial_velocity(m))
    lab = _labels_oracle(oc)
    assert M.n_dofs == oc.ndof
    gpu_lab = {(int(a), viv.FIELD[int(f)]): i for i, (a, f) in enumerate(zip(node, field))}
    assert set(gpu_lab) == set(lab.values())
    perm = np.array([gpu_lab[lab[i]] for i in range(oc.ndof)])   # oracle dof -> library dof
    oc.u_n, oc.x_n = oc.u.copy(), oc.x.copy()
    c0, hu, hx = oc.bdf_coefficients()
    J = oc.jacobian(c0, hu, hx, 0.1).tocoo()
    rp, col = M.pattern()
    rows = np.repeat(np.arange(M.n_dofs), np.diff(rp))
    have = set(zip(rows.tolist(), col.tolist()))
    need = set(zip(perm[J.row].tolist(), perm[J.col].tolist()))
    assert need <= have
    # no structural zero blocks of Section 3.2 in the pattern
    kind = np.array([viv.FIELD[int(f)][0] for f in field])
    pairs = set(zip(kind[rows].tolist(), kind[col].tolist()))
    for bad in (("p", "p"), ("l", "l"), ("x", "u"), ("x", "p"), ("x", "l")):
        assert bad not in pairs
    info = M.info
    assert info["n_fronts"] > 10 and info["max_front"] >= 2 and info["factor_flops"] > 0


def test_host_analysis_3d_matches_oracle_unknowns_and_pattern(lib):
    """Periodic hexahedral extrusion: the library numbers the oracle's
    unknowns (three components of u, x and lambda, the z position of Gamma
    held) and its pattern holds every oracle Jacobian entry that is not the
    rounding of an exact zero."""
    from oracle.solver3d import viv_oracle_case3d
    m = I.viv_cylinder_mesh3d(2, 2, 0.7)
    M = viv.Mesh(m, device=False)
    assert M.dim == 3 and M.info["dim"] == 3
    node, field = M.dof_labels()
    n = len(m["X"])
    oc = viv_oracle_case3d(m, 150.0, 6.0, 0.05, np.zeros((n, 3)))
    assert M.n_dofs == oc.ndof
    lab = _labels_oracle(oc)
    gpu_lab = {(int(a), viv.FIELD[int(f)]): i for i, (a, f) in enumerate(zip(node, field))}
    assert set(gpu_lab) == set(lab.values())
    perm = np.array([gpu_lab[lab[i]] for i in range(oc.ndof)])
    oc.u = np.random.default_rng(1).normal(size=(n, 3))
    oc.u_n, oc.x_n = oc.u.copy(), oc.x.copy()
    c0, hu, hx = oc.bdf_coefficients()
    J = oc.jacobian(c0, hu, hx, 0.05).tocoo()
    rp, col = M.pattern()
    rows = np.repeat(np.arange(M.n_dofs), np.diff(rp))
    have = set(zip(rows.tolist(), col.tolist()))
    big = np.abs(J.data) > 1e-13 * np.abs(J.data).max()
    need = set(zip(perm[J.row[big]].tolist(), perm[J.col[big]].tolist()))
    assert need <= have
    kind = np.array([viv.FIELD[int(f)][0] for f in field])
    pairs = set(zip(kind[rows].tolist(), kind[col].tolist()))
    for bad in (("p", "p"), ("l", "l"), ("x", "u"), ("x", "p"), ("x", "l")):
        assert bad not in pairs
    assert M.info["front_entries"] > 0 and M.info["factor_flops"] > 0


def test_host_analysis_triangles_match_oracle_unknowns_and_pattern(lib):
    """P2-P1 triangles with a P1 position: the library numbers the oracle's
    unknowns (no position unknowns at midside nodes) and its pattern holds
    every oracle Jacobian entry."""
    from oracle.solver_tri import viv_oracle_case_tri
    m = I.triangulate_q2(I.viv_cylinder_mesh(4))
    M = viv.Mesh(m, device=False)
    assert M.info["elem_type"] == 1 and M.dim == 2
    node, field = M.dof_labels()
    oc = viv_oracle_case_tri(m, 100.0, 8.0, 0.1, I.viv_initial_velocity(m))
    assert M.n_dofs == oc.ndof
    lab = _labels_oracle(oc)
    gpu_lab = {(int(a), viv.FIELD[int(f)]): i for i, (a, f) in enumerate(zip(node, field))}
    assert set(gpu_lab) == set(lab.values())
    perm = np.array([gpu_lab[lab[i]] for i in range(oc.ndof)])
    oc.u_n, oc.x_n = oc.u.copy(), oc.x.copy()
    c0, hu, hx = oc.bdf_coefficients()
    J = oc.jacobian(c0, hu, hx, 0.1).tocoo()
    rp, col = M.pattern()
    rows = np.repeat(np.arange(M.n_dofs), np.diff(rp))
    have = set(zip(rows.tolist(), col.tolist()))
    need = set(zip(perm[J.row].tolist(), perm[J.col].tolist()))
    assert need <= have
    # a midside node off its edge's midpoint is rejected
    bad = dict(m)
    bad["X"] = np.array(m["X"])
    bad["X"][m["conn"][0, 3], 0] += 1e-3
    with pytest.raises(viv.VivError):
        viv.Mesh(bad, device=False)


def test_bad_3d_and_triangle_meshes_are_rejected(lib):
    """Host-side validation of the 3-D and triangle descriptions: wrapped nodes
    without a span, a Gamma node whose z position is free, a face index out of
    range, and triangles on a 3-D mesh."""
    m = I.viv_cylinder_mesh3d(2, 2, 0.7)
    viv.Mesh(m, device=False)          # the valid mesh analyses
    bad = dict(m, span=0.0)
    with pytest.raises(viv.VivError):
        viv.Mesh(bad, device=False)
    bad = dict(m, tags=np.array(m["tags"]) & ~I.X_FIX_Z)
    with pytest.raises(viv.VivError):
        viv.Mesh(bad, device=False)
    gf = np.array(m["gamma_faces"])
    gf[0, 1] = 6
    with pytest.raises(viv.VivError):
        viv.Mesh(dict(m, gamma_faces=gf), device=False)
    with pytest.raises(viv.VivError):
        viv.Mesh(dict(m, elem="tri6"), device=False)


@pytest.mark.parametrize("family", ["quad", "tri", "hex"])
def test_symbolic_factorisation_covers_every_unknown_once(lib, family):
    """The nested dissection and symbolic factorisation of each element
    family: every unknown but the two border ones is a pivot of exactly one
    front, a front's order is at least its pivot count, parents sit on higher
    tree levels and the predicted storage is the sum of the fronts' squares."""
    mesh = {"quad": lambda: I.viv_cylinder_mesh(4),
            "tri": lambda: I.triangulate_q2(I.viv_cylinder_mesh(4)),
            "hex": lambda: I.viv_cylinder_mesh3d(2, 2, 0.7)}[family]()
    M = viv.Mesh(mesh, device=False)
    fr = M.fronts()
    m, p, lev, par = (fr[k].astype(np.int64) for k in ("m", "p", "level", "parent"))
    assert p.sum() == M.n_dofs - 2
    assert np.all(m >= p) and np.all(p >= 0)
    child = par >= 0
    assert np.all(lev[par[child]] > lev[child])
    assert (~child).sum() >= 1 and np.all(par < len(m))
    assert M.info["front_entries"] == int((m * m).sum())
    assert M.info["max_front"] == int(m.max())


@pytest.mark.parametrize("family", ["quad", "tri", "hex"])
def test_element_slots_cover_the_pattern(lib, family):
    """viv_mesh_element_slots: every CSR value is reached by some element or
    face pair (or is a border diagonal), and every element pair's slot lies in
    a row and a column of that element's unknowns (delta for Gamma
    positions)."""
    mesh = {"quad": lambda: I.viv_cylinder_mesh(4),
            "tri": lambda: I.triangulate_q2(I.viv_cylinder_mesh(4)),
            "hex": lambda: I.viv_cylinder_mesh3d(2, 2, 0.7)}[family]()
    M = viv.Mesh(mesh, device=False)
    rp, col = M.pattern()
    es, fs = M.element_slots()
    nnz = len(col)
    hit = np.zeros(nnz, bool)
    hit[es[es >= 0]] = True
    hit[fs[fs >= 0]] = True
    node, _ = M.dof_labels()
    n_nodes = len(mesh["X"])
    dd = [s for s in range(nnz) if node[np.searchsorted(rp, s, side="right") - 1] == n_nodes and node[col[s]] == n_nodes]
    hit[dd] = True
    assert hit.all()
    rows = np.searchsorted(rp, np.arange(nnz), side="right") - 1
    conn = np.asarray(mesh["conn"])
    for e in range(0, len(conn), max(1, len(conn) // 25)):
        s = es[e][es[e] >= 0]
        nodes = set(conn[e].tolist()) | {n_nodes}
        assert set(node[rows[s]].tolist()) <= nodes and set(node[col[s]].tolist()) <= nodes


@pytest.mark.parametrize("family", ["quad", "tri", "hex"])
def test_negatively_oriented_elements_are_rejected(lib, family):
    """Mirroring the mesh in y turns every element inside out: the analysis
    rejects it instead of producing negative Jacobian determinants."""
    mesh = {"quad": lambda: I.viv_cylinder_mesh(3),
            "tri": lambda: I.triangulate_q2(I.viv_cylinder_mesh(3)),
            "hex": lambda: I.viv_cylinder_mesh3d(2, 2, 0.7)}[family]()
    viv.Mesh(mesh, device=False)
    X = np.array(mesh["X"])
    X[:, 1] *= -1.0
    with pytest.raises(viv.VivError):
        viv.Mesh(dict(mesh, X=X), device=False)
