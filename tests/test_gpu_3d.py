"""GPU parity of the 3-D path (27-node hexahedra, periodic span) against the
FP64 oracle (oracle/solver3d.py): residual and Jacobian entry by entry,
Newton steps on a small periodic extrusion, and the stored oracle run of the
388-hexahedron cylinder case."""
import os

import numpy as np
import pytest

from paper_2609_31477_b300 import inputs as I
from oracle.solver3d import viv_oracle_case3d

from gpu_common import copy_state, perm_oracle_to_lib, push_state, rel_l2

pytestmark = pytest.mark.gpu

RE, USTAR, DT = 250.0, 7.0, 0.05
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def viv():
    import torch
    assert torch.cuda.is_available()
    from paper_2609_31477_b300 import build, viv as V
    build.build()
    V.load()
    return V


def _pair(viv, precision, m=2, layers=2, span=0.7, **kw):
    mesh = I.viv_cylinder_mesh3d(m, layers, span)
    u0 = I.viv_initial_velocity(mesh, 1.0, 1e-2, 5)
    oc = viv_oracle_case3d(mesh, RE, USTAR, DT, u0)
    M = viv.Mesh(mesh)
    assert M.dim == 3
    case = viv.viv_case(M, RE, USTAR, DT, u0, precision=precision, **kw)
    assert abs(case.resolved_params()["k"] - oc.k) <= 1e-14 * oc.k
    return mesh, oc, M, case


def _seeded(oc, seed, amp):
    """A smooth admissible state: velocity, pressure and multiplier perturbed,
    the mesh deformed in all three directions (periodically in z), delta set."""
    rng = np.random.default_rng(seed)
    U = oc.gather()
    U += amp * 0.05 * rng.standard_normal(U.shape)
    oc.scatter(U)
    X = oc.X
    zf = 2 * np.pi / oc.span
    bump = 0.02 * amp * np.sin(0.3 * X[:, 0]) * np.cos(0.25 * X[:, 1]) * (1 + 0.5 * np.sin(zf * X[:, 2]))
    for i in range(3):
        free = oc.dof_x[:, i] >= 0
        oc.x[free, i] = X[free, i] + bump[free] * (1 + i)
    oc.delta = amp * np.array([0.03, -0.02])
    oc.x[oc.cyl, :2] = X[oc.cyl, :2] + oc.delta
    oc.x[oc.cyl, 2] = X[oc.cyl, 2]


def _mid_step(oc, case, seed):
    _seeded(oc, seed, 0.5)
    prev = copy_state(oc)
    _seeded(oc, seed + 1, 0.7)
    cur = copy_state(oc)
    _seeded(oc, seed + 2, 1.0)
    it = copy_state(oc)
    push_state(case, cur)
    case.set_history(prev["u"], prev["x"])
    case.begin_step()
    push_state(case, it)
    oc.u_n, oc.x_n = cur["u"], cur["x"]
    oc.hist = (prev["u"], prev["x"])
    for k, v in it.items():
        setattr(oc, k, v.copy())
    return oc.bdf_coefficients()


def _jac_in_lib_order(oc, M, c0, hu, hx):
    perm = perm_oracle_to_lib(oc, M)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    J_o = oc.jacobian(c0, hu, hx, DT).tocsr()
    rp, col = M.pattern()
    rows = np.repeat(np.arange(M.n_dofs), np.diff(rp))
    return perm, J_o, rp, col, rows, np.asarray(J_o[inv[rows], inv[col]]).ravel()


def test_residual_and_jacobian_entrywise_3d(viv):
    mesh, oc, M, case = _pair(viv, viv.VIV_FP64)
    c0, hu, hx = _mid_step(oc, case, 21)
    nr = case.assemble(viv.VIV_RES | viv.VIV_JAC)
    perm, J_o, rp, col, rows, J_g_in_o = _jac_in_lib_order(oc, M, c0, hu, hx)
    R_o = oc.residual(c0, hu, hx, DT)
    R_g = case.residual()[perm]
    assert np.abs(R_g - R_o).max() <= 1e-12 * np.abs(R_o).max()
    assert abs(nr - np.linalg.norm(R_o)) <= 1e-12 * np.linalg.norm(R_o)
    vals = case.jacobian_values()
    jscale = np.abs(J_o.data).max()
    err = np.abs(vals - J_g_in_o)
    assert err.max() <= 1e-11 * jscale, (err.max(), jscale)
    # oracle entries outside the library's pattern are the rounding of exact
    # zeros (a rigid shift of a Gamma face leaves its area unchanged)
    outside = np.abs(J_o).sum() - np.abs(J_g_in_o).sum()
    assert outside <= 1e-12 * np.abs(J_o).sum()


def test_jacobian_fp32_volume_entrywise_3d(viv):
    mesh, oc, M, case = _pair(viv, viv.VIV_MIXED, jacobian_fp32=1)
    c0, hu, hx = _mid_step(oc, case, 31)
    case.assemble(viv.VIV_RES | viv.VIV_JAC)
    perm, J_o, rp, col, rows, J_g_in_o = _jac_in_lib_order(oc, M, c0, hu, hx)
    vals = case.jacobian_values()
    _, field = M.dof_labels()
    lam_f, border_f = [5, 6, 11], [7, 8]
    fb = np.isin(field[rows], lam_f + border_f) | np.isin(field[col], lam_f)
    err = np.abs(vals - J_g_in_o)
    jscale = np.abs(J_o.data).max()
    assert err[fb].max() <= 1e-11 * jscale
    row_scale = np.maximum(np.maximum.reduceat(np.abs(J_g_in_o), rp[:-1]), 1e-300)[rows]
    rel = err[~fb] / row_scale[~fb]
    assert rel.max() <= 1e-4, rel.max()
    assert np.median(rel) <= 1e-6, np.median(rel)


def _compare(oc, st, tol_field=1e-9, tol_delta=1e-8):
    v = oc.is_vertex
    errs = dict(u=rel_l2(st["u"], oc.u), p=rel_l2(st["p"][v], oc.p[v]), x=rel_l2(st["x"] - oc.X, oc.x - oc.X),
                lam=rel_l2(st["lam"][oc.cyl], oc.lam[oc.cyl]), delta=np.abs(st["delta"] - oc.delta).max())
    assert max(errs["u"], errs["p"], errs["x"], errs["lam"]) <= tol_field and errs["delta"] <= tol_delta, errs
    return errs


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_threshold", "mixed_reuse"])
def test_steps_match_oracle_3d(viv, precision):
    prec = viv.VIV_FP64 if precision == "fp64" else viv.VIV_MIXED
    extra = {"fp64": {}, "mixed": dict(pivoting=viv.VIV_PIVOT_WINDOW, jacobian_fp32=1),
             "mixed_threshold": dict(pivoting=viv.VIV_PIVOT_THRESHOLD),
             "mixed_reuse": dict(pivoting=viv.VIV_PIVOT_WINDOW, jacobian_fp32=1, predictor=1, factor_reuse=1)}[precision]
    mesh, oc, M, case = _pair(viv, prec, **extra)
    for _ in range(2):
        oc.step()
        info = case.step()
        assert info["res_norm"] <= 1e-10
        _compare(oc, case.get_state())
        assert np.allclose(info["force"], oc.force(), rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("precision,predictor", [("fp64", 0), ("mixed", 0), ("mixed", 1)])
def test_cylinder3d_matches_stored_oracle_run(viv, precision, predictor):
    """The 388-hexahedron periodic cylinder (Re 300, U* 8, dt 0.05), two steps,
    against the oracle's stored run (tests/golden/cylinder3d_m3_z4_re300.npz)."""
    g = np.load(os.path.join(HERE, "golden", "cylinder3d_m3_z4_re300.npz"))
    mesh = I.viv_cylinder_mesh3d(int(g["m"]), int(g["layers"]), float(g["span"]))
    u0 = I.viv_initial_velocity(mesh, 1.0, 1e-3, int(g["seed"]))
    M = viv.Mesh(mesh)
    prec = viv.VIV_FP64 if precision == "fp64" else viv.VIV_MIXED
    extra = {} if precision == "fp64" else dict(pivoting=viv.VIV_PIVOT_WINDOW, jacobian_fp32=1,
                                                 predictor=predictor)
    case = viv.viv_case(M, float(g["Re"]), float(g["Ustar"]), float(g["dt"]), u0, precision=prec, **extra)
    for s in range(int(g["steps"])):
        info = case.step()
        assert info["res_norm"] <= 1e-10
        assert np.abs(np.array(info["delta"]) - g["delta"][s]).max() <= 1e-8
        assert np.allclose(info["force"], g["force"][s], rtol=1e-8, atol=1e-10)
    st = case.get_state()
    X = np.asarray(mesh["X"])
    cyl = (mesh["tags"] & I.CYL) != 0
    n = len(X)
    vert = np.zeros(n, bool)
    vert[np.asarray(mesh["conn"])[:, [0, 2, 6, 8, 18, 20, 24, 26]].ravel()] = True
    assert rel_l2(st["u"], g["u"]) <= 1e-9
    assert rel_l2(st["p"][vert], g["p_vertex"]) <= 1e-9
    assert rel_l2(st["x"] - X, g["x_minus_X"]) <= 1e-9
    assert rel_l2(st["lam"][cyl], g["lam_gamma"]) <= 1e-9
    # the flow is genuinely three-dimensional: the seeded spanwise noise is carried
    assert np.abs(st["u"][:, 2]).max() > 1e-6
