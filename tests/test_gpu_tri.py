"""GPU parity of the paper's own discretisation (Section 3.3: P2-P1 triangles,
P1 position, P2 multiplier traces) against the FP64 oracle
(oracle/solver_tri.py): residual and Jacobian entry by entry, Newton steps,
and ten steps of the 3,104-triangle cylinder case."""
import numpy as np
import pytest

from paper_2609_31477_b300 import inputs as I
from oracle.solver_tri import viv_oracle_case_tri

from gpu_common import copy_state, perm_oracle_to_lib, push_state, rel_l2

pytestmark = pytest.mark.gpu

RE, USTAR, DT = 100.0, 8.0, 0.1


@pytest.fixture(scope="module")
def viv():
    import torch
    assert torch.cuda.is_available()
    from paper_2609_31477_b300 import build, viv as V
    build.build()
    V.load()
    return V


def _pair(viv, m, precision, **kw):
    mesh = I.triangulate_q2(I.viv_cylinder_mesh(m))
    u0 = I.viv_initial_velocity(mesh, 1.0, 1e-3, 1)
    oc = viv_oracle_case_tri(mesh, RE, USTAR, DT, u0)
    M = viv.Mesh(mesh)
    assert M.info["elem_type"] == 1
    case = viv.viv_case(M, RE, USTAR, DT, u0, precision=precision, **kw)
    return mesh, oc, M, case


def _seeded(oc, seed, amp):
    rng = np.random.default_rng(seed)
    U = oc.gather()
    U += amp * 0.05 * rng.standard_normal(U.shape)
    oc.scatter(U)
    X = oc.X
    bump = 0.02 * amp * np.sin(0.3 * X[:, 0]) * np.cos(0.25 * X[:, 1])
    for i in range(2):
        free = oc.dof_x[:, i] >= 0
        oc.x[free, i] = X[free, i] + bump[free] * (1 + i)
    oc.delta = amp * np.array([0.03, -0.02])
    oc.x[oc.cyl] = X[oc.cyl] + oc.delta
    oc._mids_from_vertices(oc.x)


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


def _jac(oc, M, c0, hu, hx):
    perm = perm_oracle_to_lib(oc, M)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    J_o = oc.jacobian(c0, hu, hx, DT).tocsr()
    rp, col = M.pattern()
    rows = np.repeat(np.arange(M.n_dofs), np.diff(rp))
    return perm, J_o, rp, col, rows, np.asarray(J_o[inv[rows], inv[col]]).ravel()


def test_residual_and_jacobian_entrywise_tri(viv):
    mesh, oc, M, case = _pair(viv, 4, viv.VIV_FP64)
    c0, hu, hx = _mid_step(oc, case, 41)
    nr = case.assemble(viv.VIV_RES | viv.VIV_JAC)
    perm, J_o, rp, col, rows, J_g_in_o = _jac(oc, M, c0, hu, hx)
    R_o = oc.residual(c0, hu, hx, DT)
    R_g = case.residual()[perm]
    assert np.abs(R_g - R_o).max() <= 1e-12 * np.abs(R_o).max()
    assert abs(nr - np.linalg.norm(R_o)) <= 1e-12 * np.linalg.norm(R_o)
    vals = case.jacobian_values()
    jscale = np.abs(J_o.data).max()
    err = np.abs(vals - J_g_in_o)
    assert err.max() <= 1e-11 * jscale, (err.max(), jscale)
    assert abs(np.abs(J_o).sum() - np.abs(J_g_in_o).sum()) <= 1e-9 * np.abs(J_o).sum()


def test_jacobian_fp32_volume_entrywise_tri(viv):
    mesh, oc, M, case = _pair(viv, 4, viv.VIV_MIXED, jacobian_fp32=1)
    c0, hu, hx = _mid_step(oc, case, 51)
    case.assemble(viv.VIV_RES | viv.VIV_JAC)
    perm, J_o, rp, col, rows, J_g_in_o = _jac(oc, M, c0, hu, hx)
    vals = case.jacobian_values()
    _, field = M.dof_labels()
    fb = np.isin(field[rows], [5, 6, 7, 8]) | np.isin(field[col], [5, 6])
    err = np.abs(vals - J_g_in_o)
    jscale = np.abs(J_o.data).max()
    assert err[fb].max() <= 1e-11 * jscale
    row_scale = np.maximum(np.maximum.reduceat(np.abs(J_g_in_o), rp[:-1]), 1e-300)[rows]
    rel = err[~fb] / row_scale[~fb]
    assert rel.max() <= 1e-4, rel.max()


def _compare(oc, st, tol_field=1e-9, tol_delta=1e-8):
    v = oc.is_vertex
    errs = dict(u=rel_l2(st["u"], oc.u), p=rel_l2(st["p"][v], oc.p[v]), x=rel_l2(st["x"] - oc.X, oc.x - oc.X),
                lam=rel_l2(st["lam"][oc.cyl], oc.lam[oc.cyl]), delta=np.abs(st["delta"] - oc.delta).max())
    assert max(errs["u"], errs["p"], errs["x"], errs["lam"]) <= tol_field and errs["delta"] <= tol_delta, errs
    par = oc.mid_parent[oc.is_mid]
    assert np.abs(st["x"][oc.is_mid] - 0.5 * (st["x"][par[:, 0]] + st["x"][par[:, 1]])).max() <= 1e-14
    return errs


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_threshold", "mixed_reuse"])
def test_steps_match_oracle_tri(viv, precision):
    prec = viv.VIV_FP64 if precision == "fp64" else viv.VIV_MIXED
    extra = {"fp64": {}, "mixed": dict(pivoting=viv.VIV_PIVOT_WINDOW, jacobian_fp32=1, predictor=1),
             "mixed_threshold": dict(pivoting=viv.VIV_PIVOT_THRESHOLD),
             "mixed_reuse": dict(pivoting=viv.VIV_PIVOT_WINDOW, jacobian_fp32=1, predictor=1, factor_reuse=1)}[precision]
    mesh, oc, M, case = _pair(viv, 4, prec, **extra)
    for _ in range(4):
        oc.step()
        info = case.step()
        assert info["res_norm"] <= 1e-10
        _compare(oc, case.get_state())
        assert np.allclose(info["force"], oc.force(), atol=1e-8)


@pytest.fixture(scope="module")
def tri_reference():
    """Oracle run of the 3,104-triangle cylinder case (the 1,552-quad mesh
    split, Re 100, U* 8, dt 0.1): states after each of 10 steps."""
    mesh = I.triangulate_q2(I.viv_cylinder_mesh(12))
    u0 = I.viv_initial_velocity(mesh, 1.0, 1e-3, 1)
    oc = viv_oracle_case_tri(mesh, RE, USTAR, DT, u0)
    states = []
    for _ in range(10):
        oc.step()
        states.append(copy_state(oc))
    return mesh, oc, states


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tri_cylinder_ten_steps_match_oracle(viv, tri_reference, precision):
    mesh, oc, states = tri_reference
    prec = viv.VIV_FP64 if precision == "fp64" else viv.VIV_MIXED
    extra = {} if precision == "fp64" else dict(pivoting=viv.VIV_PIVOT_WINDOW, jacobian_fp32=1, predictor=1)
    M = viv.Mesh(mesh)
    case = viv.viv_case(M, RE, USTAR, DT, I.viv_initial_velocity(mesh, 1.0, 1e-3, 1), precision=prec, **extra)
    for s in range(10):
        info = case.step()
        assert info["res_norm"] <= 1e-10
        for k, v in states[s].items():
            setattr(oc, k, v)
        _compare(oc, case.get_state())
