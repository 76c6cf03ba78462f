"""Parity of the CUDA path (through the C ABI) with the FP64 oracle:
residual and Jacobian entry by entry, the refined multifrontal solve, and
whole BDF/Newton steps on the cylinder meshes."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from paper_2609_31477_b300 import inputs as I
from oracle.solver import viv_oracle_case

from gpu_common import copy_state, perm_oracle_to_lib, push_state, rel_l2, seeded_state

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


def _pair(viv, m, precision, seed=3, pivoting=0, jacobian_fp32=0):
    mesh = I.viv_cylinder_mesh(m)
    u0 = I.viv_initial_velocity(mesh, 1.0, 1e-3, 1)
    oc = viv_oracle_case(mesh, RE, USTAR, DT, u0)
    M = viv.Mesh(mesh)
    case = viv.viv_case(M, RE, USTAR, DT, u0, precision=precision, pivoting=pivoting,
                        jacobian_fp32=jacobian_fp32)
    return mesh, oc, M, case


def _mid_step_state(viv, oc, case, seed):
    """U^{n-1}, U^n and a Newton iterate, identical on both sides."""
    seeded_state(oc, seed, 0.5)
    prev = copy_state(oc)
    seeded_state(oc, seed + 1, 0.7)
    cur = copy_state(oc)
    seeded_state(oc, seed + 2, 1.0)
    it = copy_state(oc)
    push_state(case, cur)
    case.set_history(prev["u"], prev["x"])
    case.begin_step()
    push_state(case, it)
    oc.u_n, oc.x_n = cur["u"], cur["x"]
    oc.hist = (prev["u"], prev["x"])
    for k, v in it.items():
        setattr(oc, k, v.copy())
    c0, hu, hx = oc.bdf_coefficients()
    return c0, hu, hx


@pytest.mark.parametrize("m", [4, 12])
def test_residual_and_jacobian_entrywise(viv, m):
    mesh, oc, M, case = _pair(viv, m, viv.VIV_FP64)
    c0, hu, hx = _mid_step_state(viv, oc, case, 11)
    perm = perm_oracle_to_lib(oc, M)
    nr = case.assemble(viv.VIV_RES | viv.VIV_JAC)
    R_o = oc.residual(c0, hu, hx, DT)
    R_g = case.residual()[perm]
    scale = np.abs(R_o).max()
    assert np.abs(R_g - R_o).max() <= 1e-12 * scale
    assert abs(nr - np.linalg.norm(R_o)) <= 1e-12 * np.linalg.norm(R_o)
    J_o = oc.jacobian(c0, hu, hx, DT).tocsr()
    rp, col = M.pattern()
    vals = case.jacobian_values()
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    rows = np.repeat(np.arange(M.n_dofs), np.diff(rp))
    J_g_in_o = np.asarray(J_o[inv[rows], inv[col]]).ravel()
    jscale = np.abs(J_o.data).max()
    err = np.abs(vals - J_g_in_o)
    assert err.max() <= 1e-11 * jscale, (err.max(), jscale, rows[err.argmax()], col[err.argmax()])
    # every oracle entry is inside the library's pattern (checked on the host too)
    assert abs(np.abs(J_o).sum() - np.abs(J_g_in_o).sum()) <= 1e-9 * np.abs(J_o).sum()


@pytest.mark.parametrize("m", [4, 12])
def test_jacobian_fp32_volume_entrywise(viv, m):
    """Mixed path with FP32 volume-element Jacobians: the Gamma-face and border
    entries (multiplier and cylinder-position rows and columns) stay FP64; the
    volume entries carry FP32 evaluation error only."""
    mesh, oc, M, case = _pair(viv, m, viv.VIV_MIXED, jacobian_fp32=1)
    c0, hu, hx = _mid_step_state(viv, oc, case, 11)
    perm = perm_oracle_to_lib(oc, M)
    case.assemble(viv.VIV_RES | viv.VIV_JAC)
    J_o = oc.jacobian(c0, hu, hx, DT).tocsr()
    rp, col = M.pattern()
    vals = case.jacobian_values()
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    rows = np.repeat(np.arange(M.n_dofs), np.diff(rp))
    J_g_in_o = np.asarray(J_o[inv[rows], inv[col]]).ravel()
    _, field = M.dof_labels()
    # face and border entries: multiplier and cylinder-position rows, multiplier
    # columns (the position columns of velocity and pressure rows are volume
    # shape-derivative entries)
    fb = np.isin(field[rows], [5, 6, 7, 8]) | np.isin(field[col], [5, 6])
    err = np.abs(vals - J_g_in_o)
    jscale = np.abs(J_o.data).max()
    assert err[fb].max() <= 1e-11 * jscale
    row_scale = np.maximum(np.maximum.reduceat(np.abs(J_g_in_o), rp[:-1]), 1e-300)[rows]
    rel = err[~fb] / row_scale[~fb]
    assert rel.max() <= 1e-4, rel.max()
    assert np.median(rel) <= 1e-6, np.median(rel)


@pytest.mark.parametrize("pivoting", ["threshold", "window"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("m", [4, 12])
def test_refined_multifrontal_solve(viv, m, precision, pivoting):
    prec = viv.VIV_FP64 if precision == "fp64" else viv.VIV_MIXED
    piv = viv.VIV_PIVOT_THRESHOLD if pivoting == "threshold" else viv.VIV_PIVOT_WINDOW
    mesh, oc, M, case = _pair(viv, m, prec, pivoting=piv)
    c0, hu, hx = _mid_step_state(viv, oc, case, 21)
    perm = perm_oracle_to_lib(oc, M)
    case.assemble(viv.VIV_RES | viv.VIV_JAC)
    case.factor()
    b = np.random.default_rng(5).standard_normal(M.n_dofs)
    y, sweeps = case.solve_rhs(b)
    J_o = oc.jacobian(c0, hu, hx, DT).tocsc()
    y_o = spla.splu(J_o).solve(b[perm])
    assert rel_l2(y[perm], y_o) <= 1e-10, (rel_l2(y[perm], y_o), sweeps)
    if prec == viv.VIV_MIXED:
        assert sweeps >= 2


@pytest.mark.parametrize("precision,pivoting", [("fp64", "threshold"), ("mixed", "window"), ("mixed", "threshold")])
@pytest.mark.parametrize("m", [4, 12])
def test_border_schur_block(viv, m, precision, pivoting):
    """The cylinder position is eliminated after the fronts as a dense FP64
    block (Eq. coupling_constraint): S_b = D - C A^{-1} B, with A the Jacobian
    without the two delta rows and columns.  Reference: the definition, with
    the oracle's Jacobian and a library sparse LU of its A.  The FP64 path
    agrees to 1e-10; the mixed path's A^{-1} B comes from FP32 factors, so
    its block carries their error (<= 1e-4), and the refined solve (tested
    above) recovers full accuracy."""
    prec = viv.VIV_FP64 if precision == "fp64" else viv.VIV_MIXED
    piv = viv.VIV_PIVOT_THRESHOLD if pivoting == "threshold" else viv.VIV_PIVOT_WINDOW
    mesh, oc, M, case = _pair(viv, m, prec, pivoting=piv)
    c0, hu, hx = _mid_step_state(viv, oc, case, 41)
    case.assemble(viv.VIV_RES | viv.VIV_JAC)
    case.factor()
    S = case.border_block()
    J = oc.jacobian(c0, hu, hx, DT).tocsr()
    d = np.asarray(oc.dof_d)
    a = np.setdiff1d(np.arange(oc.ndof), d)
    A = J[a][:, a].tocsc()
    B = J[a][:, d].toarray()
    C = J[d][:, a].toarray()
    D = J[d][:, d].toarray()
    S_o = D - C @ spla.splu(A).solve(B)
    err = np.abs(S - S_o).max() / np.abs(S_o).max()
    assert err <= (1e-10 if precision == "fp64" else 1e-4), (err, S, S_o)


def _compare_fields(oc, st, tol_field=1e-9, tol_delta=1e-8):
    verts = oc.is_vertex
    errs = dict(u=rel_l2(st["u"], oc.u), p=rel_l2(st["p"][verts], oc.p[verts]), x=rel_l2(st["x"], oc.x),
                lam=rel_l2(st["lam"][oc.cyl], oc.lam[oc.cyl]),
                delta=np.abs(st["delta"] - oc.delta).max())
    assert errs["u"] <= tol_field and errs["p"] <= tol_field and errs["x"] <= tol_field, errs
    assert errs["lam"] <= tol_field and errs["delta"] <= tol_delta, errs
    return errs


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_steps_match_oracle_small_mesh(viv, precision):
    prec = viv.VIV_FP64 if precision == "fp64" else viv.VIV_MIXED
    mesh, oc, M, case = _pair(viv, 4, prec)
    for s in range(4):
        norms = oc.step()
        info = case.step()
        assert info["res_norm"] <= 1e-10
        _compare_fields(oc, case.get_state())
        assert np.allclose(info["force"], oc.force(), atol=1e-8)


@pytest.fixture(scope="module")
def cylinder_reference():
    """Oracle run of the 1,552-quad cylinder case (Re 100, U* 8, dt 0.1):
    states after each of its 10 steps."""
    mesh = I.viv_cylinder_mesh(12)
    u0 = I.viv_initial_velocity(mesh, 1.0, 1e-3, 1)
    oc = viv_oracle_case(mesh, RE, USTAR, DT, u0)
    states = []
    for s in range(10):
        oc.step()
        states.append(copy_state(oc))
    return mesh, oc, states


@pytest.mark.parametrize("precision,pivoting,jac32,pred,reuse", [
    ("fp64", "threshold", 0, 0, 0), ("mixed", "threshold", 0, 0, 0), ("fp64", "window", 0, 0, 0),
    ("mixed", "window", 0, 0, 0), ("mixed", "window", 1, 0, 0), ("mixed", "window", 1, 1, 0),
    ("mixed", "window", 1, 1, 1)])
def test_cylinder_ten_steps_match_oracle(viv, cylinder_reference, precision, pivoting, jac32, pred, reuse):
    mesh, oc, states = cylinder_reference
    prec = viv.VIV_FP64 if precision == "fp64" else viv.VIV_MIXED
    piv = viv.VIV_PIVOT_THRESHOLD if pivoting == "threshold" else viv.VIV_PIVOT_WINDOW
    u0 = I.viv_initial_velocity(mesh, 1.0, 1e-3, 1)
    M = viv.Mesh(mesh)
    case = viv.viv_case(M, RE, USTAR, DT, u0, precision=prec, pivoting=piv, jacobian_fp32=jac32, predictor=pred,
                        factor_reuse=reuse)
    reused = 0
    for s in range(10):
        info = case.step()
        reused += info["reused_factor_solves"]
        assert info["res_norm"] <= 1e-10
        st = case.get_state()
        ref = states[s]
        for k, v in ref.items():
            setattr(oc, k, v)
        _compare_fields(oc, st)
    if reuse:   # the reuse did happen (later Newton iterations solved with the first iterate's factors)
        assert reused >= 5


def test_large_front_threshold_and_level_profile(viv):
    """The same refined solution whatever the large-front threshold (outer
    blocks on the tensor cores for every front of order >= 96, for fronts of
    order >= 256, or for none), and a per-level profile that splits the
    factorisation and solve times by tree level and kind."""
    mesh, oc, M, case = _pair(viv, 12, viv.VIV_MIXED, pivoting=viv.VIV_PIVOT_WINDOW)
    _mid_step_state(viv, oc, case, 31)
    case.assemble(viv.VIV_RES | viv.VIV_JAC)
    b = np.random.default_rng(9).standard_normal(M.n_dofs)
    levels = int(M.fronts()["level"].max()) + 1
    fact_kinds = ("front_assemble", "panel_lu", "trsm", "schur_gemm", "tc_schur_gemm", "tc_split")
    ys = {}
    for bf in (96, 1 << 30, 256):
        case.set_big_front(bf)
        case.profile(True)
        case.factor()
        ys[bf], _ = case.solve_rhs(b)
        kinds = case.profile_read()
        lv = case.profile_levels()
        case.profile(False)
        assert len(lv) == levels
        for group in (fact_kinds, ("fwd_solve", "bwd_solve")):
            per_level = sum(v for d in lv for k, v in d.items() if k in group)
            per_kind = sum(kinds[k][0] for k in group if k in kinds)
            assert 0 < per_level <= per_kind * (1 + 1e-9) + 1e-9, group
        uses_tc = any("tc_schur_gemm" in d for d in lv)
        assert uses_tc == (bf != 1 << 30)
        assert uses_tc == any("tc_split" in d for d in lv)   # every tensor-core update splits its operands
    for bf in (1 << 30, 256):
        assert rel_l2(ys[bf], ys[96]) <= 1e-10, (bf, rel_l2(ys[bf], ys[96]))


def test_autotune_per_level_keeps_the_solution(viv):
    """The autotuner's choices (large-front threshold, then per tree level the
    block LU or the per-panel kernels for the level's large fronts, windowed
    FP32 schedule) change the factorisation's path, not the refined solution:
    the same right-hand side solves to 1e-10 before and after, the mask of
    block-LU levels stays within the tree, and forcing the block LU on every
    level or on none (viv_set_block_levels) gives the same solution too."""
    mesh, oc, M, case = _pair(viv, 12, viv.VIV_MIXED, pivoting=viv.VIV_PIVOT_WINDOW)
    _mid_step_state(viv, oc, case, 41)
    case.assemble(viv.VIV_RES | viv.VIV_JAC)
    b = np.random.default_rng(11).standard_normal(M.n_dofs)
    case.factor()
    y0, _ = case.solve_rhs(b)
    bf, ms = case.autotune()
    assert bf > 0 and ms > 0
    info = M.refresh_info()
    assert 0 <= info["block_level_mask"] < (1 << info["n_levels"])
    case.factor()
    y1, _ = case.solve_rhs(b)
    assert rel_l2(y1, y0) <= 1e-10, rel_l2(y1, y0)
    # every level on the block LU, then none (viv_set_block_levels): same solution
    for mask in (-1, 0):
        case.set_block_levels(mask)
        info = M.refresh_info()
        assert info["block_level_mask"] == ((1 << info["n_levels"]) - 1 if mask < 0 else 0)
        case.factor()
        y2, _ = case.solve_rhs(b)
        assert rel_l2(y2, y0) <= 1e-10, (mask, rel_l2(y2, y0))
