"""Adaptive time stepping (Section 6: start at dt = 0.01, then steps sized for
a target Courant number of 1) with variable-step BDF2, through the C ABI,
against the oracle running the same step-size control."""
import numpy as np
import pytest

from paper_2609_31477_b300 import inputs as I
from oracle.solver import viv_oracle_case

from gpu_common import rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,pivoting,jac32,pred", [("fp64", 0, 0, 0), ("mixed", 1, 1, 1)])
def test_adaptive_steps_match_oracle(precision, pivoting, jac32, pred):
    from paper_2609_31477_b300 import build, viv
    build.build()
    viv.load()
    mesh = I.viv_cylinder_mesh(6)
    u0 = I.viv_initial_velocity(mesh, 1.0, 1e-3, 5)
    oc = viv_oracle_case(mesh, 150.0, 6.0, 0.01, u0)
    M = viv.Mesh(mesh)
    prec = viv.VIV_FP64 if precision == "fp64" else viv.VIV_MIXED
    case = viv.viv_case(M, 150.0, 6.0, 0.01, u0, precision=prec, pivoting=pivoting, jacobian_fp32=jac32,
                        predictor=pred, cfl_target=1.0, dt_max=0.08)
    dts = []
    for s in range(8):
        _, dt_o, cfl_o = oc.step_adaptive(1.0, dt_max=0.08)
        info = case.step()
        assert info["res_norm"] <= 1e-10
        assert abs(info["dt"] - dt_o) <= 1e-12 * dt_o, (s, info["dt"], dt_o)
        assert abs(info["cfl"] - cfl_o) <= 1e-9 * cfl_o, (s, info["cfl"], cfl_o)
        assert abs(info["t"] - oc.t) <= 1e-12
        dts.append(info["dt"])
    # the steps grew from 0.01 (growth capped at 1.2 per step) and vary
    assert dts[0] == 0.01 and len(set(np.round(dts, 12))) > 3
    st = case.get_state()
    v = oc.is_vertex
    assert rel_l2(st["u"], oc.u) <= 1e-9 and rel_l2(st["x"], oc.x) <= 1e-9
    assert rel_l2(st["p"][v], oc.p[v]) <= 1e-9 and rel_l2(st["lam"][oc.cyl], oc.lam[oc.cyl]) <= 1e-9
    assert np.abs(st["delta"] - oc.delta).max() <= 1e-8
    case.close()
    M.close()
