"""Physics sanity of the fast path (force coefficients and Strouhal number):
a fixed cylinder (stiff spring, k = 1e6) at Re 200 on the 1,552-quad mesh,
dt 0.05 on the mixed path as the benchmark runs it, to t = 100.  Vortex
shedding sets in from the seeded noise; over t >= 60 the drag, the lift
amplitude and the shedding frequency are those the paper reports for this
Reynolds number (Section 5.3: C_D = 1.398 +- 0.0497, C_L +- 0.723,
St = 0.199, on its own, larger mesh and domain), within bands that allow for
the smaller channel here."""
import numpy as np
import pytest

from paper_2609_31477_b300 import inputs as I

pytestmark = pytest.mark.gpu


def test_fixed_cylinder_re200_shedding():
    from paper_2609_31477_b300 import build, viv
    build.build()
    viv.load()
    mesh = I.viv_cylinder_mesh(12)
    u0 = I.viv_initial_velocity(mesh, 1.0, 1e-3, 1)
    M = viv.Mesh(mesh)
    Re, dt = 200.0, 0.05
    case = viv.Case(M, u0, 1.0, 1.0 / Re, 1e6, dt, precision=viv.VIV_MIXED, pivoting=viv.VIV_PIVOT_WINDOW,
                    jacobian_fp32=1, predictor=1)
    ts, F = [], []
    for _ in range(int(round(100.0 / dt))):
        info = case.step()
        assert info["res_norm"] <= 1e-10
        ts.append(info["t"])
        F.append(info["force"])
        # held by the stiff spring: delta = F / k (the start-up force reaches ~18)
        assert np.allclose(np.array(info["delta"]) * 1e6, info["force"], rtol=1e-6, atol=1e-9)
        assert max(abs(info["delta"][0]), abs(info["delta"][1])) < 1e-4
    case.close()
    M.close()
    r = viv.force_analysis(np.array(ts), np.array(F), rho=1.0, U=1.0, D=1.0, t_start=60.0)
    print(r)
    assert abs(r["strouhal"] - 0.199) < 0.01, r
    assert abs(r["cd_mean"] - 1.398) < 0.1, r
    assert abs(r["cl_amp"] - 0.723) < 0.08, r
    assert abs(r["cl_mean"]) < 0.02, r
