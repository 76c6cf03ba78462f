"""The coupled quasi-manufactured solution of Section 5.2 through the CUDA
path: a rigid cylinder of radius 0.15 in the unit square, moved by the
fluid force through the spring (k = 10); the manufactured pressure carries
exactly the force the coupling needs, so the multiplier and coupling rows
take no source.  The GPU state equals the oracle's, and under joint mesh and
step refinement the cylinder displacement - and so the fluid force k delta -
converges at second order (the paper's observation for the forces)."""
import numpy as np
import pytest

from paper_2609_31477_b300 import inputs as I
from oracle import mms
from oracle.solver import OracleCase

from gpu_common import rel_l2

pytestmark = pytest.mark.gpu


def _mesh(n):
    m = I.hole_square_mesh(n)
    m["tags"][np.argmin(m["X"][:, 0] + m["X"][:, 1])] |= I.P_FIX
    return m


def _gpu_run(viv, sol, n, dt, prec, T=0.1, pivoting=0):
    m = _mesh(n)
    M = viv.Mesh(m)
    case = viv.Case(M, np.zeros((len(m["X"]), 2)), sol.rho, sol.mu, sol.k, dt, precision=prec, lame_scale=1.0,
                    lame_constant=1, source=3, source_amp=sol.amp, pivoting=pivoting)
    for _ in range(int(round(T / dt))):
        info = case.step()
        assert info["res_norm"] <= 1e-10
    st = case.get_state()
    case.close()
    M.close()
    return m, st, info


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_quasi_mms_matches_oracle(precision):
    from paper_2609_31477_b300 import build, viv
    build.build()
    viv.load()
    sol = mms.QuasiMMS()
    prec = viv.VIV_FP64 if precision == "fp64" else viv.VIV_MIXED
    m, st, info = _gpu_run(viv, sol, 6, 0.02, prec)
    oc = OracleCase(m, rho=sol.rho, mu=sol.mu, k=sol.k, dt=0.02, u0=np.zeros((len(m["X"]), 2)), lame=1.0, src=sol)
    sol.set_exact_state(oc, 0.0)
    for _ in range(5):
        oc.step(dirichlet=sol.set_dirichlet)
    v = oc.is_vertex
    assert rel_l2(st["u"], oc.u) <= 1e-9 and rel_l2(st["x"] - oc.X, oc.x - oc.X) <= 1e-9
    assert rel_l2(st["p"][v], oc.p[v]) <= 1e-9 and rel_l2(st["lam"][oc.cyl], oc.lam[oc.cyl]) <= 1e-9
    assert np.abs(st["delta"] - oc.delta).max() <= 1e-8 * np.abs(oc.delta).max()
    assert np.allclose(info["force"], oc.force(), atol=1e-9)


def test_quasi_mms_force_second_order():
    from paper_2609_31477_b300 import build, viv
    build.build()
    viv.load()
    sol = mms.QuasiMMS()
    rows = []
    for n, dt in ((8, 0.02), (16, 0.01), (32, 0.005), (64, 0.0025)):
        m, s64, i64 = _gpu_run(viv, sol, n, dt, viv.VIV_FP64)
        _, s32, _ = _gpu_run(viv, sol, n, dt, viv.VIV_MIXED, pivoting=viv.VIV_PIVOT_WINDOW)
        assert rel_l2(s32["u"], s64["u"]) <= 1e-9 and np.abs(s32["delta"] - s64["delta"]).max() <= 1e-10
        c = OracleCase(m, rho=sol.rho, mu=sol.mu, k=sol.k, dt=1.0, u0=np.zeros((len(m["X"]), 2)), lame=1.0, src=sol)
        c.u, c.p, c.x = s64["u"], s64["p"], s64["x"]
        e = mms.error_norms(c, sol, 0.1)
        e["force"] = np.abs(np.array(i64["force"]) - sol.force(0.1)).max()
        rows.append(e)
    order = lambda k: [float(np.log2(rows[i][k] / rows[i + 1][k])) for i in range(len(rows) - 1)]
    print({k: [f"{r[k]:.3e}" for r in rows] for k in rows[0]})
    print({k: [round(o, 2) for o in order(k)] for k in rows[0]})
    assert min(order("force")) > 1.8, order("force")
    assert min(order("u_l2")) > 1.8, order("u_l2")
