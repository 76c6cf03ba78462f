"""Manufactured-solution verification through the CUDA path (Section 5.1):
the steady 2-D velocity/pressure on a statically deformed unit square,
Q2-Q1 with a Q2 position, both precisions.  The GPU solution equals the
oracle's discrete solution, and its errors fall at the optimal rates."""
import numpy as np
import pytest

from paper_2609_31477_b300 import inputs as I
from oracle import mms
from oracle.solver import OracleCase

from gpu_common import rel_l2

pytestmark = pytest.mark.gpu
AMP = 0.05


def _oracle(sol, n):
    m = I.square_mesh(n)
    m["tags"][0] |= I.P_FIX
    c = OracleCase(m, rho=sol.rho, mu=sol.mu, k=0.0, dt=1e8, u0=np.zeros((len(m["X"]), 2)), lame=1.0, src=sol)
    c.x[:] = c.X
    sol.set_dirichlet(c, 0.0)
    c.step(dirichlet=sol.set_dirichlet)
    return m, c


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_steady_mms_matches_oracle_and_converges(precision):
    import torch
    from paper_2609_31477_b300 import build, viv
    build.build()
    viv.load()
    prec = viv.VIV_FP64 if precision == "fp64" else viv.VIV_MIXED
    sol = mms.steady_mms(amp=AMP)
    errs = []
    for n in (8, 16):
        m, oc = _oracle(sol, n)
        # initial state: exact velocity on the boundary, the pinned pressure
        u0 = np.zeros((len(m["X"]), 2))
        fixed = (m["tags"] & I.ALL_DIRICHLET_TAG) != 0
        u0[fixed] = sol.velocity(m["X"], 0.0)[fixed]
        p0 = np.zeros(len(m["X"]))
        p0[0] = sol.pressure(m["X"][:1], 0.0)[0]
        M = viv.Mesh(m)
        case = viv.Case(M, u0, sol.rho, sol.mu, 0.0, 1e8, precision=prec, lame_scale=1.0, source=1, source_amp=AMP)
        case.set_state(p=p0)
        info = case.step()
        assert info["res_norm"] <= 1e-10
        st = case.get_state()
        v = oc.is_vertex
        assert rel_l2(st["u"], oc.u) <= 1e-9
        assert rel_l2(st["p"][v], oc.p[v]) <= 1e-9
        assert rel_l2(st["x"], oc.x) <= 1e-9
        # errors of the GPU state against the exact fields
        oc.u, oc.p, oc.x = st["u"], st["p"], st["x"]
        errs.append(mms.error_norms(oc, sol, oc.t))
        case.close()
        M.close()
    r = {k: np.log2(errs[0][k] / errs[1][k]) for k in errs[0]}
    assert abs(r["u_l2"] - 3) < 0.2 and abs(r["u_h1"] - 2) < 0.15, r
    assert abs(r["x_l2"] - 3) < 0.2 and abs(r["x_h1"] - 2) < 0.15, r
    assert r["p_l2"] > 1.7, r
