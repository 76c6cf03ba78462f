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
        case = viv.Case(M, u0, sol.rho, sol.mu, 0.0, 1e8, precision=prec, lame_scale=1.0, lame_constant=1, source=1, source_amp=AMP)
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


def _unsteady_gpu(viv, sol, n, dt, prec, T=0.2, pivoting=0):
    m = I.square_mesh(n)
    m["tags"][0] |= I.P_FIX
    M = viv.Mesh(m)
    case = viv.Case(M, np.zeros((len(m["X"]), 2)), sol.rho, sol.mu, 0.0, dt, precision=prec, lame_scale=1.0, lame_constant=1,
                    source=2, source_amp=AMP, pivoting=pivoting)
    for _ in range(int(round(T / dt))):
        info = case.step()
        assert info["res_norm"] <= 1e-10
    st = case.get_state()
    case.close()
    M.close()
    return m, st


def _errors(m, sol, st, t):
    c = OracleCase(m, rho=sol.rho, mu=sol.mu, k=0.0, dt=1.0, u0=np.zeros((len(m["X"]), 2)), lame=1.0, src=sol)
    c.u, c.p, c.x = st["u"], st["p"], st["x"]
    return mms.error_norms(c, sol, t)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_unsteady_mms_matches_oracle(precision):
    """Section 5.1's time-dependent solution (u ~ t^3, p ~ t^2, mesh moved by
    sin(pi t)) through the CUDA path: after five BDF steps (BDF1 start) on the
    16 x 16 square the GPU state equals the oracle's discrete solution."""
    from paper_2609_31477_b300 import build, viv
    build.build()
    viv.load()
    sol = mms.unsteady_mms(amp=AMP)
    prec = viv.VIV_FP64 if precision == "fp64" else viv.VIV_MIXED
    m, st = _unsteady_gpu(viv, sol, 16, 0.04, prec)
    oc = OracleCase(m, rho=sol.rho, mu=sol.mu, k=0.0, dt=0.04, u0=np.zeros((len(m["X"]), 2)), lame=1.0, src=sol)
    sol.set_exact_state(oc, 0.0)
    for _ in range(5):
        oc.step(dirichlet=sol.set_dirichlet)
    v = oc.is_vertex
    assert rel_l2(st["u"], oc.u) <= 1e-9
    assert rel_l2(st["p"][v], oc.p[v]) <= 1e-9
    assert rel_l2(st["x"] - oc.X, oc.x - oc.X) <= 1e-9


def _order(e, k):
    return [float(np.log2(e[i][k] / e[i + 1][k])) for i in range(len(e) - 1)]


def test_unsteady_mms_sweep_rates_fp64_vs_mixed():
    """The 2-D manufactured-solution workload: n^2 Q2-Q1 cells on the unit
    square, BDF2 to T = 0.2, FP64 path and mixed path (FP32 fronts, FP64
    refinement).  Three sweeps, errors against the exact fields:
      paired  n = 16, 32, 64, 128 with dt = 0.04, 0.02, 0.01, 0.005
              (dt^2 and h^3 both fall: velocity L2 at least second order);
      space   n = 8, 16, 32 with dt = 0.00025 (time error below the space error):
              u L2 3, u H1 2, x L2 3, x H1 2 (the pressure is reported);
      time    n = 64 with dt = 0.04 ... 0.005: u L2 second order.
    The two precisions give the same states to 1e-9 throughout."""
    from paper_2609_31477_b300 import build, viv
    build.build()
    viv.load()
    sol = mms.unsteady_mms(amp=AMP)
    table = {}
    for name, runs in (("paired", [(16, 0.04), (32, 0.02), (64, 0.01), (128, 0.005)]),
                       ("space", [(8, 0.00025), (16, 0.00025), (32, 0.00025)]),
                       ("time", [(64, 0.04), (64, 0.02), (64, 0.01), (64, 0.005)])):
        errs = []
        for n, dt in runs:
            m, s64 = _unsteady_gpu(viv, sol, n, dt, viv.VIV_FP64)
            _, s32 = _unsteady_gpu(viv, sol, n, dt, viv.VIV_MIXED, pivoting=viv.VIV_PIVOT_WINDOW)
            verts = np.zeros(len(m["X"]), bool)
            verts[np.asarray(m["conn"])[:, [0, 2, 6, 8]].ravel()] = True
            for k in ("u", "x"):
                assert rel_l2(s32[k], s64[k]) <= 1e-9, (name, n, dt, k)
            assert rel_l2(s32["p"][verts], s64["p"][verts]) <= 1e-9, (name, n, dt)
            errs.append(_errors(m, sol, s64, 0.2))
        table[name] = errs
        print(name, [{k: f"{v:.3e}" for k, v in e.items()} for e in errs])
        print(name, "orders", {k: [round(o, 2) for o in _order(errs, k)] for k in errs[0]})
    assert min(_order(table["paired"], "u_l2")) > 1.9
    sp = table["space"]
    assert min(_order(sp, "u_l2")) > 2.5 and min(_order(sp, "u_h1")) > 1.85
    assert min(_order(sp, "x_l2")) > 2.7 and min(_order(sp, "x_h1")) > 1.85
    assert min(_order(table["time"], "u_l2")[:2]) > 1.85
