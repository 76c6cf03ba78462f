"""Serving loop: a case gives the same result alone and in a mix of
concurrent cases; admission respects the memory budget; a failing case does
not affect the others; Poisson arrivals complete with latency statistics."""
import numpy as np
import pytest

from paper_2609_31477_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2609_31477_b300 import build, viv
    build.build()
    viv.load()
    meshes = {m: I.viv_cylinder_mesh(m) for m in (4, 6, 8)}
    dev = {m: viv.Mesh(meshes[m]) for m in meshes}
    return viv, meshes, dev


def _u0(mesh, seed):
    return I.viv_initial_velocity(mesh, 1.0, 1e-3, seed)


def test_alone_and_in_the_mix_match(env):
    viv, meshes, dev = env
    budget = 4 << 30
    alone = viv.Server(budget, max_active=1)
    rid = alone.submit(dev[6], _u0(meshes[6], 3), Re=150.0, Ustar=6.0, dt=0.05, n_steps=4)
    res = alone.wait_all(1)
    assert res[0]["status"] == "OK", res
    ref = alone.state(rid, len(meshes[6]["X"]))
    alone.close()
    mix = viv.Server(budget, max_active=6)
    others = []
    for k, (m, Re, Us) in enumerate([(4, 100.0, 8.0), (8, 250.0, 12.0), (4, 300.0, 4.0), (6, 120.0, 9.0)]):
        others.append(mix.submit(dev[m], _u0(meshes[m], 10 + k), Re=Re, Ustar=Us, dt=0.05, n_steps=4))
    rid2 = mix.submit(dev[6], _u0(meshes[6], 3), Re=150.0, Ustar=6.0, dt=0.05, n_steps=4)
    res = mix.wait_all(5)
    assert all(r["status"] == "OK" for r in res), res
    got = mix.state(rid2, len(meshes[6]["X"]))
    st = mix.stats()
    mix.close()
    assert st["peak_active"] >= 2                     # cases really overlapped
    for k in ("u", "p", "x", "lam", "delta"):
        scale = max(1.0, np.abs(ref[k]).max())
        assert np.abs(got[k] - ref[k]).max() <= 1e-12 * scale, k


def test_admission_budget_and_fault_isolation(env):
    viv, meshes, dev = env
    one = dev[6].info["device_bytes_mixed"]
    srv = viv.Server(int(1.5 * one), max_active=8)    # room for one case of this size at a time
    ids = [srv.submit(dev[6], _u0(meshes[6], s), Re=100.0, Ustar=8.0, dt=0.05, n_steps=2) for s in range(3)]
    bad_u0 = _u0(meshes[4], 1)
    bad_u0[5, 0] = np.nan
    bad = srv.submit(dev[4], bad_u0, Re=100.0, Ustar=8.0, dt=0.05, n_steps=2)
    big = srv.submit(dev[8], _u0(meshes[8], 1), Re=100.0, Ustar=8.0, dt=0.05, n_steps=2,
                     precision=viv.VIV_FP64)      # predicted bytes exceed the budget
    res = {r["id"]: r for r in srv.wait_all(5)}
    st = srv.stats()
    srv.close()
    assert all(res[i]["status"] == "OK" and res[i]["steps_done"] == 2 for i in ids), res
    assert res[bad]["status"] == "ERR_NONFINITE"
    assert res[big]["status"] == "ERR_ADMISSION"
    assert st["peak_bytes"] <= int(1.5 * one)


def test_poisson_arrivals_report_latency(env):
    viv, meshes, dev = env
    rng = np.random.default_rng(7)
    arrivals = np.cumsum(rng.exponential(0.05, size=8))
    srv = viv.Server(8 << 30, max_active=4)
    for k, a in enumerate(arrivals):
        m = (4, 6, 8)[k % 3]
        Re = rng.uniform(100, 300)
        Us = float(np.exp(rng.uniform(np.log(4), np.log(20))))
        srv.submit(dev[m], _u0(meshes[m], k), Re=Re, Ustar=Us, dt=0.05, n_steps=3, arrival_time=float(a))
    res = srv.wait_all(8)
    st = srv.stats()
    srv.close()
    assert len(res) == 8 and all(r["status"] == "OK" for r in res)
    assert st["steps"] == 24 and 0 < st["step_ms_p50"] <= st["step_ms_p99"]
    assert 0 < st["steady_ms_p50"] <= st["steady_ms_p99"] <= st["step_ms_p99"]
    assert all(r["admit_s"] >= r["submit_s"] - 1e-6 for r in res)


def test_served_cases_match_the_oracle(env):
    """Cases of a served mix (different meshes, Re and U*, overlapping on the
    device) each equal the oracle's run of the same case: fields to 1e-9
    relative L2, delta to 1e-8."""
    from oracle.solver import viv_oracle_case
    viv, meshes, dev = env
    cases = [(4, 120.0, 5.0, 21), (6, 260.0, 15.0, 22), (4, 180.0, 9.0, 23)]
    srv = viv.Server(4 << 30, max_active=3)
    ids = [srv.submit(dev[m], _u0(meshes[m], seed), Re=Re, Ustar=Us, dt=0.05, n_steps=3,
                      pivoting=viv.VIV_PIVOT_WINDOW, jacobian_fp32=1, predictor=1)
           for m, Re, Us, seed in cases]
    res = {r["id"]: r for r in srv.wait_all(len(cases))}
    st = srv.stats()
    got = [srv.state(i, len(meshes[m]["X"])) for i, (m, _, _, _) in zip(ids, cases)]
    srv.close()
    assert all(res[i]["status"] == "OK" for i in ids), res
    assert st["peak_active"] >= 2
    for (m, Re, Us, seed), g in zip(cases, got):
        oc = viv_oracle_case(meshes[m], Re, Us, 0.05, _u0(meshes[m], seed))
        for _ in range(3):
            oc.step()
        v = oc.is_vertex
        rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
        errs = (rel(g["u"], oc.u), rel(g["p"][v], oc.p[v]), rel(g["x"], oc.x), rel(g["lam"][oc.cyl], oc.lam[oc.cyl]))
        assert max(errs) <= 1e-9, (m, Re, Us, errs)
        assert np.abs(g["delta"] - oc.delta).max() <= 1e-8


def test_newton_failure_stays_inside_its_case(env):
    """A case whose Newton iteration cannot reach the tolerance in its
    iteration limit (max_newton = 1 from the previous time level) fails with
    VIV_ERR_NEWTON; the cases served beside it finish normally."""
    viv, meshes, dev = env
    srv = viv.Server(4 << 30, max_active=4)
    good = [srv.submit(dev[m], _u0(meshes[m], 30 + m), Re=150.0, Ustar=7.0, dt=0.05, n_steps=3) for m in (4, 6)]
    bad = srv.submit(dev[6], _u0(meshes[6], 40), Re=150.0, Ustar=7.0, dt=0.05, n_steps=3, max_newton=1)
    res = {r["id"]: r for r in srv.wait_all(3)}
    srv.close()
    assert res[bad]["status"] == "ERR_NEWTON" and res[bad]["steps_done"] == 0, res[bad]
    assert "Newton did not converge" in res[bad]["message"]
    for i in good:
        assert res[i]["status"] == "OK" and res[i]["steps_done"] == 3, res[i]
