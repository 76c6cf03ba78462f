"""Pins of the oracle's discretisation against exact and manufactured
solutions (Section 5.1): a closed-form solution the scheme must reproduce to
rounding, BDF2 order in time, optimal spatial rates."""
import numpy as np
import pytest

from paper_2609_31477_b300 import inputs as I
from oracle import mms
from oracle.solver import OracleCase


def _box_case(sol, n, dt):
    m = I.square_mesh(n, hole=(0.4, 0.6) if n % 5 == 0 else None)
    m["tags"][0] |= I.P_FIX
    c = OracleCase(m, rho=sol.rho, mu=sol.mu, k=sol.k, dt=dt, u0=np.zeros((len(m["X"]), 2)),
                   lame=1.0, src=sol)
    sol.set_exact_state(c, -dt)
    hist = (c.u.copy(), c.x.copy())
    sol.set_exact_state(c, 0.0)
    c.hist = hist
    return c


def test_translating_box_reproduced_to_rounding():
    sol = mms.translating_box()
    c = _box_case(sol, 10, 0.1)
    for _ in range(3):
        norms = c.step(dirichlet=sol.set_dirichlet)
        t = c.t
        assert norms[-1] <= 1e-10
        assert np.abs(c.u - sol.velocity(c.X, t)).max() < 1e-11
        assert np.abs(c.x - sol.position(c.X, t)).max() < 1e-12
        assert np.abs(c.p - sol.pressure(c.X, t))[c.is_vertex].max() < 1e-8
        assert np.allclose(c.delta, sol.delta(t), atol=1e-13)
        assert np.allclose(c.force(), sol.force(t), atol=1e-11)
        # zero-mass balance of Eq. solid_balance: k delta + int lambda = 0 (no source part)
        assert np.allclose(sol.k * c.delta - c.force(), sol.border(t), atol=1e-10)


def test_bdf2_second_order_in_time():
    sol = mms.translating_box(gamma=3.0)
    errs = []
    for dt in (0.1, 0.05, 0.025):
        c = _box_case(sol, 5, dt)
        for _ in range(round(0.4 / dt)):
            c.step(dirichlet=sol.set_dirichlet)
        errs.append(np.abs(c.u - sol.velocity(c.X, c.t)).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.85) and np.all(rates < 2.2), rates


def test_steady_mms_optimal_rates():
    sol = mms.steady_mms()
    prev = None
    for n in (4, 8, 16):
        m = I.square_mesh(n)
        m["tags"][0] |= I.P_FIX
        c = OracleCase(m, rho=sol.rho, mu=sol.mu, k=0.0, dt=1e8, u0=np.zeros((len(m["X"]), 2)),
                       lame=1.0, src=sol)
        c.x[:] = c.X
        sol.set_dirichlet(c, 0.0)
        c.step(dirichlet=sol.set_dirichlet)
        e = mms.error_norms(c, sol, c.t)
        if prev is not None:
            r = {k: np.log2(prev[k] / e[k]) for k in e}
        prev = e
    assert abs(r["u_l2"] - 3) < 0.15 and abs(r["u_h1"] - 2) < 0.1
    assert abs(r["x_l2"] - 3) < 0.15 and abs(r["x_h1"] - 2) < 0.1
    assert r["p_l2"] > 1.8


def test_unsteady_mms_bdf2_order_in_time():
    """Section 5.1's time-dependent manufactured solution (u ~ t^3, p ~ t^2, mesh
    moved by sin(pi t)): on a fixed 8 x 8 mesh the velocity error falls by 4
    per halving of dt (BDF2), while the position - a quasi-static pseudo-solid
    driven by exact boundary data - does not depend on dt at all."""
    sol = mms.unsteady_mms()
    errs, xs = [], []
    for dt in (0.04, 0.02):
        m = I.square_mesh(8)
        m["tags"][0] |= I.P_FIX
        c = OracleCase(m, rho=sol.rho, mu=sol.mu, k=0.0, dt=dt, u0=np.zeros((len(m["X"]), 2)), lame=1.0, src=sol)
        sol.set_exact_state(c, 0.0)
        for _ in range(int(round(0.2 / dt))):
            c.step(dirichlet=sol.set_dirichlet)
        assert abs(c.t - 0.2) < 1e-12
        errs.append(mms.error_norms(c, sol, c.t))
        xs.append(c.x.copy())
    ratio = errs[0]["u_l2"] / errs[1]["u_l2"]
    assert 3.6 < ratio < 4.4, ratio
    assert np.abs(xs[0] - xs[1]).max() < 1e-12
