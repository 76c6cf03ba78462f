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


def test_variable_step_bdf2_exact_and_second_order():
    """Variable-step BDF2 (the adaptive time stepping of Section 6): the nodal
    trajectories of the translating box are quadratic in time, so any
    sequence of step sizes must reproduce the exact solution to rounding; with
    the cubic time factor the error must fall by 4 when every step of a
    varying sequence is halved."""
    sol = mms.translating_box()
    seq = [0.05, 0.065, 0.04, 0.055, 0.03, 0.06]   # step ratios 1.3, 0.62, 1.38, 0.55, 2
    c = _box_case(sol, 10, seq[0])
    c.dt_prev = seq[0]   # the history level of _box_case lies one seq[0] back
    for dt in seq:
        c.dt = dt
        c.step(dirichlet=sol.set_dirichlet)
        t = c.t
        assert np.abs(c.u - sol.velocity(c.X, t)).max() < 1e-11
        assert np.abs(c.x - sol.position(c.X, t)).max() < 1e-12
        assert np.abs(c.p - sol.pressure(c.X, t))[c.is_vertex].max() < 1e-8
    sol3 = mms.translating_box(gamma=3.0)
    errs = []
    for scale in (1.0, 0.5, 0.25):
        steps = [s * scale for s in (0.05, 0.07, 0.04, 0.06) for _ in range(int(round(1 / scale)))]
        c = _box_case(sol3, 5, steps[0])
        c.dt_prev = steps[0]
        for dt in steps:
            c.dt = dt
            c.step(dirichlet=sol3.set_dirichlet)
        errs.append(np.abs(c.u - sol3.velocity(c.X, c.t)).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.85) and np.all(rates < 2.3), rates


def test_courant_number_and_step_control():
    """The Courant number of a uniform flow U on a uniform n x n mesh is
    dt U n (shortest edge 1/n); the step control moves dt towards the target
    within a factor 1/2 .. 1.2 per step and below dt_max."""
    m = I.square_mesh(8)
    c = OracleCase(m, rho=1.0, mu=0.01, k=0.0, dt=0.01, u0=np.tile([0.6, 0.8], (len(m["X"]), 1)), lame=1.0)
    assert abs(c.cfl() - 0.01 * 1.0 * 8) < 1e-14
    assert abs(c.next_dt(0.08, 1.0) - 0.012) < 1e-15        # growth capped at 1.2
    assert abs(c.next_dt(0.08, 0.09) - 0.01 * 0.09 / 0.08) < 1e-15
    assert abs(c.next_dt(0.08, 0.01) - 0.005) < 1e-15       # shrink capped at 1/2
    assert abs(c.next_dt(0.08, 1.0, dt_max=0.011) - 0.011) < 1e-15


def _quasi_case(sol, n, dt):
    m = I.hole_square_mesh(n)
    m["tags"][np.argmin(m["X"][:, 0] + m["X"][:, 1])] |= I.P_FIX   # a corner vertex, where p = 0
    c = OracleCase(m, rho=sol.rho, mu=sol.mu, k=sol.k, dt=dt, u0=np.zeros((len(m["X"]), 2)), lame=1.0, src=sol)
    sol.set_exact_state(c, 0.0)
    return c


def test_quasi_mms_pressure_carries_the_spring_force():
    """Section 5.2: on the rigid cylinder the manufactured velocity gradient
    vanishes, so the multiplier is the pressure times the normal and
    int_Gamma lambda = int_Gamma p e ds; with p = -k f (d.e) psi / (pi R0) this
    is -k f d, which is what the coupling row k delta + int_Gamma lambda = 0
    needs with delta = f d.  Quadrature on the exact moved circle."""
    sol = mms.QuasiMMS()
    th = np.linspace(0.0, 2 * np.pi, 2001)[:-1]
    e = np.stack([np.cos(th), np.sin(th)], 1)
    for t in (0.05, 0.1, 0.2):
        xc = np.array(mms.QUASI_CENTER) + np.sin(2 * np.pi * t) * sol.d
        x = xc + mms.QUASI_R0 * e
        pl = sol._p_phys(x[:, 0], x[:, 1], t)
        grad = sol._grad_u_phys(x[:, 0], x[:, 1], t)
        assert np.abs(grad).max() < 1e-12
        integral = (pl[:, None] * e).sum(0) * mms.QUASI_R0 * (2 * np.pi / len(th))
        assert np.allclose(sol.k * sol.delta(t) + integral, 0.0, atol=1e-12)
        # the cylinder moves rigidly with the manufactured velocity
        X = np.array(mms.QUASI_CENTER) + mms.QUASI_R0 * e
        assert np.allclose(sol.position(X, t) - X, sol.delta(t), atol=1e-14)


def test_quasi_mms_converges_under_joint_refinement():
    """Mesh and step halved together (4 -> 8 cells radially, dt 0.02 -> 0.01,
    to t = 0.1): the cylinder displacement (and so the fluid force k delta) and
    the velocity converge at least at second order."""
    sol = mms.QuasiMMS()
    errs = []
    for n, dt in ((4, 0.02), (8, 0.01)):
        c = _quasi_case(sol, n, dt)
        for _ in range(int(round(0.1 / dt))):
            c.step(dirichlet=sol.set_dirichlet)
        e = mms.error_norms(c, sol, c.t)
        e["delta"] = np.abs(c.delta - sol.delta(c.t)).max()
        assert np.allclose(c.force(), sol.k * c.delta, atol=1e-10)
        errs.append(e)
    assert errs[0]["delta"] / errs[1]["delta"] > 3.5, errs
    assert errs[0]["u_l2"] / errs[1]["u_l2"] > 3.5, errs
