"""Invariants of converged cylinder steps of the oracle: outflow flux equals
inflow flux, nodal no-slip on Gamma, the zero-mass force balance, mirror
symmetry without noise, Lame-scale invariance, quadratic Newton."""
import numpy as np
import pytest

from paper_2609_31477_b300 import inputs as I
from oracle import fem
from oracle.solver import viv_oracle_case


def _outlet_flux(c):
    flux = 0.0
    for e in range(len(c.conn)):
        for ed in I.EDGE_NODES:
            nodes = c.conn[e, list(ed)]
            if np.all((c.tags[nodes] & I.OUTLET) != 0):
                xf, uf = c.x[nodes], c.u[nodes]
                for q in range(3):
                    N, dN = fem.L_EDGE[q], fem.DL_EDGE[q]
                    tang = dN @ xf
                    flux += fem.GAUSS3_WTS[q] * abs(tang[1]) * (N @ uf)[0]
    return flux


@pytest.fixture(scope="module")
def stepped():
    mesh = I.viv_cylinder_mesh(4)
    u0 = I.viv_initial_velocity(mesh, 1.0, 1e-3, 1)
    c = viv_oracle_case(mesh, 100.0, 8.0, 0.1, u0)
    norms = [c.step() for _ in range(3)]
    return c, norms


def test_flux_balance(stepped):
    c, _ = stepped
    assert abs(_outlet_flux(c) - 20.0) < 1e-9


def test_noslip_force_balance_and_newton(stepped):
    c, norms = stepped
    assert c.cyl.sum() > 0
    assert np.allclose(c.k * c.delta, c.force(), atol=1e-10)
    for ns in norms:
        assert ns[-1] <= 1e-10
        # quadratic convergence: last reduction much stronger than the first
        assert ns[-1] < 1e-3 * ns[-2] ** 1.5 or ns[-1] < 1e-13


def test_noslip_holds_nodally():
    """The lambda rows make u equal the mesh velocity w = d_t(X + delta) at
    every Gamma node (Q2 multiplier against a Q2 trace)."""
    mesh = I.viv_cylinder_mesh(4)
    c = viv_oracle_case(mesh, 100.0, 8.0, 0.1, I.viv_initial_velocity(mesh, 1.0, 1e-3, 1))
    deltas = [c.delta.copy()]
    for _ in range(3):
        c.step()
        deltas.append(c.delta.copy())
    w = (1.5 * deltas[3] - 2.0 * deltas[2] + 0.5 * deltas[1]) / c.dt
    assert np.abs(c.u[c.cyl] - w).max() < 1e-10


def test_mirror_symmetry_without_noise():
    mesh = I.viv_cylinder_mesh(4)
    c = viv_oracle_case(mesh, 100.0, 8.0, 0.1, I.viv_initial_velocity(mesh, 1.0, 0.0, 1))
    c.step(); c.step()
    assert abs(c.delta[1]) < 1e-12
    X = c.X
    key = {(round(a, 9), round(b, 9)): i for i, (a, b) in enumerate(X)}
    mirror = np.array([key[(round(a, 9), round(-b, 9))] for a, b in X])
    assert np.abs(c.u[mirror, 0] - c.u[:, 0]).max() < 1e-10
    assert np.abs(c.u[mirror, 1] + c.u[:, 1]).max() < 1e-10


def test_lame_scale_invariance():
    mesh = I.viv_cylinder_mesh(4)
    u0 = I.viv_initial_velocity(mesh, 1.0, 1e-3, 1)
    a = viv_oracle_case(mesh, 100.0, 8.0, 0.1, u0)
    b = viv_oracle_case(mesh, 100.0, 8.0, 0.1, u0)
    b.lam_s = 37.0 * b.lam_s
    b.mu_s = 37.0 * b.mu_s
    a.step(); b.step()
    assert np.abs(a.u - b.u).max() < 1e-9 and np.abs(a.x - b.x).max() < 1e-10


def test_stiffness_from_reduced_velocity_pins():
    """Section 1 defines the reduced velocity of a massless cylinder as
    U_r = pi U sqrt(pi rho L / k).  The oracle's k must give back U_r = U* through
    that definition, and for the cylinder workloads (rho = U = L = 1) take the
    values the mathematics fixes: U* = 8 -> pi^3/64 = 0.484473..., U* = 10 ->
    pi^3/100 = 0.310063... (a pi^2 for pi^3 slip would give 0.154 and 0.0987)."""
    from oracle.solver import stiffness_from_reduced_velocity as kfun
    assert abs(kfun(1.0, 1.0, 8.0) - 0.48447307) < 5e-9
    assert abs(kfun(1.0, 1.0, 10.0) - 0.31006277) < 5e-9
    for rho, U, Us, L in [(1.0, 1.0, 8.0, 1.0), (2.5, 0.7, 5.5, 6.283185307179586), (1.0, 3.0, 17.0, 2.0)]:
        k = kfun(rho, U, Us, L)
        Ur = np.pi * U * np.sqrt(np.pi * rho * L / k)
        assert abs(Ur - Us) <= 1e-12 * Us
    mesh = I.viv_cylinder_mesh(4)
    c = viv_oracle_case(mesh, 100.0, 8.0, 0.1, I.viv_initial_velocity(mesh, 1.0, 0.0, 1))
    assert abs(c.k - 0.48447307) < 5e-9 and abs(c.mu - 0.01) < 1e-15
