"""Pins of the oracle's element routines against mathematics that does not
depend on the oracle: polynomial exactness, Kronecker property, exact areas,
the Jacobi-formula area variation of Section 3.2, patch tests and central
finite differences of the residual."""
import numpy as np
import pytest

from paper_2609_31477_b300 import inputs as I
from oracle import fem
from oracle.solver import OracleCase, viv_oracle_case


def test_gauss3_exact_to_degree5():
    for k in range(6):
        assert abs(np.sum(fem.GAUSS3_WTS * fem.GAUSS3_PTS ** k) - 1.0 / (k + 1)) < 1e-15
    assert abs(np.sum(fem.GAUSS3_WTS * fem.GAUSS3_PTS ** 6) - 1.0 / 7) > 1e-6


def test_q2_kronecker_and_partition_of_unity():
    L, dL = fem.lagrange2(np.array([0.0, 0.5, 1.0]))
    assert np.allclose(L, np.eye(3), atol=1e-15)
    N, dN, M, W = fem.q2_tables()
    assert np.allclose(N.sum(1), 1.0) and np.allclose(dN.sum(1), 0.0, atol=1e-14)
    assert np.allclose(M.sum(1), 1.0) and abs(W.sum() - 1.0) < 1e-15


def test_area_exact_on_straight_mesh_and_close_on_cylinder():
    m = I.square_mesh(6, hole=(1.0 / 3.0, 2.0 / 3.0))
    a = fem.element_areas(m["X"][m["conn"]]).sum()
    assert abs(a - (1.0 - 1.0 / 9.0)) < 1e-14
    m = I.viv_cylinder_mesh(12)
    a = fem.element_areas(m["X"][m["conn"]]).sum()
    exact = 30.0 * 20.0 - np.pi * 0.25
    assert abs(a - exact) / exact < 1e-7
    assert np.all(fem.element_areas(m["X"][m["conn"]]) > 0)


def test_area_variation_matches_jacobi_formula():
    """Section 3.2: d/d eps |K(x + eps dx)| = int det J tr(grad_x dx)."""
    rng = np.random.default_rng(0)
    m = I.viv_cylinder_mesh(4)
    xe = m["X"][m["conn"]][:20] + 0.01 * rng.standard_normal((20, 9, 2))
    dx = rng.standard_normal((20, 9, 2))
    cs = fem.element_areas(xe + 1e-30j * dx).imag / 1e-30
    jac = np.zeros(20)
    for q in range(9):
        g, det = fem.physical_gradients(xe, q)
        G = np.matmul(np.swapaxes(dx, 1, 2), g)
        jac += fem.W_Q[q] * det * (G[:, 0, 0] + G[:, 1, 1])
    assert np.allclose(cs, jac, rtol=1e-12, atol=1e-14)


def _small_viv(m=4, dt=0.1, sigma=1e-3):
    mesh = I.viv_cylinder_mesh(m)
    u0 = I.viv_initial_velocity(mesh, 1.0, sigma, 1)
    return viv_oracle_case(mesh, 100.0, 8.0, dt, u0)


def test_uniform_flow_and_rigid_translation_patches():
    c = _small_viv(sigma=0.0)
    rng = np.random.default_rng(1)
    x = c.X + 0.02 * rng.standard_normal(c.X.shape)      # curved, static mesh
    u = np.tile([0.7, -0.3], (c.n, 1))
    c0 = 1.5 / c.dt
    Ru, Rp, Rx, Rl, Rd = c.residual_parts(u, np.zeros(c.n), x, np.zeros((c.n, 2)), np.zeros(2),
                                          c0, -c0 * u, -c0 * x, 0.1)
    assert np.abs(Ru).max() < 1e-12 and np.abs(Rp).max() < 1e-12
    xs = c.X + np.array([0.3, -0.2])
    _, _, Rx, _, _ = c.residual_parts(u, np.zeros(c.n), xs, np.zeros((c.n, 2)), np.zeros(2),
                                      c0, -c0 * u, -c0 * xs, 0.1)
    assert np.abs(Rx).max() < 1e-9 * np.abs(c.lam_s).max()


def test_jacobian_matches_central_differences():
    c = _small_viv()
    rng = np.random.default_rng(2)
    c.u += 0.1 * rng.standard_normal(c.u.shape)
    c.p[:] = rng.standard_normal(c.n)
    c.lam[c.cyl] = rng.standard_normal((c.cyl.sum(), 2))
    U = c.gather()
    U[c.dof_d] = [0.05, -0.03]
    c.scatter(U)
    c.u_n, c.x_n = c.u.copy(), c.x.copy()
    c.hist = (c.u - 0.01, c.x.copy())
    c0, hu, hx = c.bdf_coefficients()
    J = c.jacobian(c0, hu, hx, 0.1)
    for trial in range(3):
        v = rng.standard_normal(c.ndof)
        eps = 1e-6
        c.scatter(U + eps * v); Rp_ = c.residual(c0, hu, hx, 0.1)
        c.scatter(U - eps * v); Rm_ = c.residual(c0, hu, hx, 0.1)
        c.scatter(U)
        fd = (Rp_ - Rm_) / (2 * eps)
        Jv = J @ v
        assert np.linalg.norm(Jv - fd) <= 1e-6 * np.linalg.norm(fd)


def test_block_structure_of_the_jacobian():
    """Section 3.2: zero p-p and lambda-lambda blocks; pseudo-solid rows do not
    depend on u, p or lambda."""
    c = _small_viv()
    c.u_n, c.x_n = c.u.copy(), c.x.copy()
    c0, hu, hx = c.bdf_coefficients()
    J = c.jacobian(c0, hu, hx, 0.1).tocoo()
    kind = np.empty(c.ndof, dtype="<U1")
    kind[c.dof_u[c.dof_u >= 0]] = "u"
    kind[c.dof_p[c.dof_p >= 0]] = "p"
    kind[c.dof_x[c.dof_x >= 0]] = "x"
    kind[c.dof_l[c.dof_l >= 0]] = "l"
    kind[c.dof_d] = "d"
    pairs = set(zip(kind[J.row], kind[J.col]))
    for bad in (("p", "p"), ("l", "l"), ("x", "u"), ("x", "p"), ("x", "l"), ("p", "l")):
        assert bad not in pairs
    for good in (("u", "x"), ("p", "x"), ("u", "l"), ("l", "d"), ("d", "l"), ("x", "d")):
        assert good in pairs
