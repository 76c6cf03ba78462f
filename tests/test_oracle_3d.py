"""Pins of the oracle's hexahedral routines (oracle/fem3d.py, oracle/solver3d.py)
against what the mathematics fixes, independently of their own code:

* a z-independent state on a periodic extrusion reduces, plane by plane, to
  the pinned 2-D routines times the spanwise integral of the plane's basis
  function (Q2: h/3 on vertex planes, 2h/3 on mid planes; Q1: h), with zero
  z-rows; one Newton step of the 3-D cylinder case from a z-independent state
  equals the 2-D step (the z-constant fields are an invariant subspace);
* the element integrals are covariant under rotations of space;
* a periodic box translating rigidly (with spanwise motion, and a uniform
  acceleration in x and y balanced by a linear pressure) is reproduced to
  rounding by BDF1 and BDF2;
* the assembled Jacobian matches central differences of the residual;
* a steady manufactured solution converges at the optimal orders
  (Section 5.1 reports optimal orders in three dimensions).
"""
import numpy as np
import pytest

from paper_2609_31477_b300 import inputs as I
from oracle import fem3d
from oracle.solver import OracleCase, viv_oracle_case
from oracle.solver3d import OracleCase3D, viv_oracle_case3d

SPAN = 0.7
LAYERS = 2


def _pair(m2=3, layers=LAYERS, span=SPAN):
    m2d = I.viv_cylinder_mesh(m2)
    m3d = I.extrude_periodic(m2d, layers, span)
    return m2d, m3d


def _random_2d_state(c2, rng):
    n = c2.n
    u = rng.normal(size=(n, 2))
    p = rng.normal(size=n) * c2.is_vertex
    delta = rng.normal(size=2) * 0.05
    x = c2.X + 0.01 * rng.normal(size=(n, 2))
    x[c2.cyl] = c2.X[c2.cyl] + delta
    lam = rng.normal(size=(n, 2)) * c2.cyl[:, None]
    hu = rng.normal(size=(n, 2))
    hx = rng.normal(size=(n, 2))
    return u, p, x, lam, delta, hu, hx


def _extend(v2, planes, zval=None):
    """z-constant extension of a nodal 2-D array onto the node planes."""
    v2 = np.asarray(v2)
    if v2.ndim == 1:
        return np.concatenate([v2] * planes)
    out = np.zeros((planes * len(v2), 3))
    for k in range(planes):
        out[k * len(v2):(k + 1) * len(v2), :2] = v2
        if zval is not None:
            out[k * len(v2):(k + 1) * len(v2), 2] = zval[k]
    return out


def test_z_invariant_residual_reduces_to_2d():
    m2d, m3d = _pair()
    rng = np.random.default_rng(5)
    rho, mu, k2, dt = 1.3, 0.02, 0.4, 0.05
    c2 = OracleCase(m2d, rho=rho, mu=mu, k=k2, dt=dt, u0=np.zeros((len(m2d["X"]), 2)))
    c3 = OracleCase3D(m3d, rho=rho, mu=mu, k=SPAN * k2, dt=dt, u0=np.zeros((len(m3d["X"]), 3)))
    u, p, x, lam, delta, hu, hx = _random_2d_state(c2, rng)
    c0 = 1.5 / dt
    R2 = c2.residual_parts(u, p, x, lam, delta, c0, hu, hx, 0.0)
    planes = 2 * LAYERS
    zs = np.arange(planes) * SPAN / planes
    R3 = c3.residual_parts(_extend(u, planes), _extend(p, planes) * c3.is_vertex, _extend(x, planes, zs),
                           _extend(lam, planes), delta, c0, _extend(hu, planes),
                           _extend(hx, planes, -c0 * zs), 0.0)
    h = SPAN / LAYERS
    n2 = c2.n
    for kpl in range(planes):
        wz = h / 3 if kpl % 2 == 0 else 2 * h / 3
        sl = slice(kpl * n2, (kpl + 1) * n2)
        for R3f, R2f in ((R3[0], R2[0]), (R3[2], R2[2]), (R3[3], R2[3])):
            scale = np.abs(R2f).max()
            assert np.abs(R3f[sl, :2] - wz * R2f).max() <= 1e-12 * scale
            assert np.abs(R3f[sl, 2]).max() <= 1e-12 * scale
        if kpl % 2 == 0:
            assert np.allclose(R3[1][sl], h * R2[1], rtol=0, atol=1e-12 * np.abs(R2[1]).max())
        else:
            assert np.abs(R3[1][sl]).max() == 0.0
    assert np.allclose(R3[4], SPAN * R2[4], rtol=1e-12, atol=1e-14)


def test_rotation_covariance_of_the_element_integrals():
    rng = np.random.default_rng(11)
    E = 4
    ref = np.array([[a, b, c] for c in (0, .5, 1) for b in (0, .5, 1) for a in (0, .5, 1)], dtype=float)
    Xe = ref[None] * np.array([1.0, 0.8, 1.2]) + 0.04 * rng.normal(size=(E, 27, 3))
    xe = Xe + 0.03 * rng.normal(size=(E, 27, 3))
    ue, hu, hx = (rng.normal(size=(E, 27, 3)) for _ in range(3))
    pe = rng.normal(size=(E, 8))
    lam = rng.uniform(0.5, 1.5, E)
    A = rng.normal(size=(3, 3))
    Q, r = np.linalg.qr(A)
    Q = Q * np.sign(np.diag(r))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    rot = lambda v: v @ Q.T
    args = (2.0, 1.1, 0.3)
    R = fem3d.volume_residual(Xe, xe, ue, pe, hu, hx, args[0], args[1], args[2], lam, 2 * lam)
    Rq = fem3d.volume_residual(rot(Xe), rot(xe), rot(ue), pe, rot(hu), rot(hx), args[0], args[1], args[2],
                               lam, 2 * lam)
    for a_, b_ in ((rot(R[0]), Rq[0]), (R[1], Rq[1]), (rot(R[2]), Rq[2])):
        assert np.abs(a_ - b_).max() <= 1e-12 * np.abs(b_).max()
    xf, uf, lf, hxf = (rng.normal(size=(E, 9, 3)) for _ in range(4))
    face = np.array([[s, t, 0.0] for t in (0, .5, 1) for s in (0, .5, 1)])
    xf = face[None] + 0.05 * xf
    G = fem3d.gamma_residual(xf, uf, lf, hxf, 1.7)
    Gq = fem3d.gamma_residual(rot(xf), rot(uf), rot(lf), rot(hxf), 1.7)
    for a_, b_ in zip(G, Gq):
        assert np.abs(rot(a_) - b_).max() <= 1e-12 * np.abs(b_).max()
    # a full-rank check that the z direction is not ignored: a rotation taking
    # z into x changes the unrotated residual
    assert np.abs(R[0] - Rq[0]).max() > 1e-3


def _box3d(n, layers, span):
    m2 = I.square_mesh(n)
    m2["tags"][0] |= I.P_FIX
    return I.extrude_periodic(m2, layers, span)


def test_translating_periodic_box_reproduced_to_rounding():
    """x = X + s(t), u = s'(t), s = (a t + b t^2, c t - b t^2, e t): the mesh
    moves rigidly (so w = u and the convective term vanishes, eps = 0); the
    acceleration s'' = (2b, -2b, 0) is balanced by p = -rho s''.x; BDF1 and
    BDF2 differentiate quadratics in t exactly."""
    span = 0.5
    m3 = _box3d(4, 2, span)
    rho, mu, dt = 2.5, 0.7, 0.1
    a, b, c, e = 0.3, 0.2, -0.4, 0.25
    s = lambda t: np.array([a * t + b * t * t, c * t - b * t * t, e * t])
    ds = lambda t: np.array([a + 2 * b * t, c - 2 * b * t, e])
    acc = np.array([2 * b, -2 * b, 0.0])
    cs = OracleCase3D(m3, rho=rho, mu=mu, k=0.0, dt=dt, u0=np.tile(ds(0.0), (len(m3["X"]), 1)), lame=1.0)

    def exact(c, t):
        c.x[:] = c.X + s(t)
        c.u[:] = ds(t)
        c.p[:] = -rho * (c.x[:, :2] @ acc[:2]) * c.is_vertex

    def dirichlet(c, t):
        keep_u, keep_p, keep_x = c.u.copy(), c.p.copy(), c.x.copy()
        exact(c, t)
        free_u, free_x = c.dof_u >= 0, c.dof_x >= 0
        c.u[free_u] = keep_u[free_u]
        c.x[free_x] = keep_x[free_x]
        free_p = c.dof_p >= 0
        c.p[free_p] = keep_p[free_p]

    exact(cs, 0.0)
    for _ in range(3):
        norms = cs.step(dirichlet=dirichlet)
        t = cs.t
        assert norms[-1] <= 1e-10
        assert np.abs(cs.u - ds(t)).max() < 1e-11
        assert np.abs(cs.x - cs.X - s(t)).max() < 1e-12
        pe = -rho * (cs.x[:, :2] @ acc[:2])
        assert np.abs((cs.p - pe)[cs.is_vertex]).max() < 1e-9


def test_jacobian_matches_central_differences():
    _, m3 = _pair(2, 2, SPAN)
    rng = np.random.default_rng(3)
    n = len(m3["X"])
    c = viv_oracle_case3d(m3, Re=150.0, Ustar=6.0, dt=0.05, u0=np.zeros((n, 3)))
    c.u = rng.normal(size=(n, 3))
    U0 = c.gather()
    c.scatter(U0 + 0.01 * rng.normal(size=U0.shape))
    c.u_n, c.x_n = c.u.copy(), c.x.copy()
    c0, hu, hx = c.bdf_coefficients()
    J = c.jacobian(c0, hu, hx, 0.05)
    U = c.gather()
    h = 1e-6
    cols = list(c.dof_u[c.cyl][:2, 2]) + list(c.dof_x[~c.cyl & (c.dof_x[:, 2] >= 0)][:3, 2]) + \
        list(c.dof_l[c.cyl][:2, 2]) + list(c.dof_d) + list(rng.integers(0, c.ndof, 6))
    for j in cols:
        e = np.zeros_like(U)
        e[j] = h
        c.scatter(U + e)
        Rp = c.residual(c0, hu, hx, 0.05)
        c.scatter(U - e)
        Rm = c.residual(c0, hu, hx, 0.05)
        c.scatter(U)
        fd = (Rp - Rm) / (2 * h)
        col = J[:, j].toarray().ravel()
        assert np.abs(col - fd).max() <= 1e-6 * max(1.0, np.abs(fd).max()), j


def test_z_invariant_step_matches_the_2d_step():
    m2d, m3d = _pair(2, 2, SPAN)
    n2, n3 = len(m2d["X"]), len(m3d["X"])
    u2 = I.viv_initial_velocity(m2d, sigma=1e-2, seed=7)
    c2 = viv_oracle_case(m2d, Re=120.0, Ustar=7.0, dt=0.1, u0=u2)
    u3 = np.zeros((n3, 3))
    u3[:, :2] = np.tile(u2, (2 * 2, 1))
    c3 = viv_oracle_case3d(m3d, Re=120.0, Ustar=7.0, dt=0.1, u0=u3)
    assert abs(c3.k - SPAN * c2.k) < 1e-14
    for _ in range(2):
        c2.step()
        c3.step()
    planes = 4
    ref = np.abs(c2.u).max()
    for kpl in range(planes):
        sl = slice(kpl * n2, (kpl + 1) * n2)
        assert np.abs(c3.u[sl, :2] - c2.u).max() <= 1e-9 * ref
        assert np.abs(c3.u[sl, 2]).max() <= 1e-9 * ref
        assert np.abs(c3.x[sl, :2] - c2.x).max() <= 1e-11
        if kpl % 2 == 0:   # vertex planes carry the pressure
            vert = c2.is_vertex
            assert np.array_equal(c3.is_vertex[sl], vert)
            assert np.abs(c3.p[sl][vert] - c2.p[vert]).max() <= 1e-8 * max(1.0, np.abs(c2.p).max())
    assert np.allclose(c3.delta, c2.delta, rtol=1e-8, atol=1e-13)
    assert np.allclose(c3.force(), SPAN * c2.force(), rtol=1e-8, atol=1e-12)


def test_steady_mms_orders_in_3d():
    """Section 5.1 reports optimal convergence in three dimensions too.  A
    steady manufactured solution on the unit box, periodic in z, with a mesh
    deformed inside (n^3 Q2-Q1 hexahedra, n = 3 and 4): the velocity L2 and
    H1 errors and the position L2 error fall at close to the optimal orders
    3, 2 and 3 of these spaces (2.95, 2.02, 3.01 from n = 4 to 6), the
    pressure at least at order 2."""
    from oracle import mms
    sol = mms.SteadyMMS3D()
    errs = []
    for n in (3, 4):
        m = I.extrude_periodic(I.square_mesh(n), n, 1.0)
        X = m["X"]
        d = np.linalg.norm(X - 0.5, axis=1)
        vert = np.zeros(len(X), bool)
        vert[m["conn"][:, fem3d.VERTEX_LOCAL].ravel()] = True
        d[~vert] = 9.0
        m["tags"][np.argmin(d)] |= I.P_FIX
        c = OracleCase3D(m, rho=sol.rho, mu=sol.mu, k=0.0, dt=1e8, u0=np.zeros((len(X), 3)), lame=1.0, src=sol)
        sol.set_dirichlet(c, 0.0)
        c.step(dirichlet=sol.set_dirichlet)
        errs.append(mms.error_norms3d(c, sol))
    r = {k: np.log(errs[0][k] / errs[1][k]) / np.log(4 / 3) for k in errs[0]}
    assert r["u_l2"] > 2.3 and r["u_h1"] > 1.7 and r["x_l2"] > 2.6 and r["p_l2"] > 1.8, r
