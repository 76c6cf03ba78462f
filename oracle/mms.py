"""Manufactured and closed-form solutions that pin the oracle (test infrastructure).

Section 5.1 verifies the solver with manufactured solutions: arbitrary smooth
u, p, x fields with the matching source terms added to each equation.  Two
families are built here with sympy:

  * TranslatingBox - a rigid translation of the whole mesh x = X + a t, a
    velocity that is linear in space, u = (alpha + beta t + gamma t^3)(c + D x),
    and a linear pressure, on a square with a square hole (the rigid body
    Gamma).  Q2 velocity, Q1 pressure and Q2 position represent these fields
    exactly on affine cells, and with gamma = 0 the nodal trajectories are
    quadratic in time, which BDF2 integrates exactly.  The discrete solution
    must then equal the exact one to rounding; with gamma != 0 the error is the
    BDF2 truncation error and must fall as dt^2.
  * SteadyMMS - the 2-D velocity and pressure of Section 5.1 (without the time
    factors) on a unit square whose mesh is statically deformed by
    x = X + A sin(pi X) sin(pi Y) (1, 1), run with a very large time step so the
    converged step is the steady problem; errors must fall at the optimal rates.
  * UnsteadyMMS - the same fields with Section 5.1's time factors (t^3 for the
    velocity, t^2 for the pressure) on a mesh moved by
    x = X + A sin(pi t) sin(pi X) sin(pi Y) (1, 1): BDF2 must be second order in
    time and the spatial rates optimal.

Each provides: volume(Xq, t) -> (f_u, g_p, f_x), gamma(Xq, t) -> g_lambda,
border(t) -> F, exact nodal values and a Dirichlet setter.
"""
from __future__ import annotations

import numpy as np
import sympy as sy

X_, Y_, x_, y_, t_ = sy.symbols("X Y x y t", real=True)


def _vec_fun(exprs, args):
    f = sy.lambdify(args, exprs, "numpy")

    def call(*a):
        shape = np.broadcast(*a).shape
        dt_ = np.result_type(*a, np.float64)   # complex arguments (complex step) stay complex
        out = f(*a)
        return np.stack([np.broadcast_to(np.asarray(o, dtype=dt_), shape) for o in out], axis=-1)
    return call


class _Manufactured:
    """Common machinery: u(x,y,t), p(x,y,t) in physical coordinates, the
    motion chi(X,Y,t), fluid and pseudo-solid coefficients."""

    def __init__(self, u, p, chi, rho, mu, lam_s, mu_s, k=0.0, hole=None):
        self.rho, self.mu, self.lam_s, self.mu_s, self.k = rho, mu, lam_s, mu_s, k
        ux, uy = u
        # fluid source: rho (d_t u|_x + (u.grad) u) - div sigma
        grad = sy.Matrix([[sy.diff(ux, x_), sy.diff(ux, y_)], [sy.diff(uy, x_), sy.diff(uy, y_)]])
        sigma = -p * sy.eye(2) + mu * (grad + grad.T)
        uvec = sy.Matrix([ux, uy])
        conv = grad * uvec
        divs = sy.Matrix([sy.diff(sigma[0, 0], x_) + sy.diff(sigma[0, 1], y_),
                          sy.diff(sigma[1, 0], x_) + sy.diff(sigma[1, 1], y_)])
        fu = rho * (sy.diff(uvec, t_) + conv) - divs
        gp = grad[0, 0] + grad[1, 1]
        # pseudo-solid source: -div_X sigma_s(chi)
        cx, cy = chi
        F = sy.Matrix([[sy.diff(cx, X_), sy.diff(cx, Y_)], [sy.diff(cy, X_), sy.diff(cy, Y_)]])
        eps = (F + F.T) / 2 - sy.eye(2)
        sig_s = lam_s * (eps[0, 0] + eps[1, 1]) * sy.eye(2) + 2 * mu_s * eps
        fx = -sy.Matrix([sy.diff(sig_s[0, 0], X_) + sy.diff(sig_s[0, 1], Y_),
                         sy.diff(sig_s[1, 0], X_) + sy.diff(sig_s[1, 1], Y_)])
        sub = {x_: cx, y_: cy}
        self._fu = _vec_fun([fu[0].subs(sub), fu[1].subs(sub)], (X_, Y_, t_))
        self._gp = sy.lambdify((X_, Y_, t_), gp.subs(sub), "numpy")
        # the same fluid sources as fields of the physical coordinates
        self._fu_x = _vec_fun([fu[0], fu[1]], (x_, y_, t_))
        self._gp_x = sy.lambdify((x_, y_, t_), gp, "numpy")
        self._fx = _vec_fun([fx[0], fx[1]], (X_, Y_, t_))
        wx, wy = sy.diff(cx, t_), sy.diff(cy, t_)
        self._gl = _vec_fun([ux.subs(sub) - wx, uy.subs(sub) - wy], (X_, Y_, t_))
        self._u_phys = _vec_fun([ux, uy], (x_, y_, t_))
        self._grad_u_phys = _vec_fun([grad[0, 0], grad[0, 1], grad[1, 0], grad[1, 1]], (x_, y_, t_))
        self._p_phys = sy.lambdify((x_, y_, t_), p, "numpy")
        self._chi = _vec_fun([cx, cy], (X_, Y_, t_))
        self._grad_chi = _vec_fun([F[0, 0], F[0, 1], F[1, 0], F[1, 1]], (X_, Y_, t_))
        self.sigma = sigma
        self.hole = hole
        self._border = None
        if hole is not None:
            a, b = hole
            # int_Gamma sigma.n ds with n the outward normal of the fluid (into the hole),
            # on the hole moved by chi (a rigid translation on Gamma)
            dx = cx.subs({X_: a, Y_: a}) - a
            dy = cy.subs({X_: a, Y_: a}) - a
            s = sy.symbols("s", real=True)
            tot = sy.zeros(2, 1)
            # side X = a: fluid normal +x;  X = b: -x;  Y = a: +y;  Y = b: -y
            for (px, py, n) in (((a + dx), (s + dy), (1, 0)), ((b + dx), (s + dy), (-1, 0)),
                                ((s + dx), (a + dy), (0, 1)), ((s + dx), (b + dy), (0, -1))):
                sig = sigma.subs({x_: px, y_: py})
                tvec = sig * sy.Matrix(n)
                tot += sy.Matrix([sy.integrate(tvec[0], (s, a, b)), sy.integrate(tvec[1], (s, a, b))])
            F_border = self.k * sy.Matrix([dx, dy]) + tot
            self._border = _vec_fun([sy.simplify(F_border[0]), sy.simplify(F_border[1])], (t_,))
            self._delta = _vec_fun([dx, dy], (t_,))
            self._force = _vec_fun([-tot[0], -tot[1]], (t_,))

    # ---- source interface used by oracle.fem --------------------------------
    def volume(self, Xq, t):
        X, Y = Xq[..., 0], Xq[..., 1]
        gp = np.broadcast_to(np.asarray(self._gp(X, Y, t), dtype=np.float64), X.shape)
        return self._fu(X, Y, t), gp, self._fx(X, Y, t)

    def volume_at(self, xq, Xq, t):
        """Fluid sources at the physical points xq (the discrete current
        position of the quadrature points), pseudo-solid source at the
        reference points Xq.  For a P1 position field x_h differs from chi by
        O(h^2), and evaluating the Eulerian sources at chi(Xq) would leave an
        O(h^2) defect in the continuity equations' compatibility, which a
        single pinned pressure vertex amplifies."""
        x, y = xq[..., 0], xq[..., 1]
        gp = np.broadcast_to(np.asarray(self._gp_x(x, y, t)), x.shape)
        return self._fu_x(x, y, t), gp, self._fx(Xq[..., 0], Xq[..., 1], t)

    def gamma(self, Xq, t):
        return self._gl(Xq[..., 0], Xq[..., 1], t)

    def border(self, t):
        if self._border is None:
            return np.zeros(2)
        return self._border(np.float64(t))

    # ---- exact values -------------------------------------------------------
    def position(self, X, t):
        return self._chi(X[..., 0], X[..., 1], t)

    def velocity(self, X, t):
        x = self.position(X, t)
        return self._u_phys(x[..., 0], x[..., 1], t)

    def pressure(self, X, t):
        x = self.position(X, t)
        return np.broadcast_to(np.asarray(self._p_phys(x[..., 0], x[..., 1], t), dtype=np.float64),
                               X.shape[:-1])

    def delta(self, t):
        return self._delta(np.float64(t)) if self.hole is not None else np.zeros(2)

    def force(self, t):
        """Exact F_fluid = -int_Gamma sigma.n (n outward from the fluid)."""
        return self._force(np.float64(t))

    def set_dirichlet(self, case, t):
        """Hold every prescribed component at its exact value at time t."""
        from .solver import U_FIX_X, U_FIX_Y, X_FIX_X, X_FIX_Y, P_FIX
        tg = case.tags
        ue = self.velocity(case.X, t)
        xe = self.position(case.X, t)
        pe = self.pressure(case.X, t)
        for i, bit in enumerate((U_FIX_X, U_FIX_Y)):
            m = (tg & bit) != 0
            case.u[m, i] = ue[m, i]
        for i, bit in enumerate((X_FIX_X, X_FIX_Y)):
            m = ((tg & bit) != 0) & ~case.cyl
            case.x[m, i] = xe[m, i]
        m = (tg & P_FIX) != 0
        case.p[m] = pe[m]

    def set_exact_state(self, case, t):
        """Exact nodal u, x (and p, delta) at time t."""
        case.u[:] = self.velocity(case.X, t)
        case.x[:] = self.position(case.X, t)
        case.p[:] = self.pressure(case.X, t)
        if case.has_body:
            case.delta = self.delta(t)


def translating_box(gamma=0.0, rho=9.876, mu=1.234, k=2.5, hole=(0.4, 0.6)):
    """Closed-form patch solution on a square with a square hole, moving
    rigidly with x = X + a t; see the module docstring."""
    a = (sy.Rational(3, 10), -sy.Rational(1, 5))
    chi = (X_ + a[0] * t_, Y_ + a[1] * t_)
    s = 1 + 2 * t_ + gamma * t_ ** 3
    ux = s * (1 + sy.Rational(1, 2) * x_ + y_)
    uy = s * (sy.Rational(1, 2) - sy.Rational(7, 10) * x_ + sy.Rational(1, 5) * y_)
    p = (1 + t_) * (sy.Rational(3, 10) + sy.Rational(4, 5) * x_ - sy.Rational(3, 5) * y_)
    return _Manufactured((ux, uy), p, chi, rho, mu, 1.0, 1.0, k=k, hole=hole)


def steady_mms(rho=9.876, mu=1.234, amp=0.05):
    """Section 5.1's 2-D velocity and pressure (time factors dropped) on a
    statically deformed unit-square mesh, lambda_s = mu_s = 1."""
    pi = sy.pi
    chi = (X_ + amp * sy.sin(pi * X_) * sy.sin(pi * Y_), Y_ + amp * sy.sin(pi * X_) * sy.sin(pi * Y_))
    ux = sy.sin(pi * x_) * sy.cos(pi * y_)
    uy = sy.sin(pi * x_) * sy.sin(pi * y_)
    p = sy.cos(pi * x_) * sy.cos(pi * y_)
    return _Manufactured((ux, uy), p, chi, rho, mu, 1.0, 1.0)


def unsteady_mms(rho=9.876, mu=1.234, amp=0.05):
    """Section 5.1's time-dependent 2-D manufactured solution:
    u = t^3 (sin pi x cos pi y, sin pi x sin pi y), p = t^2 cos pi x cos pi y
    on the unit square, with the mesh moved by
    x = X + amp sin(pi t) sin(pi X) sin(pi Y) (1, 1) (zero on the boundary),
    lambda_s = mu_s = 1; all-Dirichlet velocity and position."""
    pi = sy.pi
    bump = amp * sy.sin(pi * t_) * sy.sin(pi * X_) * sy.sin(pi * Y_)
    chi = (X_ + bump, Y_ + bump)
    ux = t_ ** 3 * sy.sin(pi * x_) * sy.cos(pi * y_)
    uy = t_ ** 3 * sy.sin(pi * x_) * sy.sin(pi * y_)
    p = t_ ** 2 * sy.cos(pi * x_) * sy.cos(pi * y_)
    return _Manufactured((ux, uy), p, chi, rho, mu, 1.0, 1.0)


QUASI_CENTER = (0.5, 0.5)
QUASI_R0, QUASI_R1 = 0.15, 0.45
QUASI_D_DIR = (0.8, 0.6)


def _kernel_numpy(R0, R1):
    """psi(r) = 1 - phi(s), s = (r - R0)/(R1 - R0) clamped to [0, 1], and its
    first three r-derivatives (zero where s is clamped: phi'(0) = phi'(1) =
    phi''(0) = phi''(1) = 0, so psi is C^2)."""
    L = R1 - R0

    def s_of(r):
        return np.clip((np.asarray(r, dtype=np.float64) - R0) / L, 0.0, 1.0)

    def inside(r):
        r = np.asarray(r, dtype=np.float64)
        return (r > R0) & (r < R1)

    psi0 = lambda r: 1.0 - (6 * s_of(r) ** 5 - 15 * s_of(r) ** 4 + 10 * s_of(r) ** 3)
    psi1 = lambda r: np.where(inside(r), -(30 * s_of(r) ** 4 - 60 * s_of(r) ** 3 + 30 * s_of(r) ** 2) / L, 0.0)
    psi2 = lambda r: np.where(inside(r), -(120 * s_of(r) ** 3 - 180 * s_of(r) ** 2 + 60 * s_of(r)) / L ** 2, 0.0)
    psi3 = lambda r: np.where(inside(r), -(360 * s_of(r) ** 2 - 360 * s_of(r) + 60) / L ** 3, 0.0)
    return {"Psi": psi0, "Psi1": psi1, "Psi2": psi2, "Psi3": psi3}


class Psi3(sy.Function):
    pass


class Psi2(sy.Function):
    def fdiff(self, argindex=1):
        return Psi3(self.args[0])


class Psi1(sy.Function):
    def fdiff(self, argindex=1):
        return Psi2(self.args[0])


class Psi(sy.Function):
    """The bell-shaped kernel of Section 5.1; evaluated numerically (see
    _kernel_numpy) so that the symbolic calculus stays small."""

    def fdiff(self, argindex=1):
        return Psi1(self.args[0])


class QuasiMMS:
    """Section 5.2's coupled quasi-manufactured solution on the unit square
    around a rigid cylinder of radius R0 centred at X_c:
      x = X + f(t) d psi(|X - X_c|),      u = f'(t) d psi(|x - x_c(t)|),
      p = -k f(t) / (pi R0) (d . e) psi(|x - x_c(t)|),  e = (x - x_c)/|x - x_c|,
    x_c(t) = X_c + f(t) d, f(t) = sin(2 pi t), psi(r) = 1 - phi((r - R0)/(R1 - R0))
    with phi(s) = 6 s^5 - 15 s^4 + 10 s^3 (psi = 1 up to R0, 0 beyond R1).
    The cylinder moves rigidly (delta = f d), u equals the mesh velocity on it
    and the velocity gradient vanishes there, so the multiplier rows and the
    coupling row k delta + int_Gamma lambda = 0 hold without source terms
    (int_Gamma p e ds = -k f d); only the momentum, continuity and
    pseudo-solid equations get sources, derived here with sympy:
      f_u = rho (d_t u|_x + (u . grad) u) - div sigma(u, p),  g_p = div u,
      f_x = -div_X sigma_s(x)  (lambda_s = mu_s = 1).
    The total displacement d = amp (0.8, 0.6) with amp <= 0.05 keeps psi = 0
    on the outer boundary, so the Dirichlet data there are u = 0, x = X (and a
    pinned pressure 0)."""

    def __init__(self, k=10.0, amp=0.05, rho=1.0, mu=0.1):
        pi = sy.pi
        cx, cy = QUASI_CENTER
        R0 = QUASI_R0
        self.rho, self.mu, self.k, self.lam_s, self.mu_s = rho, mu, k, 1.0, 1.0
        self.hole = None
        dx, dy = amp * QUASI_D_DIR[0], amp * QUASI_D_DIR[1]
        f = sy.sin(2 * pi * t_)
        fp = sy.diff(f, t_)
        xcx, xcy = cx + f * dx, cy + f * dy
        r = sy.sqrt((x_ - xcx) ** 2 + (y_ - xcy) ** 2)
        ux, uy = fp * dx * Psi(r), fp * dy * Psi(r)
        p = -k * f / (pi * R0) * (dx * (x_ - xcx) + dy * (y_ - xcy)) / r * Psi(r)
        grad = sy.Matrix([[sy.diff(ux, x_), sy.diff(ux, y_)], [sy.diff(uy, x_), sy.diff(uy, y_)]])
        sigma = -p * sy.eye(2) + mu * (grad + grad.T)
        uvec = sy.Matrix([ux, uy])
        divs = sy.Matrix([sy.diff(sigma[0, 0], x_) + sy.diff(sigma[0, 1], y_),
                          sy.diff(sigma[1, 0], x_) + sy.diff(sigma[1, 1], y_)])
        fu = rho * (sy.diff(uvec, t_) + grad * uvec) - divs
        gp = grad[0, 0] + grad[1, 1]
        RX = sy.sqrt((X_ - cx) ** 2 + (Y_ - cy) ** 2)
        chx, chy = X_ + f * dx * Psi(RX), Y_ + f * dy * Psi(RX)
        F = sy.Matrix([[sy.diff(chx, X_), sy.diff(chx, Y_)], [sy.diff(chy, X_), sy.diff(chy, Y_)]])
        eps = (F + F.T) / 2 - sy.eye(2)
        sig_s = (eps[0, 0] + eps[1, 1]) * sy.eye(2) + 2 * eps
        fx = -sy.Matrix([sy.diff(sig_s[0, 0], X_) + sy.diff(sig_s[0, 1], Y_),
                         sy.diff(sig_s[1, 0], X_) + sy.diff(sig_s[1, 1], Y_)])
        mods = [_kernel_numpy(QUASI_R0, QUASI_R1), "numpy"]

        def vec(exprs, args):
            fn = sy.lambdify(args, exprs, modules=mods)

            def call(*a):
                shape = np.broadcast(*a).shape
                return np.stack([np.broadcast_to(np.asarray(o, dtype=np.float64), shape) for o in fn(*a)], axis=-1)
            return call

        def scal(expr, args):
            fn = sy.lambdify(args, expr, modules=mods)
            return lambda *a: np.broadcast_to(np.asarray(fn(*a), dtype=np.float64), np.broadcast(*a).shape)

        self._fu_x = vec([fu[0], fu[1]], (x_, y_, t_))
        self._gp_x = scal(gp, (x_, y_, t_))
        self._fx = vec([fx[0], fx[1]], (X_, Y_, t_))
        self._u_phys = vec([ux, uy], (x_, y_, t_))
        self._grad_u_phys = vec([grad[0, 0], grad[0, 1], grad[1, 0], grad[1, 1]], (x_, y_, t_))
        self._p_phys = scal(p, (x_, y_, t_))
        self._chi = vec([chx, chy], (X_, Y_, t_))
        self._grad_chi = vec([F[0, 0], F[0, 1], F[1, 0], F[1, 1]], (X_, Y_, t_))
        self.d = np.array([dx, dy], dtype=np.float64)
        self.amp = amp

    # ---- source interface used by oracle.fem --------------------------------
    def volume(self, Xq, t):
        xq = self._chi(Xq[..., 0], Xq[..., 1], t)
        return (self._fu_x(xq[..., 0], xq[..., 1], t), self._gp_x(xq[..., 0], xq[..., 1], t),
                self._fx(Xq[..., 0], Xq[..., 1], t))

    def volume_at(self, xq, Xq, t):
        """Fluid sources at the physical points xq (the discrete current
        position of the quadrature points), pseudo-solid source at the
        reference points Xq.  For a P1 position field x_h differs from chi by
        O(h^2), and evaluating the Eulerian sources at chi(Xq) would leave an
        O(h^2) defect in the continuity equations' compatibility, which a
        single pinned pressure vertex amplifies."""
        x, y = xq[..., 0], xq[..., 1]
        gp = np.broadcast_to(np.asarray(self._gp_x(x, y, t)), x.shape)
        return self._fu_x(x, y, t), gp, self._fx(Xq[..., 0], Xq[..., 1], t)

    def gamma(self, Xq, t):
        return np.zeros(Xq.shape[:-1] + (2,))

    def border(self, t):
        return np.zeros(2)

    # ---- exact values -------------------------------------------------------
    def position(self, X, t):
        return self._chi(X[..., 0], X[..., 1], t)

    def velocity(self, X, t):
        x = self.position(X, t)
        return self._u_phys(x[..., 0], x[..., 1], t)

    def pressure(self, X, t):
        x = self.position(X, t)
        return self._p_phys(x[..., 0], x[..., 1], t)

    def delta(self, t):
        return np.sin(2 * np.pi * t) * self.d

    def force(self, t):
        """F_fluid = -int_Gamma lambda = k delta (the spring balance)."""
        return self.k * self.delta(t)

    set_dirichlet = _Manufactured.set_dirichlet
    set_exact_state = _Manufactured.set_exact_state


def error_norms(case, sol, t):
    """Errors of the discrete state against the exact fields:
    u in L2 and H1-seminorm and p in L2 over Omega_t, x in L2 and H1-seminorm
    over Omega_0 (Section 5.1's norms, measured with 3x3 Gauss points)."""
    from . import fem
    c = case.conn
    Xe, xe, ue = case.X[c], case.x[c], case.u[c]
    pe = case.p[c[:, fem.VERTEX_LOCAL]]
    eu2 = eu1 = ep2 = ex2 = ex1 = 0.0
    for q in range(9):
        N, M, w = fem.N_Q[q], fem.M_Q[q], fem.W_Q[q]
        g, det = fem.physical_gradients(xe, q)
        g0, det0 = fem.physical_gradients(Xe, q)
        Xq = np.einsum('a,eai->ei', N, Xe)
        xq = np.einsum('a,eai->ei', N, xe)
        uh = np.einsum('a,eai->ei', N, ue)
        Lh = np.einsum('eai,eaj->eij', ue, g)
        ph = np.einsum('c,ec->e', M, pe)
        ux = sol._u_phys(xq[:, 0], xq[:, 1], t)
        Lx = sol._grad_u_phys(xq[:, 0], xq[:, 1], t).reshape(-1, 2, 2)
        px = np.broadcast_to(sol._p_phys(xq[:, 0], xq[:, 1], t), ph.shape)
        eu2 += np.sum(w * det * np.sum((uh - ux) ** 2, axis=1))
        eu1 += np.sum(w * det * np.sum((Lh - Lx) ** 2, axis=(1, 2)))
        ep2 += np.sum(w * det * (ph - px) ** 2)
        Fh = np.einsum('eai,eaj->eij', xe, g0)
        Fx = sol._grad_chi(Xq[:, 0], Xq[:, 1], t).reshape(-1, 2, 2)
        xx = sol._chi(Xq[:, 0], Xq[:, 1], t)
        ex2 += np.sum(w * det0 * np.sum((xq - xx) ** 2, axis=1))
        ex1 += np.sum(w * det0 * np.sum((Fh - Fx) ** 2, axis=(1, 2)))
    return dict(u_l2=np.sqrt(eu2), u_h1=np.sqrt(eu1), p_l2=np.sqrt(ep2),
                x_l2=np.sqrt(ex2), x_h1=np.sqrt(ex1))


def error_norms_tri(case, sol, t):
    """The norms of `error_norms` for a P2-P1 triangle case with a P1
    position (oracle/solver_tri.py), measured with the 7-point rule: u and p
    on the current (affine) triangles, x on the reference ones."""
    from . import fem_tri
    c = case.conn
    cv = c[:, :3]
    Xv, xv, ue, pv = case.X[cv], case.x[cv], case.u[c], case.p[cv]
    _, Jinv, det = fem_tri.affine(xv)
    _, Jinv0, det0 = fem_tri.affine(Xv)
    h0 = np.matmul(fem_tri.DM[None], Jinv0)             # reference P1 gradients (E, 3, 2)
    Fh = np.einsum('evi,evj->eij', xv, h0)              # grad_X x_h, constant per triangle
    eu2 = eu1 = ep2 = ex2 = ex1 = 0.0
    for q in range(len(fem_tri.QWTS)):
        N, M, w = fem_tri.N_Q[q], fem_tri.M_Q[q], fem_tri.QWTS[q]
        g = np.matmul(fem_tri.DN_Q[q][None], Jinv)
        Xq = np.einsum('v,evi->ei', M, Xv)
        xq = np.einsum('v,evi->ei', M, xv)
        uh = np.einsum('a,eai->ei', N, ue)
        Lh = np.einsum('eai,eaj->eij', ue, g)
        ph = np.einsum('v,ev->e', M, pv)
        ux = sol._u_phys(xq[:, 0], xq[:, 1], t)
        Lx = sol._grad_u_phys(xq[:, 0], xq[:, 1], t).reshape(-1, 2, 2)
        px = np.broadcast_to(sol._p_phys(xq[:, 0], xq[:, 1], t), ph.shape)
        eu2 += np.sum(w * det * np.sum((uh - ux) ** 2, axis=1))
        eu1 += np.sum(w * det * np.sum((Lh - Lx) ** 2, axis=(1, 2)))
        ep2 += np.sum(w * det * (ph - px) ** 2)
        Fx = sol._grad_chi(Xq[:, 0], Xq[:, 1], t).reshape(-1, 2, 2)
        xx = sol._chi(Xq[:, 0], Xq[:, 1], t)
        ex2 += np.sum(w * det0 * np.sum((xq - xx) ** 2, axis=1))
        ex1 += np.sum(w * det0 * np.sum((Fh - Fx) ** 2, axis=(1, 2)))
    return dict(u_l2=np.sqrt(eu2), u_h1=np.sqrt(eu1), p_l2=np.sqrt(ep2),
                x_l2=np.sqrt(ex2), x_h1=np.sqrt(ex1))


# --- 3-D: a steady manufactured solution on a box periodic in z -------------------
Z_, z_ = sy.symbols("Z z", real=True)


class SteadyMMS3D:
    """Section 5.1's three-dimensional check, as a steady problem on the box
    [0,1]^2 x [0,1) periodic in z (the spanwise direction of the 3-D
    workload): smooth velocity and pressure with 2 pi z dependence, a mesh
    deformed by x = X + A sin(pi X) sin(pi Y) (1, 1, cos 2 pi Z) (identity on
    the x and y faces, periodic in z), lambda_s = mu_s = 1, and the matching
    sources: f_u = rho (u.grad) u - div sigma, g_p = div u,
    f_x = -div_X sigma_s(chi).  The fluid sources are fields of the physical
    coordinates, evaluated at the discrete current quadrature points."""

    def __init__(self, rho=9.876, mu=1.234, amp=0.05):
        self.rho, self.mu = rho, mu
        pi = sy.pi
        c2 = sy.cos(2 * pi * z_)
        u = sy.Matrix([sy.sin(pi * x_) * sy.cos(pi * y_) * c2,
                       sy.cos(pi * x_) * sy.sin(pi * y_) * c2,
                       sy.sin(pi * x_) * sy.sin(pi * y_) * sy.sin(2 * pi * z_)])
        p = sy.cos(pi * x_) * sy.cos(pi * y_) * sy.cos(2 * pi * z_)
        xs = (x_, y_, z_)
        grad = sy.Matrix(3, 3, lambda i, j: sy.diff(u[i], xs[j]))
        sigma = -p * sy.eye(3) + mu * (grad + grad.T)
        divs = sy.Matrix([sum(sy.diff(sigma[i, j], xs[j]) for j in range(3)) for i in range(3)])
        fu = rho * grad * u - divs
        gp = grad[0, 0] + grad[1, 1] + grad[2, 2]
        bump = amp * sy.sin(pi * X_) * sy.sin(pi * Y_)
        chi = sy.Matrix([X_ + bump, Y_ + bump, Z_ + bump * sy.cos(2 * pi * Z_)])
        Xs = (X_, Y_, Z_)
        F = sy.Matrix(3, 3, lambda i, j: sy.diff(chi[i], Xs[j]))
        eps = (F + F.T) / 2 - sy.eye(3)
        sig_s = (eps[0, 0] + eps[1, 1] + eps[2, 2]) * sy.eye(3) + 2 * eps
        fx = -sy.Matrix([sum(sy.diff(sig_s[i, j], Xs[j]) for j in range(3)) for i in range(3)])
        self._fu = _vec_fun(list(fu), xs)
        self._gp = sy.lambdify(xs, gp, "numpy")
        self._fx = _vec_fun(list(fx), Xs)
        self._u = _vec_fun(list(u), xs)
        self._grad_u = _vec_fun(list(grad), xs)
        self._p = sy.lambdify(xs, p, "numpy")
        self._chi = _vec_fun(list(chi), Xs)

    def volume_at(self, xq, Xq, t):
        x, y, z = xq[..., 0], xq[..., 1], xq[..., 2]
        gp = np.broadcast_to(np.asarray(self._gp(x, y, z)), x.shape)
        return self._fu(x, y, z), gp, self._fx(Xq[..., 0], Xq[..., 1], Xq[..., 2])

    def set_dirichlet(self, case, t):
        """Prescribed components at their exact values (positions through chi,
        velocity and pressure at the prescribed positions)."""
        from .solver3d import U_FIX_X, U_FIX_Y, U_FIX_Z, X_FIX_X, X_FIX_Y, X_FIX_Z, P_FIX
        tg = case.tags
        xe = self._chi(case.X[:, 0], case.X[:, 1], case.X[:, 2])
        for i, bit in enumerate((X_FIX_X, X_FIX_Y, X_FIX_Z)):
            m = (tg & bit) != 0
            case.x[m, i] = xe[m, i]
        ue = self._u(xe[:, 0], xe[:, 1], xe[:, 2])
        for i, bit in enumerate((U_FIX_X, U_FIX_Y, U_FIX_Z)):
            m = (tg & bit) != 0
            case.u[m, i] = ue[m, i]
        m = (tg & P_FIX) != 0
        case.p[m] = np.broadcast_to(self._p(xe[:, 0], xe[:, 1], xe[:, 2]), m.shape)[m]


def error_norms3d(case, sol):
    """u in L2 and H1-seminorm and p in L2 over the current hexahedra,
    x in L2 over the reference ones (3x3x3 Gauss points)."""
    from . import fem3d
    c = case.conn
    Xe = case.X[c] + case.shift
    xe = case.x[c] + case.shift
    ue = case.u[c]
    pe = case.p[c[:, fem3d.VERTEX_LOCAL]]
    eu2 = eu1 = ep2 = ex2 = 0.0
    for q in range(27):
        N, M, w = fem3d.N_Q[q], fem3d.M_Q[q], fem3d.W_Q[q]
        g, det = fem3d.physical_gradients(xe, q)
        _, det0 = fem3d.physical_gradients(Xe, q)
        xq = np.einsum('a,eai->ei', N, xe)
        Xq = np.einsum('a,eai->ei', N, Xe)
        uh = np.einsum('a,eai->ei', N, ue)
        Lh = np.einsum('eai,eaj->eij', ue, g)
        ph = np.einsum('c,ec->e', M, pe)
        ux = sol._u(xq[:, 0], xq[:, 1], xq[:, 2])
        Lx = sol._grad_u(xq[:, 0], xq[:, 1], xq[:, 2]).reshape(-1, 3, 3)
        px = np.broadcast_to(sol._p(xq[:, 0], xq[:, 1], xq[:, 2]), ph.shape)
        xx = sol._chi(Xq[:, 0], Xq[:, 1], Xq[:, 2])
        eu2 += np.sum(w * det * np.sum((uh - ux) ** 2, axis=1))
        eu1 += np.sum(w * det * np.sum((Lh - Lx) ** 2, axis=(1, 2)))
        ep2 += np.sum(w * det * (ph - px) ** 2)
        ex2 += np.sum(w * det0 * np.sum((xq - xx) ** 2, axis=1))
    return dict(u_l2=np.sqrt(eu2), u_h1=np.sqrt(eu1), p_l2=np.sqrt(ep2), x_l2=np.sqrt(ex2))
