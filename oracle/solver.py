"""Oracle case: unknowns, global residual and Jacobian, BDF time stepping and
Newton-Raphson (test infrastructure; FP64, slow, plain).

Follows:
  * Eq. NR_iteration: J(U_m) dU_m = -NL(U_m), U_{m+1} = U_m + dU_m, stopped
    when ||NL||_2 <= tol (absolute, over all unknowns), followed by one more
    iteration so that the state lands at round-off rather than anywhere below
    the tolerance - the stopping rule is the reading taken here; the paper
    does not state one.
  * BDF2 in time with a BDF1 first step and constant dt (Section 3, Section 6);
    the time derivatives of u and x are taken along node trajectories.
  * Eq. lambda_coupling / Eq. coupling_constraint: every Gamma node sits at
    x_a = X_a + delta with delta in R^2; the border rows are
    k delta + int_Gamma lambda = 0 (Eq. solid_balance with
    F_fluid = -int_Gamma lambda).  The pseudo-solid has no rows at Gamma nodes.
  * Dirichlet conditions Eq. flowBC / Eq. psBC, held by node tags.
  * Lame coefficients lambda_s = mu_s = min|K_0| / |K_0| per element (reference
    areas); the paper's distance-based formula in Section 6 is garbled, a
    per-element inverse area normalised by the smallest element is the reading
    taken here (any constant factor leaves the solution unchanged).
The linear solve is a library sparse LU (SuperLU through scipy) - a library
primitive used as one step.  The Jacobian is assembled from element
Jacobians obtained by complex-step differentiation of the element residual.
"""
from __future__ import annotations

import math
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem

U_FIX_X, U_FIX_Y, X_FIX_X, X_FIX_Y, CYL, P_FIX = 1, 2, 4, 8, 16, 64
EDGE_NODES = ((0, 3, 6), (2, 5, 8), (0, 1, 2), (6, 7, 8))
H_CS = 1e-30


def sparse_lu(J):
    """Library sparse LU (SuperLU) of the Jacobian, with a minimum-degree
    ordering of A^T + A: the same exact factorisation up to rounding as any
    other ordering, with a fraction of COLAMD's fill on these matrices."""
    return spla.splu(J.tocsc(), permc_spec="MMD_AT_PLUS_A")


def stiffness_from_reduced_velocity(rho, U_inf, Ustar, L=1.0):
    """U_r = pi U sqrt(pi rho L / k) (Section 1) solved for k."""
    return math.pi ** 3 * rho * L * U_inf ** 2 / Ustar ** 2


class OracleCase:
    """A mesh, its parameters and the time-stepping state.

    State arrays are nodal: u (n,2), p (n,) [vertices only], x (n,2),
    lam (n,2) [Gamma nodes only], delta (2,).  Prescribed components keep the
    value they hold in the initial state.
    """

    def __init__(self, mesh, rho, mu, k, dt, u0, lame="inverse_area", src=None):
        self.mesh = mesh
        self.X = np.asarray(mesh["X"], dtype=np.float64)
        self.conn = np.asarray(mesh["conn"], dtype=np.int64)
        self.tags = np.asarray(mesh["tags"], dtype=np.int64)
        gf = np.asarray(mesh["gamma_faces"], dtype=np.int64).reshape(-1, 2)
        self.faces = np.array([[self.conn[e, a] for a in EDGE_NODES[ed]] for e, ed in gf],
                              dtype=np.int64).reshape(-1, 3)
        self.rho, self.mu, self.k, self.dt = rho, mu, k, dt
        self.dt_prev = dt     # size of the previous step (variable-step BDF2)
        self.src = src
        n = len(self.X)
        self.n = n
        Xe = self.X[self.conn]
        area = fem.element_areas(Xe)
        if lame == "inverse_area":
            # lambda_s = mu_s proportional to 1/|K_0|; the constant is the smallest
            # reference area, so the coefficients lie in (0, 1] (the solution does
            # not depend on it: the pseudo-solid equations are homogeneous)
            self.lam_s = area.min() / area
        else:
            self.lam_s = np.full(len(self.conn), float(lame))
        self.mu_s = self.lam_s.copy()
        self._number_dofs()
        # state
        self.u = np.array(u0, dtype=np.float64).reshape(n, 2).copy()
        self.p = np.zeros(n)
        self.x = self.X.copy()
        self.lam = np.zeros((n, 2))
        self.delta = np.zeros(2)
        self.t = 0.0
        self.nstep = 0
        self.hist = None          # (u_nm1, x_nm1) once a step has been taken

    # ---- unknown numbering: field-major, fixed components excluded ---------
    def _number_dofs(self):
        n, t = self.n, self.tags
        is_vertex = np.zeros(n, bool)
        is_vertex[self.conn[:, fem.VERTEX_LOCAL].ravel()] = True
        self.is_vertex = is_vertex
        cyl = (t & CYL) != 0
        self.cyl = cyl
        idx = 0
        self.dof_u = -np.ones((n, 2), np.int64)
        free_u = np.stack([(t & U_FIX_X) == 0, (t & U_FIX_Y) == 0], axis=1)
        for a in range(n):
            for i in range(2):
                if free_u[a, i]:
                    self.dof_u[a, i] = idx
                    idx += 1
        self.dof_p = -np.ones(n, np.int64)
        for a in range(n):
            if is_vertex[a] and (t[a] & P_FIX) == 0:
                self.dof_p[a] = idx
                idx += 1
        self.dof_x = -np.ones((n, 2), np.int64)
        free_x = np.stack([(t & X_FIX_X) == 0, (t & X_FIX_Y) == 0], axis=1)
        for a in range(n):
            if cyl[a]:
                continue
            for i in range(2):
                if free_x[a, i]:
                    self.dof_x[a, i] = idx
                    idx += 1
        self.dof_l = -np.ones((n, 2), np.int64)
        for a in range(n):
            if cyl[a]:
                for i in range(2):
                    self.dof_l[a, i] = idx
                    idx += 1
        self.has_body = bool(cyl.any())
        self.dof_d = np.array([idx, idx + 1]) if self.has_body else -np.ones(2, np.int64)
        if self.has_body:
            idx += 2
        self.ndof = idx
        # column map of position components: Gamma nodes alias to delta
        self.col_x = self.dof_x.copy()
        for a in np.nonzero(cyl)[0]:
            self.col_x[a] = self.dof_d

    # ---- state <-> unknown vector -----------------------------------------
    def gather(self):
        U = np.zeros(self.ndof)
        m = self.dof_u >= 0
        U[self.dof_u[m]] = self.u[m]
        m = self.dof_p >= 0
        U[self.dof_p[m]] = self.p[m]
        m = self.dof_x >= 0
        U[self.dof_x[m]] = self.x[m]
        m = self.dof_l >= 0
        U[self.dof_l[m]] = self.lam[m]
        if self.has_body:
            U[self.dof_d] = self.delta
        return U

    def scatter(self, U):
        m = self.dof_u >= 0
        self.u[m] = U[self.dof_u[m]]
        m = self.dof_p >= 0
        self.p[m] = U[self.dof_p[m]]
        m = self.dof_x >= 0
        self.x[m] = U[self.dof_x[m]]
        m = self.dof_l >= 0
        self.lam[m] = U[self.dof_l[m]]
        if self.has_body:
            self.delta = U[self.dof_d].copy()
            self.x[self.cyl] = self.X[self.cyl] + self.delta

    # ---- time discretisation ------------------------------------------------
    def bdf_coefficients(self):
        """(c0, hu, hx): nodal rates are c0*v + h (BDF1 first step, then BDF2).

        BDF2 with a step ratio w = dt / dt_prev is the derivative at t^{n+1} of the
        quadratic through (t^{n-1}, v^{n-1}), (t^n, v^n), (t^{n+1}, v^{n+1}):
        v' = [(1 + 2w)/(1 + w) v^{n+1} - (1 + w) v^n + w^2/(1 + w) v^{n-1}] / dt,
        which is (3 v^{n+1} - 4 v^n + v^{n-1}) / (2 dt) for equal steps."""
        dt = self.dt
        if self.hist is None:
            return 1.0 / dt, -self.u_n / dt, -self.x_n / dt
        u_nm1, x_nm1 = self.hist
        w = dt / self.dt_prev
        c0 = (1 + 2 * w) / ((1 + w) * dt)
        a_n, a_nm1 = -(1 + w) / dt, w * w / ((1 + w) * dt)
        return c0, a_n * self.u_n + a_nm1 * u_nm1, a_n * self.x_n + a_nm1 * x_nm1

    def cfl(self):
        """dt max_e (max_a |u_a| / h_e): velocity magnitude over the element's
        nodes, h_e its shortest edge between corner nodes in the current
        configuration (the convective Courant number of Section 6's adaptive
        time stepping)."""
        c = self.conn
        corners = self.x[c[:, [0, 2, 8, 6]]]
        h = np.min(np.linalg.norm(corners - np.roll(corners, -1, axis=1), axis=2), axis=1)
        umax = np.max(np.linalg.norm(self.u[c], axis=2), axis=1)
        return float(self.dt * np.max(umax / h))

    def next_dt(self, cfl, cfl_target, dt_max=0.0):
        """Step size after a step of size dt that ended at Courant number cfl:
        dt (cfl_target / cfl), kept within [dt / 2, 1.2 dt] (a step ratio below
        1 + sqrt 2 keeps variable-step BDF2 zero-stable) and below dt_max."""
        r = cfl_target / cfl if cfl > 0 else 1.2
        dt = self.dt * min(1.2, max(0.5, r))
        return min(dt, dt_max) if dt_max > 0 else dt

    # ---- residual ----------------------------------------------------------
    def _element_inputs(self, u, p, x, hu, hx):
        c = self.conn
        pe = p[c[:, fem.VERTEX_LOCAL]]
        return self.X[c], x[c], u[c], pe, hu[c], hx[c]

    def residual_parts(self, u, p, x, lam, delta, c0, hu, hx, t):
        """Nodal residual arrays (complex-capable) for the given state."""
        n = self.n
        Xe, xe, ue, pe, hue, hxe = self._element_inputs(u, p, x, hu, hx)
        Ru_e, Rp_e, Rx_e = fem.volume_residual(Xe, xe, ue, pe, hue, hxe, c0, self.rho, self.mu,
                                               self.lam_s, self.mu_s, self.src, t)
        dt_ = Ru_e.dtype
        Ru = np.zeros((n, 2), dt_)
        Rp = np.zeros(n, dt_)
        Rx = np.zeros((n, 2), dt_)
        Rl = np.zeros((n, 2), dt_)
        np.add.at(Ru, self.conn, Ru_e)
        np.add.at(Rp, self.conn[:, fem.VERTEX_LOCAL], Rp_e)
        np.add.at(Rx, self.conn, Rx_e)
        Rd = self.k * delta.astype(dt_)
        if len(self.faces):
            f = self.faces
            Ruf, Rlf, Rdf = fem.gamma_residual(self.X[f], x[f], u[f], lam[f], hx[f], c0, self.src, t)
            np.add.at(Ru, f, Ruf)
            np.add.at(Rl, f, Rlf)
            Rd = Rd + Rdf.sum(axis=0)
            if self.src is not None:
                Rd = Rd - self.src.border(t)
        return Ru, Rp, Rx, Rl, Rd

    def residual_vector(self, parts):
        Ru, Rp, Rx, Rl, Rd = parts
        R = np.zeros(self.ndof, dtype=Ru.dtype)
        m = self.dof_u >= 0
        R[self.dof_u[m]] = Ru[m]
        m = self.dof_p >= 0
        R[self.dof_p[m]] = Rp[m]
        m = self.dof_x >= 0
        R[self.dof_x[m]] = Rx[m]
        m = self.dof_l >= 0
        R[self.dof_l[m]] = Rl[m]
        if self.has_body:
            R[self.dof_d] = Rd
        return R

    def residual(self, c0, hu, hx, t):
        return self.residual_vector(self.residual_parts(self.u, self.p, self.x, self.lam,
                                                        self.delta, c0, hu, hx, t))

    # ---- Jacobian by element-local complex step ----------------------------
    def jacobian(self, c0, hu, hx, t):
        """Sparse J = dNL/dU (Section 3.2), assembled from element Jacobians
        that are complex-step derivatives of the element residual."""
        rows, cols, vals = [], [], []
        c = self.conn
        E = len(c)
        Xe, xe, ue, pe, hue, hxe = self._element_inputs(self.u, self.p, self.x, hu, hx)
        vert = c[:, fem.VERTEX_LOCAL]
        row_u = self.dof_u[c]                 # (E,9,2)
        row_p = self.dof_p[vert]              # (E,4)
        row_x = self.dof_x[c]                 # Gamma and fixed rows are -1
        col_u, col_p, col_x = row_u, row_p, self.col_x[c]

        def emit(R_parts, col):
            Ru_e, Rp_e, Rx_e = R_parts
            for r_idx, R in ((row_u, Ru_e), (row_p, Rp_e), (row_x, Rx_e)):
                d = R.imag / H_CS
                m = (r_idx >= 0) & (col[(slice(None),) + (None,) * (r_idx.ndim - 1)] >= 0) & (d != 0)
                cc = np.broadcast_to(col[(slice(None),) + (None,) * (r_idx.ndim - 1)], r_idx.shape)
                rows.append(r_idx[m]); cols.append(cc[m]); vals.append(d[m])

        # one complex perturbation per local input; perturbations are stacked
        # along the element axis in chunks to keep numpy calls large
        local = [("u", a, i) for a in range(9) for i in range(2)] + \
                [("x", a, i) for a in range(9) for i in range(2)] + [("p", c_, 0) for c_ in range(4)]
        chunk = max(1, 200000 // max(E, 1))
        for s0 in range(0, len(local), chunk):
            part = local[s0:s0 + chunk]
            P = len(part)
            ue_c = np.tile(ue.astype(complex), (P, 1, 1))
            xe_c = np.tile(xe.astype(complex), (P, 1, 1))
            pe_c = np.tile(pe.astype(complex), (P, 1))
            for k_, (kind, a, i) in enumerate(part):
                sl = slice(k_ * E, (k_ + 1) * E)
                if kind == "u":
                    ue_c[sl, a, i] += 1j * H_CS
                elif kind == "x":
                    xe_c[sl, a, i] += 1j * H_CS
                else:
                    pe_c[sl, a] += 1j * H_CS
            parts = fem.volume_residual(np.tile(Xe, (P, 1, 1)), xe_c, ue_c, pe_c,
                                        np.tile(hue, (P, 1, 1)), np.tile(hxe, (P, 1, 1)),
                                        c0, self.rho, self.mu, np.tile(self.lam_s, P),
                                        np.tile(self.mu_s, P), self.src, t)
            for k_, (kind, a, i) in enumerate(part):
                sl = slice(k_ * E, (k_ + 1) * E)
                col = col_u[:, a, i] if kind == "u" else (col_x[:, a, i] if kind == "x" else col_p[:, a])
                emit(tuple(r[sl] for r in parts), col)
        if len(self.faces):
            f = self.faces
            Xf, xf, uf, lf, hxf = self.X[f], self.x[f], self.u[f], self.lam[f], hx[f]
            r_u, r_l = self.dof_u[f], self.dof_l[f]
            for b in range(3):
                for i in range(2):
                    for which in ("u", "x", "l"):
                        uf_c, xf_c, lf_c = uf.astype(complex), xf.astype(complex), lf.astype(complex)
                        if which == "u":
                            uf_c[:, b, i] += 1j * H_CS
                            col = r_u[:, b, i]
                        elif which == "x":
                            xf_c[:, b, i] += 1j * H_CS
                            col = self.col_x[f][:, b, i]
                        else:
                            lf_c[:, b, i] += 1j * H_CS
                            col = r_l[:, b, i]
                        Ru, Rl, Rd = fem.gamma_residual(Xf, xf_c, uf_c, lf_c, hxf, c0, self.src, t)
                        for r_idx, R in ((r_u, Ru), (r_l, Rl)):
                            d = R.imag / H_CS
                            m = (r_idx >= 0) & (col[:, None, None] >= 0) & (d != 0)
                            cc = np.broadcast_to(col[:, None, None], r_idx.shape)
                            rows.append(r_idx[m]); cols.append(cc[m]); vals.append(d[m])
                        d = Rd.imag / H_CS
                        rr = np.broadcast_to(self.dof_d[None, :], d.shape)
                        m = (col[:, None] >= 0) & (d != 0)
                        cc = np.broadcast_to(col[:, None], d.shape)
                        rows.append(rr[m]); cols.append(cc[m]); vals.append(d[m])
            # k * delta in the border rows
            rows.append(self.dof_d); cols.append(self.dof_d); vals.append(np.full(2, self.k))
        r = np.concatenate(rows); cc = np.concatenate(cols); v = np.concatenate(vals)
        return sp.coo_matrix((v, (r, cc)), shape=(self.ndof, self.ndof)).tocsr()

    # ---- one time step --------------------------------------------------------
    def step(self, tol=1e-10, max_newton=25, dirichlet=None, verbose=False):
        """Advance one BDF step with Newton-Raphson; returns the list of
        residual norms (one per residual evaluation)."""
        self.u_n, self.x_n = self.u.copy(), self.x.copy()
        c0, hu, hx = self.bdf_coefficients()
        t_new = self.t + self.dt
        if dirichlet is not None:
            dirichlet(self, t_new)
        norms = []
        extra = False   # the one Newton iteration taken after the test has passed
        for it in range(max_newton + 2):
            R = self.residual(c0, hu, hx, t_new)
            nr = float(np.linalg.norm(R))
            norms.append(nr)
            if verbose:
                print(f"  newton {it}: |R| = {nr:.3e}")
            if nr <= tol:
                if extra or it == 0:
                    break
                extra = True
            elif it >= max_newton:
                raise RuntimeError(f"Newton did not converge: {norms}")
            J = self.jacobian(c0, hu, hx, t_new)
            dU = sparse_lu(J).solve(-R)
            self.scatter(self.gather() + dU)
        self.hist = (self.u_n, self.x_n)
        self.t = t_new
        self.nstep += 1
        self.dt_prev = self.dt
        return norms

    def step_adaptive(self, cfl_target, dt_max=0.0, **kw):
        """One step with the current dt, then the next dt from the Courant number
        of the new state (Section 6: a target CFL of 1 as a simple convection
        error estimator).  Returns (norms, dt used, cfl reached)."""
        dt = self.dt
        norms = self.step(**kw)
        cfl = self.cfl()
        self.dt = self.next_dt(cfl, cfl_target, dt_max)
        return norms, dt, cfl

    def force(self):
        """F_fluid = -int_Gamma lambda on the current boundary."""
        if not len(self.faces):
            return np.zeros(2)
        f = self.faces
        z = np.zeros((len(f), 3, 2))
        _, _, Rd = fem.gamma_residual(self.X[f], self.x[f], z, self.lam[f], z, 0.0)
        return -Rd.sum(axis=0)


def viv_oracle_case(mesh, Re, Ustar, dt, u0, U_inf=1.0, D=1.0, rho=1.0):
    """Cylinder VIV case: mu from Re = rho U D / mu, k from the reduced velocity."""
    mu = rho * U_inf * D / Re
    k = stiffness_from_reduced_velocity(rho, U_inf, Ustar)
    return OracleCase(mesh, rho=rho, mu=mu, k=k, dt=dt, u0=u0)
