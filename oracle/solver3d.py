"""Oracle case on hexahedral meshes, periodic in z (test infrastructure; FP64,
slow, plain).

The unknowns, time stepping and Newton iteration are those of the 2-D oracle
case (`solver.OracleCase`, Eq. NR_iteration, BDF2 with a BDF1 start), with
three velocity, position and multiplier components per node.  The readings
taken for the spanwise direction:
  * The cylinder moves rigidly in x and y only (two position unknowns delta,
    as in the paper's 3-D runs of Section 6): a Gamma node sits at
    x = X + (delta_x, delta_y, 0), so its z position stays at X_z.  The
    border rows are k delta + int_Gamma lambda_{x,y} = 0 (Eq. solid_balance,
    with k the stiffness of the whole span).
  * The multiplier has three components: the no-slip condition u = w holds
    for every component on Gamma.
  * Periodicity in z is on the displacement x - X and on u, p, lambda: an
    element whose nodes wrap across the seam sees them at their stored
    coordinates + span e_z (reference and current alike); the mesh velocity
    w = c0 x + hx is formed from the stored positions, so the seam shift,
    constant in time, does not enter it.
  * Lame coefficients lambda_s = mu_s = min|K_0| / |K_0| with element volumes.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem3d
from .solver import OracleCase, H_CS, stiffness_from_reduced_velocity

U_FIX_X, U_FIX_Y, X_FIX_X, X_FIX_Y, CYL, P_FIX, U_FIX_Z, X_FIX_Z = 1, 2, 4, 8, 16, 64, 128, 256


class OracleCase3D(OracleCase):
    """State arrays: u (n,3), p (n,) [vertices], x (n,3), lam (n,3) [Gamma],
    delta (2,)."""

    def __init__(self, mesh, rho, mu, k, dt, u0, lame="inverse_volume", src=None):
        self.mesh = mesh
        self.X = np.asarray(mesh["X"], dtype=np.float64)
        self.conn = np.asarray(mesh["conn"], dtype=np.int64)
        self.tags = np.asarray(mesh["tags"], dtype=np.int64)
        self.span = float(mesh.get("span", 0.0))
        wrap = np.asarray(mesh.get("wrap", np.zeros(len(self.conn), np.int64)), dtype=np.int64)
        bits = (wrap[:, None] >> np.arange(27)[None, :]) & 1
        self.shift = np.zeros(self.conn.shape + (3,))          # (E, 27, 3) seam shift per local node
        self.shift[:, :, 2] = bits * self.span
        gf = np.asarray(mesh["gamma_faces"], dtype=np.int64).reshape(-1, 2)
        loc = np.array([fem3d.FACE_NODES[f] for f in gf[:, 1]], dtype=np.int64).reshape(-1, 9)
        self.faces = np.take_along_axis(self.conn[gf[:, 0]], loc, axis=1) if len(gf) else np.zeros((0, 9), np.int64)
        self.fshift = np.take_along_axis(self.shift[gf[:, 0]], loc[:, :, None], axis=1) if len(gf) \
            else np.zeros((0, 9, 3))
        self.rho, self.mu, self.k, self.dt = rho, mu, k, dt
        self.dt_prev = dt
        self.src = src   # (steady manufactured solutions only: no Gamma source)
        n = len(self.X)
        self.n = n
        vol = fem3d.element_volumes(self.X[self.conn] + self.shift)
        self.lam_s = vol.min() / vol if lame == "inverse_volume" else np.full(len(self.conn), float(lame))
        self.mu_s = self.lam_s.copy()
        self._number_dofs()
        self.u = np.array(u0, dtype=np.float64).reshape(n, 3).copy()
        self.p = np.zeros(n)
        self.x = self.X.copy()
        self.lam = np.zeros((n, 3))
        self.delta = np.zeros(2)
        self.t = 0.0
        self.nstep = 0
        self.hist = None

    def _number_dofs(self):
        """Field-major numbering like the 2-D case: u, p, x, lambda, delta."""
        n, t = self.n, self.tags
        is_vertex = np.zeros(n, bool)
        is_vertex[self.conn[:, fem3d.VERTEX_LOCAL].ravel()] = True
        self.is_vertex = is_vertex
        cyl = (t & CYL) != 0
        self.cyl = cyl
        idx = 0
        self.dof_u = -np.ones((n, 3), np.int64)
        free_u = np.stack([(t & U_FIX_X) == 0, (t & U_FIX_Y) == 0, (t & U_FIX_Z) == 0], axis=1)
        for a in range(n):
            for i in range(3):
                if free_u[a, i]:
                    self.dof_u[a, i] = idx
                    idx += 1
        self.dof_p = -np.ones(n, np.int64)
        for a in range(n):
            if is_vertex[a] and (t[a] & P_FIX) == 0:
                self.dof_p[a] = idx
                idx += 1
        self.dof_x = -np.ones((n, 3), np.int64)
        free_x = np.stack([(t & X_FIX_X) == 0, (t & X_FIX_Y) == 0, (t & X_FIX_Z) == 0], axis=1)
        for a in range(n):
            if cyl[a]:
                continue
            for i in range(3):
                if free_x[a, i]:
                    self.dof_x[a, i] = idx
                    idx += 1
        self.dof_l = -np.ones((n, 3), np.int64)
        for a in range(n):
            if cyl[a]:
                for i in range(3):
                    self.dof_l[a, i] = idx
                    idx += 1
        self.has_body = bool(cyl.any())
        self.dof_d = np.array([idx, idx + 1]) if self.has_body else -np.ones(2, np.int64)
        if self.has_body:
            idx += 2
        self.ndof = idx
        # Gamma nodes: x and y position columns are delta's, z is held
        self.col_x = self.dof_x.copy()
        for a in np.nonzero(cyl)[0]:
            self.col_x[a, :2] = self.dof_d
            self.col_x[a, 2] = -1

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
            self.x[self.cyl, :2] = self.X[self.cyl, :2] + self.delta
            self.x[self.cyl, 2] = self.X[self.cyl, 2]

    def cfl(self):
        raise NotImplementedError("the Courant number is defined for the 2-D case only")

    def _element_inputs(self, u, p, x, hu, hx):
        c = self.conn
        return (self.X[c] + self.shift, x[c] + self.shift, u[c], p[c[:, fem3d.VERTEX_LOCAL]], hu[c], hx[c])

    def _element_hx(self, hx, c0):
        # w = c0 (x + s) + hx_e must equal c0 x + hx: hx_e = hx - c0 s
        return hx[self.conn] - c0 * self.shift

    def residual_parts(self, u, p, x, lam, delta, c0, hu, hx, t):
        n = self.n
        Xe, xe, ue, pe, hue, _ = self._element_inputs(u, p, x, hu, hx)
        hxe = self._element_hx(hx, c0)
        Ru_e, Rp_e, Rx_e = fem3d.volume_residual(Xe, xe, ue, pe, hue, hxe, c0, self.rho, self.mu,
                                                 self.lam_s, self.mu_s, self.src)
        dt_ = Ru_e.dtype
        Ru = np.zeros((n, 3), dt_)
        Rp = np.zeros(n, dt_)
        Rx = np.zeros((n, 3), dt_)
        Rl = np.zeros((n, 3), dt_)
        np.add.at(Ru, self.conn, Ru_e)
        np.add.at(Rp, self.conn[:, fem3d.VERTEX_LOCAL], Rp_e)
        np.add.at(Rx, self.conn, Rx_e)
        Rd = self.k * delta.astype(dt_)
        if len(self.faces):
            f = self.faces
            Ruf, Rlf, Rdf = fem3d.gamma_residual(x[f] + self.fshift, u[f], lam[f], hx[f] - c0 * self.fshift, c0)
            np.add.at(Ru, f, Ruf)
            np.add.at(Rl, f, Rlf)
            Rd = Rd + Rdf[:, :2].sum(axis=0)
        return Ru, Rp, Rx, Rl, Rd

    def jacobian(self, c0, hu, hx, t):
        """Sparse J assembled from complex-step element Jacobians (Section 3.2)."""
        rows, cols, vals = [], [], []
        c = self.conn
        E = len(c)
        Xe, xe, ue, pe, hue, _ = self._element_inputs(self.u, self.p, self.x, hu, hx)
        hxe = self._element_hx(hx, c0)
        vert = c[:, fem3d.VERTEX_LOCAL]
        row_u, row_p, row_x = self.dof_u[c], self.dof_p[vert], self.dof_x[c]
        col_u, col_p, col_x = row_u, row_p, self.col_x[c]

        def emit(parts, col):
            for r_idx, R in zip((row_u, row_p, row_x), parts):
                d = R.imag / H_CS
                cb = col[(slice(None),) + (None,) * (r_idx.ndim - 1)]
                m = (r_idx >= 0) & (cb >= 0) & (d != 0)
                cc = np.broadcast_to(cb, r_idx.shape)
                rows.append(r_idx[m]); cols.append(cc[m]); vals.append(d[m])

        local = [("u", a, i) for a in range(27) for i in range(3)] + \
                [("x", a, i) for a in range(27) for i in range(3)] + [("p", c_, 0) for c_ in range(8)]
        chunk = max(1, 60000 // max(E, 1))
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
            parts = fem3d.volume_residual(np.tile(Xe, (P, 1, 1)), xe_c, ue_c, pe_c, np.tile(hue, (P, 1, 1)),
                                          np.tile(hxe, (P, 1, 1)), c0, self.rho, self.mu,
                                          np.tile(self.lam_s, P), np.tile(self.mu_s, P), self.src)
            for k_, (kind, a, i) in enumerate(part):
                sl = slice(k_ * E, (k_ + 1) * E)
                col = col_u[:, a, i] if kind == "u" else (col_x[:, a, i] if kind == "x" else col_p[:, a])
                emit(tuple(r[sl] for r in parts), col)
        if len(self.faces):
            f = self.faces
            xf = self.x[f] + self.fshift
            hxf = hx[f] - c0 * self.fshift
            uf, lf = self.u[f], self.lam[f]
            r_u, r_l, cx = self.dof_u[f], self.dof_l[f], self.col_x[f]
            for b in range(9):
                for i in range(3):
                    for which in ("u", "x", "l"):
                        uf_c, xf_c, lf_c = uf.astype(complex), xf.astype(complex), lf.astype(complex)
                        if which == "u":
                            uf_c[:, b, i] += 1j * H_CS
                            col = r_u[:, b, i]
                        elif which == "x":
                            xf_c[:, b, i] += 1j * H_CS
                            col = cx[:, b, i]
                        else:
                            lf_c[:, b, i] += 1j * H_CS
                            col = r_l[:, b, i]
                        Ru, Rl, Rd = fem3d.gamma_residual(xf_c, uf_c, lf_c, hxf, c0)
                        for r_idx, R in ((r_u, Ru), (r_l, Rl)):
                            d = R.imag / H_CS
                            m = (r_idx >= 0) & (col[:, None, None] >= 0) & (d != 0)
                            cc = np.broadcast_to(col[:, None, None], r_idx.shape)
                            rows.append(r_idx[m]); cols.append(cc[m]); vals.append(d[m])
                        d = Rd[:, :2].imag / H_CS
                        rr = np.broadcast_to(self.dof_d[None, :], d.shape)
                        m = (col[:, None] >= 0) & (d != 0)
                        cc = np.broadcast_to(col[:, None], d.shape)
                        rows.append(rr[m]); cols.append(cc[m]); vals.append(d[m])
            rows.append(self.dof_d); cols.append(self.dof_d); vals.append(np.full(2, self.k))
        r = np.concatenate(rows); cc = np.concatenate(cols); v = np.concatenate(vals)
        return sp.coo_matrix((v, (r, cc)), shape=(self.ndof, self.ndof)).tocsr()

    def force(self):
        """F_fluid = -int_Gamma lambda (x and y components)."""
        if not len(self.faces):
            return np.zeros(2)
        f = self.faces
        z = np.zeros((len(f), 9, 3))
        _, _, Rd = fem3d.gamma_residual(self.x[f] + self.fshift, z, self.lam[f], z, 0.0)
        return -Rd[:, :2].sum(axis=0)


def viv_oracle_case3d(mesh, Re, Ustar, dt, u0, U_inf=1.0, D=1.0, rho=1.0):
    """3-D cylinder case: mu from Re; k from the reduced velocity with the
    span as the length that carries the force."""
    mu = rho * U_inf * D / Re
    k = stiffness_from_reduced_velocity(rho, U_inf, Ustar, L=mesh["span"])
    return OracleCase3D(mesh, rho=rho, mu=mu, k=k, dt=dt, u0=u0)
