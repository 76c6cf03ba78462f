"""Oracle case on P2-P1 triangles with a P1 mesh position (test
infrastructure; FP64, slow, plain) - the paper's own discretisation
(Section 3.3).

Unknowns, BDF time stepping, Newton iteration, the Gamma aliasing to delta
and the border rows are those of the 2-D Q2 case (`solver.OracleCase`); what
changes is where the position lives:
  * the position unknowns sit at the triangle vertices only; a midside
    node's position is the mean of its edge's end vertices (the P1 field
    evaluated there), kept in the nodal array for the Gamma-edge integrals
    and the output;
  * the pseudo-solid rows are the vertex rows (P1 test functions);
  * Gamma edges are straight, and the multiplier is the P2 trace on them
    (their vertices and midpoints);
  * lambda_s = mu_s = min|K_0| / |K_0| with triangle areas.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem, fem_tri
from .solver import OracleCase, H_CS, stiffness_from_reduced_velocity, U_FIX_X, U_FIX_Y, X_FIX_X, X_FIX_Y, CYL, P_FIX

VERT = np.array([0, 1, 2])


class OracleCaseTri(OracleCase):
    def __init__(self, mesh, rho, mu, k, dt, u0, lame="inverse_area", src=None):
        self.mesh = mesh
        self.X = np.asarray(mesh["X"], dtype=np.float64)
        self.conn = np.asarray(mesh["conn"], dtype=np.int64)
        self.tags = np.asarray(mesh["tags"], dtype=np.int64)
        gf = np.asarray(mesh["gamma_faces"], dtype=np.int64).reshape(-1, 2)
        self.faces = np.array([[self.conn[e, a] for a in fem_tri.EDGE_NODES[ed]] for e, ed in gf],
                              dtype=np.int64).reshape(-1, 3)
        self.rho, self.mu, self.k, self.dt = rho, mu, k, dt
        self.dt_prev = dt
        self.src = src
        n = len(self.X)
        self.n = n
        # midside node -> its edge's end vertices
        self.mid_parent = -np.ones((n, 2), np.int64)
        for m_, a, b in fem_tri.MID_EDGES:
            self.mid_parent[self.conn[:, m_], 0] = self.conn[:, a]
            self.mid_parent[self.conn[:, m_], 1] = self.conn[:, b]
        self.is_mid = self.mid_parent[:, 0] >= 0
        area = fem_tri.element_areas(self.X[self.conn[:, VERT]])
        self.lam_s = area.min() / area if lame == "inverse_area" else np.full(len(self.conn), float(lame))
        self.mu_s = self.lam_s.copy()
        self._number_dofs()
        self.u = np.array(u0, dtype=np.float64).reshape(n, 2).copy()
        self.p = np.zeros(n)
        self.x = self.X.copy()
        self.lam = np.zeros((n, 2))
        self.delta = np.zeros(2)
        self.t = 0.0
        self.nstep = 0
        self.hist = None

    def _number_dofs(self):
        """u at every node, p and x at the vertices, lambda at the Gamma nodes,
        delta last (field-major, like the Q2 case)."""
        n, t = self.n, self.tags
        is_vertex = np.zeros(n, bool)
        is_vertex[self.conn[:, VERT].ravel()] = True
        self.is_vertex = is_vertex
        cyl = (t & CYL) != 0
        self.cyl = cyl
        idx = 0
        self.dof_u = -np.ones((n, 2), np.int64)
        for a in range(n):
            for i, bit in enumerate((U_FIX_X, U_FIX_Y)):
                if not t[a] & bit:
                    self.dof_u[a, i] = idx
                    idx += 1
        self.dof_p = -np.ones(n, np.int64)
        for a in range(n):
            if is_vertex[a] and not t[a] & P_FIX:
                self.dof_p[a] = idx
                idx += 1
        self.dof_x = -np.ones((n, 2), np.int64)
        for a in range(n):
            if cyl[a] or not is_vertex[a]:
                continue
            for i, bit in enumerate((X_FIX_X, X_FIX_Y)):
                if not t[a] & bit:
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
        self.col_x = self.dof_x.copy()
        for a in np.nonzero(cyl)[0]:
            self.col_x[a] = self.dof_d

    def _mids_from_vertices(self, x):
        m = self.is_mid
        x[m] = 0.5 * (x[self.mid_parent[m, 0]] + x[self.mid_parent[m, 1]])

    def scatter(self, U):
        super().scatter(U)
        self._mids_from_vertices(self.x)

    def cfl(self):
        raise NotImplementedError("the Courant number is defined for the Q2 case only")

    def _vertex_inputs(self, u, p, x, hu, hx):
        c = self.conn
        cv = c[:, VERT]
        return self.X[cv], x[cv], u[c], p[cv], hu[c], hx[cv]

    def residual_parts(self, u, p, x, lam, delta, c0, hu, hx, t):
        n = self.n
        Xv, xv, ue, pv, hue, hxv = self._vertex_inputs(u, p, x, hu, hx)
        Ru_e, Rp_e, Rx_e = fem_tri.volume_residual(Xv, xv, ue, pv, hue, hxv, c0, self.rho, self.mu,
                                                   self.lam_s, self.mu_s, self.src, t)
        dt_ = Ru_e.dtype
        Ru = np.zeros((n, 2), dt_)
        Rp = np.zeros(n, dt_)
        Rx = np.zeros((n, 2), dt_)
        Rl = np.zeros((n, 2), dt_)
        np.add.at(Ru, self.conn, Ru_e)
        np.add.at(Rp, self.conn[:, VERT], Rp_e)
        np.add.at(Rx, self.conn[:, VERT], Rx_e)
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

    def jacobian(self, c0, hu, hx, t):
        """Sparse J from complex-step element Jacobians (Section 3.2): the
        volume terms perturbed in u (6 nodes), the vertex positions and the
        vertex pressures; the Gamma-edge terms in u, lambda and (through delta)
        a rigid shift of the edge."""
        rows, cols, vals = [], [], []
        c = self.conn
        cv = c[:, VERT]
        E = len(c)
        Xv, xv, ue, pv, hue, hxv = self._vertex_inputs(self.u, self.p, self.x, hu, hx)
        row_u, row_p, row_x = self.dof_u[c], self.dof_p[cv], self.dof_x[cv]
        col_u, col_p, col_x = row_u, row_p, self.col_x[cv]

        def emit(parts, col):
            for r_idx, R in zip((row_u, row_p, row_x), parts):
                d = R.imag / H_CS
                cb = col[(slice(None),) + (None,) * (r_idx.ndim - 1)]
                m = (r_idx >= 0) & (cb >= 0) & (d != 0)
                rows.append(r_idx[m]); cols.append(np.broadcast_to(cb, r_idx.shape)[m]); vals.append(d[m])

        local = [("u", a, i) for a in range(6) for i in range(2)] + \
                [("x", v, i) for v in range(3) for i in range(2)] + [("p", v, 0) for v in range(3)]
        P = len(local)
        ue_c = np.tile(ue.astype(complex), (P, 1, 1))
        xv_c = np.tile(xv.astype(complex), (P, 1, 1))
        pv_c = np.tile(pv.astype(complex), (P, 1))
        for k_, (kind, a, i) in enumerate(local):
            sl = slice(k_ * E, (k_ + 1) * E)
            if kind == "u":
                ue_c[sl, a, i] += 1j * H_CS
            elif kind == "x":
                xv_c[sl, a, i] += 1j * H_CS
            else:
                pv_c[sl, a] += 1j * H_CS
        parts = fem_tri.volume_residual(np.tile(Xv, (P, 1, 1)), xv_c, ue_c, pv_c, np.tile(hue, (P, 1, 1)),
                                        np.tile(hxv, (P, 1, 1)), c0, self.rho, self.mu, np.tile(self.lam_s, P),
                                        np.tile(self.mu_s, P), self.src, t)
        for k_, (kind, a, i) in enumerate(local):
            sl = slice(k_ * E, (k_ + 1) * E)
            col = col_u[:, a, i] if kind == "u" else (col_x[:, a, i] if kind == "x" else col_p[:, a])
            emit(tuple(r[sl] for r in parts), col)
        if len(self.faces):
            f = self.faces
            Xf, xf, uf, lf, hxf = self.X[f], self.x[f], self.u[f], self.lam[f], hx[f]
            r_u, r_l = self.dof_u[f], self.dof_l[f]

            def emit_face(Ru, Rl, Rd, col):
                for r_idx, R in ((r_u, Ru), (r_l, Rl)):
                    d = R.imag / H_CS
                    m = (r_idx >= 0) & (col[:, None, None] >= 0) & (d != 0)
                    rows.append(r_idx[m]); cols.append(np.broadcast_to(col[:, None, None], r_idx.shape)[m])
                    vals.append(d[m])
                d = Rd.imag / H_CS
                m = (col[:, None] >= 0) & (d != 0)
                rows.append(np.broadcast_to(self.dof_d[None, :], d.shape)[m])
                cols.append(np.broadcast_to(col[:, None], d.shape)[m]); vals.append(d[m])

            for b in range(3):
                for i in range(2):
                    for which in ("u", "l"):
                        uf_c, lf_c = uf.astype(complex), lf.astype(complex)
                        if which == "u":
                            uf_c[:, b, i] += 1j * H_CS
                            col = r_u[:, b, i]
                        else:
                            lf_c[:, b, i] += 1j * H_CS
                            col = r_l[:, b, i]
                        emit_face(*fem.gamma_residual(Xf, xf.astype(complex), uf_c, lf_c, hxf, c0, self.src, t), col)
            for i in range(2):   # delta_i: every node of the edge moves by the same shift
                xf_c = xf.astype(complex)
                xf_c[:, :, i] += 1j * H_CS
                emit_face(*fem.gamma_residual(Xf, xf_c, uf.astype(complex), lf.astype(complex), hxf, c0,
                                              self.src, t), np.full(len(f), self.dof_d[i]))
            rows.append(self.dof_d); cols.append(self.dof_d); vals.append(np.full(2, self.k))
        r = np.concatenate(rows); cc = np.concatenate(cols); v = np.concatenate(vals)
        return sp.coo_matrix((v, (r, cc)), shape=(self.ndof, self.ndof)).tocsr()


def viv_oracle_case_tri(mesh, Re, Ustar, dt, u0, U_inf=1.0, D=1.0, rho=1.0):
    mu = rho * U_inf * D / Re
    k = stiffness_from_reduced_velocity(rho, U_inf, Ustar)
    return OracleCaseTri(mesh, rho=rho, mu=mu, k=k, dt=dt, u0=u0)
