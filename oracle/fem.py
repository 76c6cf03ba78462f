"""Q2-Q1 finite element routines of the oracle (plain numpy, FP64/complex128).

Test infrastructure: only tests, the smoke check and the CPU baseline use it.

Follows the paper's weak form (Eq. weak_system) and nonlinear functional
(Eq. nonlinear_functional), restated for quadrilaterals:
  velocity u and mesh position x: continuous Q2 (9-node quads),
  pressure p: continuous Q1 on the element vertices,
  multiplier lambda: Q2 traces on the cylinder boundary Gamma.
The paper's own spaces are simplicial P2-P1 with a P1 position (Section 3.3);
the quadrilateral Q2-Q1 / Q2-position choice is the reading taken here.

Every function accepts complex arrays so that the Jacobian can be formed by
complex-step differentiation: J v = Im NL(U + i h v) / h, which is the
Gateaux derivative of Section 3.2 to rounding for h = 1e-30.

Parity: pinned by the closed-form translating-box solution (exact to
rounding), manufactured-solution convergence rates, the area identity,
patch tests and central finite differences (tests/test_oracle_fem.py,
tests/test_oracle_mms.py).
"""
from __future__ import annotations

import numpy as np

# ---- 1-D building blocks on [0, 1] ------------------------------------------
_G = np.sqrt(15.0) / 10.0
GAUSS3_PTS = np.array([0.5 - _G, 0.5, 0.5 + _G])
GAUSS3_WTS = np.array([5.0, 8.0, 5.0]) / 18.0


def lagrange2(s):
    """Quadratic Lagrange polynomials on nodes 0, 1/2, 1 and their derivatives."""
    s = np.asarray(s, dtype=np.float64)
    L = np.stack([(1 - s) * (1 - 2 * s), 4 * s * (1 - s), s * (2 * s - 1)], axis=-1)
    dL = np.stack([4 * s - 3, 4 - 8 * s, 4 * s - 1], axis=-1)
    return L, dL


def lagrange1(s):
    s = np.asarray(s, dtype=np.float64)
    return np.stack([1 - s, s], axis=-1), np.stack([-np.ones_like(s), np.ones_like(s)], axis=-1)


# ---- 2-D tensor-product tables at the 3x3 Gauss points -----------------------
VERTEX_LOCAL = np.array([0, 2, 6, 8])      # local node index of the Q1 vertices


def q2_tables():
    """N (9 qp, 9), dN (9 qp, 9, 2), M (9 qp, 4) and weights (9,).
    qp index = 3*j + i (i along xi); node index = 3*b + a (a along xi)."""
    L, dL = lagrange2(GAUSS3_PTS)
    l1, _ = lagrange1(GAUSS3_PTS)
    N = np.zeros((9, 9))
    dN = np.zeros((9, 9, 2))
    M = np.zeros((9, 4))
    W = np.zeros(9)
    for j in range(3):
        for i in range(3):
            q = 3 * j + i
            W[q] = GAUSS3_WTS[i] * GAUSS3_WTS[j]
            for b in range(3):
                for a in range(3):
                    N[q, 3 * b + a] = L[i, a] * L[j, b]
                    dN[q, 3 * b + a, 0] = dL[i, a] * L[j, b]
                    dN[q, 3 * b + a, 1] = L[i, a] * dL[j, b]
            for d in range(2):
                for c in range(2):
                    M[q, 2 * d + c] = l1[i, c] * l1[j, d]
    return N, dN, M, W


N_Q, DN_Q, M_Q, W_Q = q2_tables()
L_EDGE, DL_EDGE = lagrange2(GAUSS3_PTS)     # (3 qp, 3 nodes) along a Q2 edge


def _inv2(J):
    """Inverse and determinant of a stack of 2x2 matrices J[..., i, j]."""
    det = J[..., 0, 0] * J[..., 1, 1] - J[..., 0, 1] * J[..., 1, 0]
    inv = np.empty_like(J)
    inv[..., 0, 0] = J[..., 1, 1] / det
    inv[..., 1, 1] = J[..., 0, 0] / det
    inv[..., 0, 1] = -J[..., 0, 1] / det
    inv[..., 1, 0] = -J[..., 1, 0] / det
    return inv, det


def physical_gradients(coords, q):
    """Geometry at quadrature point q of each element.

    coords: (E, 9, 2) nodal coordinates (reference X or current x).
    Returns g (E, 9, 2) with g[e, a, :] = grad N_a (= J^{-T} grad_xi N_a) and
    det J (E,), where J_ij = d coord_i / d xi_j.
    """
    J = np.matmul(np.swapaxes(coords, 1, 2), DN_Q[q])      # J_ij = sum_a coord_a,i dN_a/dxi_j
    Jinv, det = _inv2(J)
    g = np.matmul(DN_Q[q], Jinv)                            # g_a,i = sum_j dN_a/dxi_j Jinv_ji
    return g, det


def element_areas(Xe):
    """|K0| = sum_q det J0 w_q for each element (reference configuration)."""
    area = np.zeros(Xe.shape[0])
    for q in range(9):
        _, det0 = physical_gradients(Xe, q)
        area = area + det0 * W_Q[q]
    return area


def volume_residual(Xe, xe, ue, pe, hu, hx, c0, rho, mu, lam_s, mu_s, src=None, t=0.0):
    """Element contributions to NL(U) for the volume terms (Eq. weak_system).

    Xe, xe, ue, hu, hx: (E, 9, 2); pe: (E, 4); lam_s, mu_s: (E,).
    The nodal ALE rates are u_dot_a = c0 u_a + hu_a and w_a = c0 x_a + hx_a
    (BDF along node trajectories; w = d_t x is the mesh velocity).

      Ru[a, i] = int_Omega_t  N_a rho (u_dot + ((u - w).grad) u)_i
                              + (grad N_a)_j sigma_ij,  sigma = -p I + 2 mu d(u)
      Rp[c]    = - int_Omega_t M_c div u
      Rx[a, i] = int_Omega_0  lam_s (grad_X N_a)_i (div_X x - d)
                              + 2 mu_s (grad_X N_a)_j eps_ij,
                 eps = (grad_X x + grad_X x^T)/2 - I = sym grad_X (x - X)
    `src` (manufactured solutions only) supplies f_u, g_p, f_x at the
    reference quadrature points: Ru -= int N f_u, Rp += int M g_p,
    Rx -= int_Omega_0 N f_x.
    """
    E = Xe.shape[0]
    dt_ = np.result_type(xe, ue, pe, hu, hx)
    Ru = np.zeros((E, 9, 2), dtype=dt_)
    Rp = np.zeros((E, 4), dtype=dt_)
    Rx = np.zeros((E, 9, 2), dtype=dt_)
    udot_n = c0 * ue + hu
    w_n = c0 * xe + hx
    for q in range(9):
        N = N_Q[q]
        M = M_Q[q]
        wq = W_Q[q]
        # current configuration (depends on the unknown positions)
        g, det = physical_gradients(xe, q)
        u = np.matmul(N, ue)
        udot = np.matmul(N, udot_n)
        w = np.matmul(N, w_n)
        L = np.matmul(np.swapaxes(ue, 1, 2), g)          # L_ij = du_i/dx_j
        p = np.matmul(pe, M)
        conv = np.matmul(L, (u - w)[:, :, None])[:, :, 0]
        sigma = (mu * (L + np.swapaxes(L, 1, 2))).astype(dt_)
        sigma[:, 0, 0] -= p
        sigma[:, 1, 1] -= p
        inertia = rho * (udot + conv)
        Ru += wq * det[:, None, None] * (N[None, :, None] * inertia[:, None, :]
                                         + np.matmul(g, np.swapaxes(sigma, 1, 2)))
        divu = L[:, 0, 0] + L[:, 1, 1]
        Rp += wq * det[:, None] * (-M[None, :] * divu[:, None])
        # reference configuration (fixed)
        g0, det0 = physical_gradients(Xe, q)
        # eps = sym(grad_X x) - I, formed from the displacement x - X: identical
        # because grad_X X = I for the isoparametric map, without the cancellation
        # of O(|x|) terms against the identity
        Fd = np.matmul(np.swapaxes(xe - Xe, 1, 2), g0)     # d(x - X)_i / dX_j
        eps = 0.5 * (Fd + np.swapaxes(Fd, 1, 2))
        tr = eps[:, 0, 0] + eps[:, 1, 1]
        Rx += wq * det0[:, None, None] * (lam_s[:, None, None] * g0 * tr[:, None, None]
                                          + 2.0 * mu_s[:, None, None] * np.matmul(g0, np.swapaxes(eps, 1, 2)))
        if src is not None:
            Xq = np.matmul(N, Xe)
            fu, gp, fx = src.volume(Xq, t)
            Ru -= wq * det[:, None, None] * N[None, :, None] * fu[:, None, :]
            Rp += wq * det[:, None] * M[None, :] * gp[:, None]
            Rx -= wq * det0[:, None, None] * N[None, :, None] * fx[:, None, :]
    return Ru, Rp, Rx


def gamma_residual(Xf, xf, uf, lf, hxf, c0, src=None, t=0.0):
    """Contributions of one Q2 edge of Gamma (3 nodes, in order along the edge).

      Ru[b, i]   = - int_Gamma_t N_b lambda_i        (momentum, Eq. weak_system)
      Rl[b, i]   = - int_Gamma_t N_b (u - w)_i        (no-slip constraint)
      Rd[i]      =   int_Gamma_t lambda_i             (force in the border row)
    Xf, xf, uf, lf, hxf: (F, 3, 2).  ds is measured on the current edge.
    `src` adds the manufactured no-slip data: Rl += int N g_l.
    """
    F_ = xf.shape[0]
    dt_ = np.result_type(xf, uf, lf, hxf)
    Ru = np.zeros((F_, 3, 2), dtype=dt_)
    Rl = np.zeros((F_, 3, 2), dtype=dt_)
    Rd = np.zeros((F_, 2), dtype=dt_)
    w_n = c0 * xf + hxf
    for q in range(3):
        N = L_EDGE[q]
        dN = DL_EDGE[q]
        tang = np.einsum('b,ebi->ei', dN, xf)
        ds = np.sqrt(tang[:, 0] ** 2 + tang[:, 1] ** 2) * GAUSS3_WTS[q]
        lam = np.einsum('b,ebi->ei', N, lf)
        u = np.einsum('b,ebi->ei', N, uf)
        w = np.einsum('b,ebi->ei', N, w_n)
        Ru -= ds[:, None, None] * N[None, :, None] * lam[:, None, :]
        rl = u - w
        if src is not None:
            Xq = np.einsum('b,ebi->ei', N, Xf)
            rl = rl - src.gamma(Xq, t)
        Rl -= ds[:, None, None] * N[None, :, None] * rl[:, None, :]
        Rd += ds[:, None] * lam
    return Ru, Rl, Rd
