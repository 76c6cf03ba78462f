"""Q2-Q1 hexahedral element routines of the oracle (plain numpy, FP64/complex128).

Test infrastructure: only tests, the smoke check and the CPU baseline use it.

The three-dimensional form of the weak system of Section 3 (Eq. weak_system)
on 27-node hexahedra: velocity u and mesh position x continuous Q2, pressure
continuous Q1 on the eight vertices, multiplier lambda the Q2 trace on the
cylinder surface Gamma (9-node faces).  The integrands are those of the 2-D
routines in `fem.py`, with every index running over three components.

Local numbering: node 9 c + 3 b + a (a along xi, b along eta, c along zeta),
Gauss point 9 k + 3 j + i, pressure vertex 4 f + 2 d + c0 (local node
18 f + 6 d + 2 c0).  Faces: 0 xi=0, 1 xi=1, 2 eta=0, 3 eta=1, 4 zeta=0,
5 zeta=1; a face's 9 nodes are ordered 3 t + s with s along the first and t
along the second in-face reference direction (xi before eta before zeta).

Parity: pinned by the reduction of a z-independent state on an extruded mesh
to the pinned 2-D routines, by covariance under rotations of space, by the
closed-form translating box reproduced to rounding, and by the optimal
convergence orders of a manufactured solution (tests/test_oracle_3d.py).
"""
from __future__ import annotations

import numpy as np

from .fem import GAUSS3_PTS, GAUSS3_WTS, lagrange1, lagrange2, N_Q as N_FACE, DN_Q as DN_FACE, W_Q as W_FACE

VERTEX_LOCAL = np.array([0, 2, 6, 8, 18, 20, 24, 26])


def _face_nodes():
    out = []
    for f in range(6):
        axis, side = f // 2, 2 * (f % 2)
        nodes = []
        for t in range(3):
            for s in range(3):
                idx = [0, 0, 0]
                free = [ax for ax in range(3) if ax != axis]
                idx[axis] = side
                idx[free[0]] = s
                idx[free[1]] = t
                nodes.append(9 * idx[2] + 3 * idx[1] + idx[0])
        out.append(tuple(nodes))
    return tuple(out)


FACE_NODES = _face_nodes()


def hex_tables():
    """N (27 qp, 27), dN (27 qp, 27, 3), M (27 qp, 8) and weights (27,)."""
    L, dL = lagrange2(GAUSS3_PTS)
    l1, _ = lagrange1(GAUSS3_PTS)
    N = np.zeros((27, 27))
    dN = np.zeros((27, 27, 3))
    M = np.zeros((27, 8))
    W = np.zeros(27)
    for k in range(3):
        for j in range(3):
            for i in range(3):
                q = 9 * k + 3 * j + i
                W[q] = GAUSS3_WTS[i] * GAUSS3_WTS[j] * GAUSS3_WTS[k]
                for c in range(3):
                    for b in range(3):
                        for a in range(3):
                            n = 9 * c + 3 * b + a
                            N[q, n] = L[i, a] * L[j, b] * L[k, c]
                            dN[q, n, 0] = dL[i, a] * L[j, b] * L[k, c]
                            dN[q, n, 1] = L[i, a] * dL[j, b] * L[k, c]
                            dN[q, n, 2] = L[i, a] * L[j, b] * dL[k, c]
                for f in range(2):
                    for d in range(2):
                        for c0 in range(2):
                            M[q, 4 * f + 2 * d + c0] = l1[i, c0] * l1[j, d] * l1[k, f]
    return N, dN, M, W


N_Q, DN_Q, M_Q, W_Q = hex_tables()


def _inv3(J):
    """Inverse and determinant of a stack of 3x3 matrices (cofactor formula)."""
    a, b, c = J[..., 0, 0], J[..., 0, 1], J[..., 0, 2]
    d, e, f = J[..., 1, 0], J[..., 1, 1], J[..., 1, 2]
    g, h, i = J[..., 2, 0], J[..., 2, 1], J[..., 2, 2]
    A = e * i - f * h
    B = -(d * i - f * g)
    C = d * h - e * g
    det = a * A + b * B + c * C
    inv = np.empty_like(J)
    inv[..., 0, 0] = A / det
    inv[..., 1, 0] = B / det
    inv[..., 2, 0] = C / det
    inv[..., 0, 1] = -(b * i - c * h) / det
    inv[..., 1, 1] = (a * i - c * g) / det
    inv[..., 2, 1] = -(a * h - b * g) / det
    inv[..., 0, 2] = (b * f - c * e) / det
    inv[..., 1, 2] = -(a * f - c * d) / det
    inv[..., 2, 2] = (a * e - b * d) / det
    return inv, det


def physical_gradients(coords, q):
    """grad N_a (E, 27, 3) and det J (E,) at Gauss point q; coords (E, 27, 3)."""
    J = np.matmul(np.swapaxes(coords, 1, 2), DN_Q[q])      # J_ij = d coord_i / d xi_j
    Jinv, det = _inv3(J)
    return np.matmul(DN_Q[q], Jinv), det


def element_volumes(Xe):
    vol = np.zeros(Xe.shape[0])
    for q in range(27):
        _, det0 = physical_gradients(Xe, q)
        vol = vol + det0 * W_Q[q]
    return vol


def volume_residual(Xe, xe, ue, pe, hu, hx, c0, rho, mu, lam_s, mu_s, src=None):
    """Element volume terms of Eq. weak_system on hexahedra: with
    u_dot = c0 u + hu, w = c0 x + hx (nodal rates),
      Ru[a,i] = int_Ot N_a rho (u_dot + ((u - w).grad) u)_i + (grad N_a)_j sigma_ij,
      Rp[c]   = -int_Ot M_c div u,
      Rx[a,i] = int_O0 lam_s (grad_X N_a)_i tr eps + 2 mu_s (grad_X N_a)_j eps_ij,
    sigma = -p I + mu (grad u + grad u^T), eps = sym grad_X (x - X).
    Xe, xe, ue, hu, hx: (E, 27, 3); pe: (E, 8); lam_s, mu_s: (E,).
    `src` (manufactured solutions only) supplies f_u, g_p at the current
    physical quadrature points and f_x at the reference ones:
    Ru -= int N f_u, Rp += int M g_p, Rx -= int_O0 N f_x."""
    E = Xe.shape[0]
    dt_ = np.result_type(xe, ue, pe, hu, hx)
    Ru = np.zeros((E, 27, 3), dtype=dt_)
    Rp = np.zeros((E, 8), dtype=dt_)
    Rx = np.zeros((E, 27, 3), dtype=dt_)
    udot_n = c0 * ue + hu
    w_n = c0 * xe + hx
    eye = np.eye(3)
    for q in range(27):
        N, M, wq = N_Q[q], M_Q[q], W_Q[q]
        g, det = physical_gradients(xe, q)
        u = np.matmul(N, ue)
        udot = np.matmul(N, udot_n)
        w = np.matmul(N, w_n)
        L = np.matmul(np.swapaxes(ue, 1, 2), g)          # L_ij = du_i/dx_j
        p = np.matmul(pe, M)
        conv = np.matmul(L, (u - w)[:, :, None])[:, :, 0]
        sigma = mu * (L + np.swapaxes(L, 1, 2)) - p[:, None, None] * eye
        inertia = rho * (udot + conv)
        Ru += wq * det[:, None, None] * (N[None, :, None] * inertia[:, None, :]
                                         + np.matmul(g, np.swapaxes(sigma, 1, 2)))
        divu = L[:, 0, 0] + L[:, 1, 1] + L[:, 2, 2]
        Rp += wq * det[:, None] * (-M[None, :] * divu[:, None])
        g0, det0 = physical_gradients(Xe, q)
        Fd = np.matmul(np.swapaxes(xe - Xe, 1, 2), g0)     # d(x - X)_i / dX_j
        eps = 0.5 * (Fd + np.swapaxes(Fd, 1, 2))
        tr = eps[:, 0, 0] + eps[:, 1, 1] + eps[:, 2, 2]
        Rx += wq * det0[:, None, None] * (lam_s[:, None, None] * g0 * tr[:, None, None]
                                          + 2.0 * mu_s[:, None, None] * np.matmul(g0, np.swapaxes(eps, 1, 2)))
        if src is not None:
            fu, gp, fx = src.volume_at(np.matmul(N, xe), np.matmul(N, Xe), 0.0)
            Ru -= wq * det[:, None, None] * N[None, :, None] * fu[:, None, :]
            Rp += wq * det[:, None] * M[None, :] * gp[:, None]
            Rx -= wq * det0[:, None, None] * N[None, :, None] * fx[:, None, :]
    return Ru, Rp, Rx


def gamma_residual(xf, uf, lf, hxf, c0):
    """Terms of one 9-node face of Gamma (nodes in face order):
      Ru[b,i] = -int N_b lambda_i dA,  Rl[b,i] = -int N_b (u - w)_i dA,
      Rd[i]   =  int lambda_i dA,
    dA = |dx/ds x dx/dt| ds dt on the current face, 3x3 Gauss points."""
    F_ = xf.shape[0]
    dt_ = np.result_type(xf, uf, lf, hxf)
    Ru = np.zeros((F_, 9, 3), dtype=dt_)
    Rl = np.zeros((F_, 9, 3), dtype=dt_)
    Rd = np.zeros((F_, 3), dtype=dt_)
    w_n = c0 * xf + hxf
    for q in range(9):
        N = N_FACE[q]
        t1 = np.einsum('b,ebi->ei', DN_FACE[q, :, 0], xf)
        t2 = np.einsum('b,ebi->ei', DN_FACE[q, :, 1], xf)
        nrm = np.stack([t1[:, 1] * t2[:, 2] - t1[:, 2] * t2[:, 1],
                        t1[:, 2] * t2[:, 0] - t1[:, 0] * t2[:, 2],
                        t1[:, 0] * t2[:, 1] - t1[:, 1] * t2[:, 0]], 1)
        dA = np.sqrt(nrm[:, 0] ** 2 + nrm[:, 1] ** 2 + nrm[:, 2] ** 2) * W_FACE[q]
        lam = np.einsum('b,ebi->ei', N, lf)
        rl = np.einsum('b,ebi->ei', N, uf) - np.einsum('b,ebi->ei', N, w_n)
        Ru -= dA[:, None, None] * N[None, :, None] * lam[:, None, :]
        Rl -= dA[:, None, None] * N[None, :, None] * rl[:, None, :]
        Rd += dA[:, None] * lam
    return Ru, Rl, Rd
