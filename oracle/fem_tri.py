"""Taylor-Hood P2-P1 triangle routines of the oracle with a P1 mesh position
(plain numpy, FP64/complex128).

Test infrastructure: only tests, the smoke check and the CPU baseline use it.

The paper's own spaces (Section 3.3): velocity continuous P2 on 6-node
triangles, pressure continuous P1, mesh position continuous P1 (the current
mesh has straight edges and an affine map per triangle), multiplier the P2
trace on Gamma.  The integrands are those of `fem.volume_residual`
(Eq. weak_system); the mesh velocity is the P1 interpolant of the vertex
rates w_v = c0 x_v + hx_v.

Local numbering: vertices 0, 1, 2, midpoints of edges 0-1, 1-2, 2-0 (3, 4,
5).  Barycentric l0 = 1 - s - t, l1 = s, l2 = t on the reference triangle
(0,0), (1,0), (0,1).  Quadrature: Radon's 7-point rule, exact for degree 5.

Parity: pinned by the rule's exactness on monomials, the basis' nodal and
partition-of-unity properties, the closed-form translating box reproduced to
rounding, central differences of the residual, and the convergence orders
Section 5.1 reports for these spaces (tests/test_oracle_tri.py).
"""
from __future__ import annotations

import numpy as np

_SQ15 = np.sqrt(15.0)
_A, _B = (6.0 - _SQ15) / 21.0, (6.0 + _SQ15) / 21.0
QPTS = np.array([[1.0 / 3.0, 1.0 / 3.0],
                 [_A, _A], [1.0 - 2.0 * _A, _A], [_A, 1.0 - 2.0 * _A],
                 [_B, _B], [1.0 - 2.0 * _B, _B], [_B, 1.0 - 2.0 * _B]])
QWTS = np.array([9.0 / 80.0] + [(155.0 - _SQ15) / 2400.0] * 3 + [(155.0 + _SQ15) / 2400.0] * 3)
EDGE_NODES = ((0, 3, 1), (1, 4, 2), (2, 5, 0))
MID_EDGES = ((3, 0, 1), (4, 1, 2), (5, 2, 0))   # (midpoint node, its edge's end vertices)


def p2_basis(s, t):
    """P2 values (..., 6) and reference gradients (..., 6, 2) at (s, t)."""
    s = np.asarray(s, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    l = [1.0 - s - t, s, t]
    dl = [np.array([-1.0, -1.0]), np.array([1.0, 0.0]), np.array([0.0, 1.0])]
    N = np.stack([l[0] * (2 * l[0] - 1), l[1] * (2 * l[1] - 1), l[2] * (2 * l[2] - 1),
                  4 * l[0] * l[1], 4 * l[1] * l[2], 4 * l[2] * l[0]], axis=-1)
    dN = np.stack([(4 * l[i] - 1)[..., None] * dl[i] for i in range(3)] +
                  [4 * (l[j][..., None] * dl[i] + l[i][..., None] * dl[j]) for i, j in ((0, 1), (1, 2), (2, 0))],
                  axis=-2)
    return N, dN


def p1_basis(s, t):
    s = np.asarray(s, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    return np.stack([1.0 - s - t, s, t], axis=-1)


N_Q, DN_Q = p2_basis(QPTS[:, 0], QPTS[:, 1])       # (7, 6), (7, 6, 2)
M_Q = p1_basis(QPTS[:, 0], QPTS[:, 1])             # (7, 3)
DM = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])   # P1 reference gradients (3, 2)


def affine(xv):
    """Affine map of each triangle from its vertices xv (E, 3, 2): J (E, 2, 2)
    with J_ij = d x_i / d s_j, its inverse and determinant."""
    J = np.stack([xv[:, 1] - xv[:, 0], xv[:, 2] - xv[:, 0]], axis=-1)
    det = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
    inv = np.empty_like(J)
    inv[:, 0, 0] = J[:, 1, 1] / det
    inv[:, 1, 1] = J[:, 0, 0] / det
    inv[:, 0, 1] = -J[:, 0, 1] / det
    inv[:, 1, 0] = -J[:, 1, 0] / det
    return J, inv, det


def element_areas(Xv):
    return 0.5 * affine(Xv)[2]


def volume_residual(Xv, xv, ue, pv, hu, hxv, c0, rho, mu, lam_s, mu_s, src=None, t=0.0):
    """Element contributions of Eq. weak_system on P2-P1 triangles with a P1
    position.  Xv, xv, hxv: (E, 3, 2) vertex arrays; ue, hu: (E, 6, 2); pv:
    (E, 3).  Returns Ru (E, 6, 2), Rp (E, 3), Rx (E, 3, 2) (pseudo-solid rows
    at the vertices).  `src` (manufactured solutions) supplies f_u, g_p at the
    current physical quadrature points and f_x at the reference ones."""
    E = Xv.shape[0]
    dt_ = np.result_type(xv, ue, pv, hu, hxv)
    Ru = np.zeros((E, 6, 2), dtype=dt_)
    Rp = np.zeros((E, 3), dtype=dt_)
    Rx = np.zeros((E, 3, 2), dtype=dt_)
    udot_n = c0 * ue + hu
    w_v = c0 * xv + hxv
    _, Jinv, det = affine(xv)
    _, Jinv0, det0 = affine(Xv)
    g1_0 = np.matmul(DM[None], Jinv0)                      # grad_X of the P1 functions (E, 3, 2)
    Fd = np.matmul(np.swapaxes(xv - Xv, 1, 2), g1_0)       # d(x - X)_i / dX_j, constant per element
    eps = 0.5 * (Fd + np.swapaxes(Fd, 1, 2))
    tr = eps[:, 0, 0] + eps[:, 1, 1]
    for q in range(len(QWTS)):
        N, M, wq = N_Q[q], M_Q[q], QWTS[q]
        g = np.matmul(DN_Q[q][None], Jinv)                 # (E, 6, 2)
        u = np.matmul(N, ue)
        udot = np.matmul(N, udot_n)
        w = np.matmul(M, w_v)
        L = np.matmul(np.swapaxes(ue, 1, 2), g)
        p = np.matmul(pv, M)
        conv = np.matmul(L, (u - w)[:, :, None])[:, :, 0]
        sigma = (mu * (L + np.swapaxes(L, 1, 2))).astype(dt_)
        sigma[:, 0, 0] -= p
        sigma[:, 1, 1] -= p
        inertia = rho * (udot + conv)
        Ru += wq * det[:, None, None] * (N[None, :, None] * inertia[:, None, :]
                                         + np.matmul(g, np.swapaxes(sigma, 1, 2)))
        divu = L[:, 0, 0] + L[:, 1, 1]
        Rp += wq * det[:, None] * (-M[None, :] * divu[:, None])
        Rx += wq * det0[:, None, None] * (lam_s[:, None, None] * g1_0 * tr[:, None, None]
                                          + 2.0 * mu_s[:, None, None] * np.matmul(g1_0, np.swapaxes(eps, 1, 2)))
        if src is not None:
            # Eulerian sources at the discrete physical point (see mms.volume_at)
            Xq = np.matmul(M, Xv)
            fu, gp, fx = src.volume_at(np.matmul(M, xv), Xq, t)
            Ru -= wq * det[:, None, None] * N[None, :, None] * fu[:, None, :]
            Rp += wq * det[:, None] * M[None, :] * gp[:, None]
            Rx -= wq * det0[:, None, None] * M[None, :, None] * fx[:, None, :]
    return Ru, Rp, Rx
