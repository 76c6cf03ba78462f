"""Seeded synthetic inputs shared by the CUDA path, the tests and the bench.

This module holds geometry and random numbers only: meshes (node coordinates,
Q2 connectivity, boundary tags, the cylinder boundary faces) and the seeded
initial-velocity perturbation.  It contains none of the solver's arithmetic
(no shape functions, no quadrature, no residuals), so both the oracle and the
CUDA path may consume what it produces.

Geometry follows the two-dimensional cylinder configuration of the paper's
VIV study (Section 6: a cylinder of diameter D centred at X_c in a rectangular
channel, uniform inflow, slip walls, natural outflow; Eq. (flowBC), Eq. (psBC)),
meshed here with quadratic quadrilaterals: an O-grid around the cylinder that
is blended onto a square, surrounded by graded Cartesian blocks.

Node tags are bit flags that say which nodal degrees of freedom are held by a
Dirichlet condition; the value held is whatever the initial state carries.
"""
from __future__ import annotations

import math
import numpy as np

# --- boundary tag bits (per node) ---------------------------------------------
U_FIX_X = 1    # velocity x-component prescribed
U_FIX_Y = 2    # velocity y-component prescribed
X_FIX_X = 4    # mesh position x-component prescribed
X_FIX_Y = 8    # mesh position y-component prescribed
CYL = 16       # node on the rigid cylinder boundary Gamma (multiplier lives here)
OUTLET = 32    # informational: natural outflow boundary
P_FIX = 64     # pressure prescribed at this (vertex) node: removes the constant
U_FIX_Z = 128  # velocity z-component prescribed (3-D meshes)
X_FIX_Z = 256  # mesh position z-component prescribed (3-D meshes)
               # pressure mode of all-Dirichlet problems (Q = L^2/R, Section 3.1)

INLET_TAG = U_FIX_X | U_FIX_Y | X_FIX_X | X_FIX_Y   # u = u_in, x = X
OUTLET_TAG = OUTLET | X_FIX_X | X_FIX_Y              # stress free, x = X
WALL_TAG = U_FIX_Y | X_FIX_Y                         # u.n = 0, x.n = X.n
ALL_DIRICHLET_TAG = U_FIX_X | U_FIX_Y | X_FIX_X | X_FIX_Y

# local edge ids of a 9-node quad (lexicographic node index 3*b + a, a along xi)
EDGE_NODES = ((0, 3, 6), (2, 5, 8), (0, 1, 2), (6, 7, 8))


class _NodeTable:
    """Merges coincident nodes produced by different mesh blocks."""

    def __init__(self, tol=1e-9):
        self.tol = tol
        self.index = {}
        self.coords = []

    def get(self, x, y):
        key = (int(round(x / self.tol)), int(round(y / self.tol)))
        idx = self.index.get(key)
        if idx is None:
            idx = len(self.coords)
            self.index[key] = idx
            self.coords.append((x, y))
        return idx


def _graded(h0, length, n):
    """n cell widths summing to `length`, the first equal to h0 and growing
    geometrically; uniform when h0*n already covers the length."""
    if h0 * n >= length:
        return np.full(n, length / n)
    lo, hi = 1.0, 2.0
    while h0 * (hi ** n - 1) / (hi - 1) < length:
        hi *= 2
    for _ in range(200):
        q = 0.5 * (lo + hi)
        s = h0 * (q ** n - 1) / (q - 1)
        if s < length:
            lo = q
        else:
            hi = q
    q = 0.5 * (lo + hi)
    w = h0 * q ** np.arange(n)
    return w * (length / w.sum())


def _q2_line(vertices):
    """Vertex coordinates -> Q2 node coordinates (vertices and midpoints)."""
    v = np.asarray(vertices, dtype=np.float64)
    out = np.empty(2 * len(v) - 1)
    out[0::2] = v
    out[1::2] = 0.5 * (v[:-1] + v[1:])
    return out


def viv_cylinder_mesh(m=12, D=1.0, Xc=(0.0, 0.0), half=3.0,
                      box=(-10.0, 20.0, -10.0, 10.0), q_radial=1.15):
    """Q2 quadrilateral mesh of the channel [x0,x1]x[y0,y1] around a cylinder.

    m is the number of cells along one side of the square [-half,half]^2 that
    holds the O-grid; the O-grid has 4m cells around and m cells radially, and
    the Cartesian surround has 8m/12 (left, top, bottom) and 20m/12 (right)
    graded cells.  m = 12 gives 1,552 quads; m = 60 gives 38,800.
    Returns a dict with X (n,2), conn (E,9), tags (n,), gamma_faces (F,2)
    [element, local edge], Xc, D.
    """
    x0, x1, y0, y1 = box
    cx, cy = Xc
    r_in = 0.5 * D
    nodes = _NodeTable()
    conn = []
    gamma_faces = []

    # ---- O-grid: xi runs outward (radial), eta runs counter-clockwise -------
    n_around = 8 * m              # Q2 nodes around
    q = q_radial ** (12.0 / m)
    sv = (q ** np.arange(m + 1) - 1.0) / (q ** m - 1.0)
    s_nodes = _q2_line(sv)        # 2m+1 radial node parameters
    perim = 8.0 * half

    def square_point(t):
        t = t % perim
        h = half
        if t < h:
            return h, t
        t -= h
        if t < 2 * h:
            return h - t, h
        t -= 2 * h
        if t < 2 * h:
            return -h, h - t
        t -= 2 * h
        if t < 2 * h:
            return -h + t, -h
        t -= 2 * h
        return h, -h + t

    # the square's corners (ring index m + shift) must be quad corners (even
    # ring index) so that the O-grid cells meet the Cartesian cells edge to
    # edge; odd m starts the ring one node later
    shift = m % 2
    ring = np.empty((n_around, 2 * m + 1), dtype=np.int64)
    for k in range(n_around):
        th = 2.0 * math.pi * (k + shift) / n_around
        c = (cx + r_in * math.cos(th), cy + r_in * math.sin(th))
        sq = square_point(perim * (k + shift) / n_around)
        s_pt = (cx + sq[0], cy + sq[1])
        for r, s in enumerate(s_nodes):
            if r == 0:
                px, py = c
            elif r == 2 * m:
                px, py = s_pt
            else:
                px = (1 - s) * c[0] + s * s_pt[0]
                py = (1 - s) * c[1] + s * s_pt[1]
            ring[k, r] = nodes.get(px, py)
    for i in range(4 * m):
        for j in range(m):
            el = []
            for b in range(3):
                k = (2 * i + b) % n_around
                for a in range(3):
                    el.append(ring[k, 2 * j + a])
            if j == 0:
                gamma_faces.append((len(conn), 0))
            conn.append(el)

    # ---- Cartesian surround --------------------------------------------------
    nl = max(1, round(8 * m / 12))
    nr = max(1, round(20 * m / 12))
    nb = max(1, round(8 * m / 12))
    nt = max(1, round(8 * m / 12))
    h0 = 2.0 * half / m
    wl = _graded(h0, (cx - half) - x0, nl)[::-1]
    wr = _graded(h0, x1 - (cx + half), nr)
    wb = _graded(h0, (cy - half) - y0, nb)[::-1]
    wt = _graded(h0, y1 - (cy + half), nt)
    xv = np.concatenate([[x0], x0 + np.cumsum(wl)[:-1], np.linspace(cx - half, cx + half, m + 1),
                         (cx + half) + np.cumsum(wr)])
    yv = np.concatenate([[y0], y0 + np.cumsum(wb)[:-1], np.linspace(cy - half, cy + half, m + 1),
                         (cy + half) + np.cumsum(wt)])
    xv[-1], yv[-1] = x1, y1
    xq, yq = _q2_line(xv), _q2_line(yv)
    for cj in range(len(yv) - 1):
        for ci in range(len(xv) - 1):
            if nl <= ci < nl + m and nb <= cj < nb + m:
                continue
            el = []
            for b in range(3):
                for a in range(3):
                    el.append(nodes.get(xq[2 * ci + a], yq[2 * cj + b]))
            conn.append(el)

    X = np.array(nodes.coords, dtype=np.float64)
    tags = np.zeros(len(X), dtype=np.int32)
    tol = 1e-9
    tags[np.abs(X[:, 1] - y0) < tol] |= WALL_TAG
    tags[np.abs(X[:, 1] - y1) < tol] |= WALL_TAG
    tags[np.abs(X[:, 0] - x1) < tol] |= OUTLET_TAG
    tags[np.abs(X[:, 0] - x0) < tol] |= INLET_TAG
    rr = np.hypot(X[:, 0] - cx, X[:, 1] - cy)
    tags[np.abs(rr - r_in) < 1e-9] |= CYL
    return dict(X=X, conn=np.array(conn, dtype=np.int64), tags=tags,
                gamma_faces=np.array(gamma_faces, dtype=np.int64).reshape(-1, 2),
                Xc=np.array([cx, cy], dtype=np.float64), D=float(D), name=f"viv_ogrid_m{m}")


def square_mesh(n, hole=None, lo=0.0, hi=1.0):
    """Uniform n x n Q2 mesh of [lo,hi]^2 with every outer node fully
    Dirichlet (u and x).  `hole=(a,b)` removes the cells inside [a,b]^2 (a and
    b must fall on cell boundaries) and tags its boundary as the rigid body
    Gamma."""
    h = (hi - lo) / n
    nodes = _NodeTable()
    xq = _q2_line(np.linspace(lo, hi, n + 1))
    conn, gamma_faces = [], []
    inside = None
    if hole is not None:
        ia, ib = round((hole[0] - lo) / h), round((hole[1] - lo) / h)
        inside = (ia, ib)
    for cj in range(n):
        for ci in range(n):
            if inside and inside[0] <= ci < inside[1] and inside[0] <= cj < inside[1]:
                continue
            el = []
            for b in range(3):
                for a in range(3):
                    el.append(nodes.get(xq[2 * ci + a], xq[2 * cj + b]))
            if inside:
                ia, ib = inside
                if ci == ia - 1 and ia <= cj < ib:
                    gamma_faces.append((len(conn), 1))
                if ci == ib and ia <= cj < ib:
                    gamma_faces.append((len(conn), 0))
                if cj == ia - 1 and ia <= ci < ib:
                    gamma_faces.append((len(conn), 3))
                if cj == ib and ia <= ci < ib:
                    gamma_faces.append((len(conn), 2))
            conn.append(el)
    X = np.array(nodes.coords, dtype=np.float64)
    tags = np.zeros(len(X), dtype=np.int32)
    tol = 1e-9
    outer = ((np.abs(X[:, 0] - lo) < tol) | (np.abs(X[:, 0] - hi) < tol)
             | (np.abs(X[:, 1] - lo) < tol) | (np.abs(X[:, 1] - hi) < tol))
    tags[outer] |= ALL_DIRICHLET_TAG
    if hole is not None:
        a, b = hole
        on = (((np.abs(X[:, 0] - a) < tol) | (np.abs(X[:, 0] - b) < tol)) & (X[:, 1] > a - tol) & (X[:, 1] < b + tol)) | \
             (((np.abs(X[:, 1] - a) < tol) | (np.abs(X[:, 1] - b) < tol)) & (X[:, 0] > a - tol) & (X[:, 0] < b + tol))
        tags[on] |= CYL
        c = 0.5 * (a + b)
    else:
        c = 0.5 * (lo + hi)
    return dict(X=X, conn=np.array(conn, dtype=np.int64), tags=tags,
                gamma_faces=np.array(gamma_faces, dtype=np.int64).reshape(-1, 2),
                Xc=np.array([c, c]), D=(hole[1] - hole[0]) if hole else 0.0,
                name=f"square_n{n}" + ("_hole" if hole else ""))


def hole_square_mesh(n, R0=0.15, center=(0.5, 0.5), lo=0.0, hi=1.0):
    """Q2 O-grid of the square [lo,hi]^2 around a circular hole of radius R0:
    4n cells around, n cells radially, blended linearly from the circle (nodes
    on the circle, midpoints included) to the square boundary.  Outer nodes are
    fully Dirichlet (u and x), hole nodes are the rigid body Gamma.  This is
    the geometry of the coupled manufactured solution of Section 5.2 (a rigid
    cylinder of radius R0 inside the unit square)."""
    cx, cy = center
    half = 0.5 * (hi - lo)
    nodes = _NodeTable()
    conn, gamma_faces = [], []
    n_around = 8 * n
    s_nodes = _q2_line(np.linspace(0.0, 1.0, n + 1))
    perim = 8.0 * half

    def square_point(t):
        t = t % perim
        h = half
        if t < h:
            return h, t
        t -= h
        if t < 2 * h:
            return h - t, h
        t -= 2 * h
        if t < 2 * h:
            return -h, h - t
        t -= 2 * h
        if t < 2 * h:
            return -h + t, -h
        t -= 2 * h
        return h, -h + t

    ring = np.empty((n_around, 2 * n + 1), dtype=np.int64)
    for k in range(n_around):
        th = 2.0 * math.pi * k / n_around
        c = (cx + R0 * math.cos(th), cy + R0 * math.sin(th))
        sq = square_point(perim * k / n_around)
        s_pt = (cx + sq[0], cy + sq[1])
        for r, sv in enumerate(s_nodes):
            if r == 0:
                px, py = c
            elif r == 2 * n:
                px, py = s_pt
            else:
                px = (1 - sv) * c[0] + sv * s_pt[0]
                py = (1 - sv) * c[1] + sv * s_pt[1]
            ring[k, r] = nodes.get(px, py)
    for i in range(4 * n):
        for j in range(n):
            el = []
            for b in range(3):
                k = (2 * i + b) % n_around
                for a in range(3):
                    el.append(ring[k, 2 * j + a])
            if j == 0:
                gamma_faces.append((len(conn), 0))
            conn.append(el)
    X = np.array(nodes.coords, dtype=np.float64)
    tags = np.zeros(len(X), dtype=np.int32)
    tol = 1e-9
    outer = ((np.abs(X[:, 0] - lo) < tol) | (np.abs(X[:, 0] - hi) < tol)
             | (np.abs(X[:, 1] - lo) < tol) | (np.abs(X[:, 1] - hi) < tol))
    tags[outer] |= ALL_DIRICHLET_TAG
    tags[np.abs(np.hypot(X[:, 0] - cx, X[:, 1] - cy) - R0) < 1e-9] |= CYL
    return dict(X=X, conn=np.array(conn, dtype=np.int64), tags=tags,
                gamma_faces=np.array(gamma_faces, dtype=np.int64).reshape(-1, 2),
                Xc=np.array([cx, cy], dtype=np.float64), D=2.0 * R0, name=f"hole_square_n{n}")


# --- simplicial variant: 6-node triangles with straight edges ----------------------
# local triangle node order: vertices 0, 1, 2, then the midpoints of edges
# 0-1 (3), 1-2 (4), 2-0 (5); local edge e runs (v_e, midpoint, v_{e+1})
def triangulate_q2(mesh):
    """Split every Q2 quad of a 2-D mesh along a diagonal into two 6-node
    triangles - along 0-8, (q0, q2, q8 | q1, q5, q4) and (q0, q8, q6 | q4, q7,
    q3), or, where that would leave a triangle with all three vertices on the
    mesh boundary (a mesh corner), along 2-6, (q0, q2, q6 | q1, q4, q3) and
    (q2, q8, q6 | q5, q7, q4): Taylor-Hood P2-P1 leaves the pressure of such
    a triangle uncontrolled.  Every midside node moves to the midpoint of its
    edge's end nodes, so that the edges are straight (the geometry of a P1
    position field; the cylinder becomes a polygon).  Tags are kept; Gamma
    edges map to the triangle edges on the same quad edge.  Returns X, conn
    (2E, 6), tags, gamma_faces (F, 2) [element, local edge 0..2], elem =
    "tri6"."""
    X = np.array(mesh["X"], dtype=np.float64)
    q = np.asarray(mesh["conn"], dtype=np.int64)
    E = len(q)
    # boundary vertices: the end nodes of quad edges that belong to one quad only
    edges = {}
    for a, b in ((0, 2), (2, 8), (8, 6), (6, 0)):
        for e in range(E):
            key = (min(q[e, a], q[e, b]), max(q[e, a], q[e, b]))
            edges[key] = edges.get(key, 0) + 1
    on_bnd = np.zeros(len(X), bool)
    for (a, b), cnt in edges.items():
        if cnt == 1:
            on_bnd[a] = on_bnd[b] = True
    bad08 = (on_bnd[q[:, 0]] & on_bnd[q[:, 2]] & on_bnd[q[:, 8]]) | (on_bnd[q[:, 0]] & on_bnd[q[:, 8]] & on_bnd[q[:, 6]])
    bad26 = (on_bnd[q[:, 0]] & on_bnd[q[:, 2]] & on_bnd[q[:, 6]]) | (on_bnd[q[:, 2]] & on_bnd[q[:, 8]] & on_bnd[q[:, 6]])
    flip = bad08 & ~bad26
    conn = np.empty((2 * E, 6), dtype=np.int64)
    conn[0::2] = np.where(flip[:, None], q[:, [0, 2, 6, 1, 4, 3]], q[:, [0, 2, 8, 1, 5, 4]])
    conn[1::2] = np.where(flip[:, None], q[:, [2, 8, 6, 5, 7, 4]], q[:, [0, 8, 6, 4, 7, 3]])
    for c in (conn[0::2], conn[1::2]):
        for mid, (a, b) in ((3, (0, 1)), (4, (1, 2)), (5, (2, 0))):
            X[c[:, mid]] = 0.5 * (X[c[:, a]] + X[c[:, b]])
    # quad edge -> (triangle offset, local edge); diagonal 0-8: xi=0 -> T2 edge 2,
    # xi=1 -> T1 edge 1, eta=0 -> T1 edge 0, eta=1 -> T2 edge 1; diagonal 2-6:
    # xi=0 -> T1 edge 2, xi=1 -> T2 edge 0, eta=0 -> T1 edge 0, eta=1 -> T2 edge 1
    emap = {0: (1, 2), 1: (0, 1), 2: (0, 0), 3: (1, 1)}
    emap_flip = {0: (0, 2), 1: (1, 0), 2: (0, 0), 3: (1, 1)}
    gf = [(2 * e + (emap_flip if flip[e] else emap)[ed][0], (emap_flip if flip[e] else emap)[ed][1])
          for e, ed in np.asarray(mesh["gamma_faces"]).reshape(-1, 2)]
    out = dict(mesh)
    out.update(X=X, conn=conn, gamma_faces=np.array(gf, dtype=np.int64).reshape(-1, 2), elem="tri6",
               name=mesh.get("name", "mesh") + "_tri")
    return out


# --- 3-D: periodic extrusion of a 2-D Q2 mesh into 27-node hexahedra -------------
# local hex node index 9 c + 3 b + a (a along xi, b along eta, c along zeta);
# local faces 0: xi=0, 1: xi=1, 2: eta=0, 3: eta=1, 4: zeta=0, 5: zeta=1
def extrude_periodic(mesh2d, layers, span):
    """Extrude a 2-D Q2 mesh over z in [0, span) into `layers` layers of Q2
    hexahedra, periodic in z: node plane 2*layers is node plane 0, and the
    nodes of the last layer's top face carry a wrap bit (their coordinates are
    the stored ones + span e_z).  Periodicity is on the displacement x - X
    (the position itself jumps by span e_z across the seam).

    Tags: a 2-D node whose velocity (position) is fully prescribed has its z
    component prescribed too; cylinder nodes keep their z position (the rigid
    body moves in x and y only); a prescribed pressure stays on plane 0 only.
    Gamma faces become the zeta-extruded faces of the 2-D Gamma edges
    (2-D edge 0..3 -> hex face 0..3).  Returns X (n,3), conn (E,27), tags,
    gamma_faces (F,2), wrap (E,) node bit masks, span, Xc, D."""
    assert layers >= 2, "a periodic extrusion needs at least two layers"
    X2 = np.asarray(mesh2d["X"], dtype=np.float64)
    c2 = np.asarray(mesh2d["conn"], dtype=np.int64)
    t2 = np.asarray(mesh2d["tags"], dtype=np.int64)
    n2, E2 = len(X2), len(c2)
    planes = 2 * layers
    dz = span / planes
    X = np.zeros((planes * n2, 3))
    for k in range(planes):
        X[k * n2:(k + 1) * n2, :2] = X2
        X[k * n2:(k + 1) * n2, 2] = k * dz
    tags = np.zeros(planes * n2, dtype=np.int32)
    t3 = t2.copy()
    full_u = (t2 & (U_FIX_X | U_FIX_Y)) == (U_FIX_X | U_FIX_Y)
    full_x = (t2 & (X_FIX_X | X_FIX_Y)) == (X_FIX_X | X_FIX_Y)
    t3[full_u] |= U_FIX_Z
    t3[full_x | ((t2 & CYL) != 0)] |= X_FIX_Z
    for k in range(planes):
        tk = t3 if k == 0 else (t3 & ~P_FIX)
        tags[k * n2:(k + 1) * n2] = tk
    conn = np.zeros((layers * E2, 27), dtype=np.int64)
    wrap = np.zeros(layers * E2, dtype=np.int64)
    for l in range(layers):
        for c in range(3):
            plane = 2 * l + c
            wrapped = plane >= planes
            for b in range(3):
                for a in range(3):
                    conn[l * E2:(l + 1) * E2, 9 * c + 3 * b + a] = (plane % planes) * n2 + c2[:, 3 * b + a]
                    if wrapped:
                        wrap[l * E2:(l + 1) * E2] |= 1 << (9 * c + 3 * b + a)
    gf2 = np.asarray(mesh2d["gamma_faces"], dtype=np.int64).reshape(-1, 2)
    gf = np.concatenate([np.stack([gf2[:, 0] + l * E2, gf2[:, 1]], 1) for l in range(layers)]) \
        if len(gf2) else np.zeros((0, 2), dtype=np.int64)
    return dict(X=X, conn=conn, tags=tags, gamma_faces=gf.reshape(-1, 2), wrap=wrap, span=float(span),
                Xc=np.asarray(mesh2d.get("Xc", np.zeros(2)), dtype=np.float64), D=float(mesh2d.get("D", 0.0)),
                name=f"{mesh2d.get('name', 'mesh')}_z{layers}")


def viv_cylinder_mesh3d(m=7, layers=24, span=2.0 * math.pi, **kw):
    """The cylinder O-grid of `viv_cylinder_mesh(m)` extruded over a periodic
    span (m = 7: 555 quads per section, 24 layers: 13,320 hexahedra)."""
    return extrude_periodic(viv_cylinder_mesh(m, **kw), layers, span)


# --- seeded normal samples: splitmix64 + Box-Muller ----------------------------
_M64 = (1 << 64) - 1


def _splitmix64(state):
    state = (state + 0x9E3779B97F4A7C15) & _M64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return state, z ^ (z >> 31)


def seeded_normals(seed, n):
    """n standard normal samples from splitmix64 (Vigna) + Box-Muller."""
    out = np.empty(n, dtype=np.float64)
    s = seed & _M64
    i = 0
    while i < n:
        s, a = _splitmix64(s)
        s, b = _splitmix64(s)
        u1 = ((a >> 11) + 1) * (1.0 / 9007199254740993.0)   # (0,1]
        u2 = (b >> 11) * (1.0 / 9007199254740992.0)         # [0,1)
        r = math.sqrt(-2.0 * math.log(u1))
        out[i] = r * math.cos(2.0 * math.pi * u2)
        if i + 1 < n:
            out[i + 1] = r * math.sin(2.0 * math.pi * u2)
        i += 2
    return out


def viv_initial_velocity(mesh, U_inf=1.0, sigma=1e-3, seed=1):
    """Nodal initial velocity: uniform inflow (U_inf, 0[, 0]) plus seeded
    N(0, sigma^2) noise on every component that no Dirichlet tag holds.
    Prescribed components carry their boundary value (inflow, or 0 normal to
    walls).  2-D or 3-D by the mesh's coordinates."""
    n, D = np.shape(mesh["X"])
    u = np.zeros((n, D))
    u[:, 0] = U_inf
    if sigma > 0:
        u += sigma * seeded_normals(seed, D * n).reshape(n, D)
    t = mesh["tags"]
    fx = (t & U_FIX_X) != 0
    fy = (t & U_FIX_Y) != 0
    u[fx, 0] = U_inf
    u[fy, 1] = 0.0
    if D == 3:
        u[(t & U_FIX_Z) != 0, 2] = 0.0
    return u


# the workloads used by the tests and the bench, by name
def viv_case(name):
    """Named VIV workloads: mesh refinement m, Reynolds number, reduced
    velocity, time step, steps."""
    table = {
        "viv_re100_m12": dict(m=12, Re=100.0, Ustar=8.0, dt=0.1, steps=10),
        "viv_re200_m60": dict(m=60, Re=200.0, Ustar=10.0, dt=0.02, steps=500),
        # 3-D: the section of viv_cylinder_mesh(m) extruded into `layers` periodic layers
        "viv3d_re300_m7_z24": dict(m=7, layers=24, span=2.0 * math.pi, Re=300.0, Ustar=8.0, dt=0.05,
                                   steps=100),
    }
    return dict(table[name])
