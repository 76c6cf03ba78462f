"""Helpers shared by the GPU parity tests: matching the oracle's unknowns to
the library's, and seeded states."""
import numpy as np

from paper_2609_31477_b300 import inputs as I, viv


def oracle_labels(c):
    lab = np.empty(c.ndof, dtype=object)
    D = c.dof_u.shape[1]
    for a in range(c.n):
        for i, f in enumerate(("ux", "uy", "uz")[:D]):
            if c.dof_u[a, i] >= 0:
                lab[c.dof_u[a, i]] = (a, f)
        if c.dof_p[a] >= 0:
            lab[c.dof_p[a]] = (a, "p")
        for i, f in enumerate(("xx", "xy", "xz")[:D]):
            if c.dof_x[a, i] >= 0:
                lab[c.dof_x[a, i]] = (a, f)
        for i, f in enumerate(("lx", "ly", "lz")[:D]):
            if c.dof_l[a, i] >= 0:
                lab[c.dof_l[a, i]] = (a, f)
    if c.has_body:
        lab[c.dof_d[0]] = (c.n, "dx")
        lab[c.dof_d[1]] = (c.n, "dy")
    return lab


def perm_oracle_to_lib(oc, M):
    node, field = M.dof_labels()
    lib = {(int(a), viv.FIELD[int(f)]): i for i, (a, f) in enumerate(zip(node, field))}
    lab = oracle_labels(oc)
    return np.array([lib[lab[i]] for i in range(oc.ndof)])


def seeded_state(oc, seed, amp=1.0):
    """A smooth, admissible, non-trivial state on the oracle case: velocity
    perturbed, pressure and multiplier random, mesh deformed, delta set;
    prescribed components untouched."""
    rng = np.random.default_rng(seed)
    X = oc.X
    U = oc.gather()
    U += amp * 0.05 * rng.standard_normal(U.shape)
    oc.scatter(U)
    bump = 0.02 * amp * np.sin(0.3 * X[:, 0]) * np.cos(0.25 * X[:, 1])
    for i in range(2):
        free = oc.dof_x[:, i] >= 0
        oc.x[free, i] = X[free, i] + bump[free] * (1 + i)
    if oc.has_body:
        oc.delta = amp * np.array([0.03, -0.02])
        oc.x[oc.cyl] = X[oc.cyl] + oc.delta


def copy_state(oc):
    return dict(u=oc.u.copy(), p=oc.p.copy(), x=oc.x.copy(), lam=oc.lam.copy(), delta=oc.delta.copy())


def push_state(case, st, t=0.0):
    case.set_state(st["u"], st["p"], st["x"], st["lam"], st["delta"], t)


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
