"""Writes the oracle's reference run of a cylinder case to tests/golden/.

The stored values come from the FP64 oracle alone (oracle/ plus the seeded
mesh and initial-velocity generators of paper_2609_31477_b300.inputs, which
hold no solver arithmetic).  The GPU parity tests compare the CUDA path with
them at a mesh size the oracle needs minutes for.

  python tests/golden/make_cylinder_golden.py            # every case below
  python tests/golden/make_cylinder_golden.py cylinder3d_m3_z4_re300

Case: O-grid refinement m = 28 (8,556 Q2-Q1 quads, 145,850 unknowns), Re 200,
U* 10, dt 0.02, uniform inflow plus seeded N(0, 1e-3^2) noise (seed 1), BDF1
then BDF2, Newton to ||NL||_2 <= 1e-10 (Eq. NR_iteration), three steps - the
cylinder workload of Section 6 at a size whose largest front (1,763 rows)
exceeds what one CTA's shared memory holds on the FP32 path.

3-D case: the same workload extruded in z with periodic ends (the spanwise
reading of Section 6's 3-D runs), Re 300, U* 8 with the span as the length
carrying the force, dt 0.05, seeded noise on all three velocity components,
two steps.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from paper_2609_31477_b300 import inputs as I  # noqa: E402
from oracle.solver import viv_oracle_case  # noqa: E402
from oracle.solver3d import viv_oracle_case3d  # noqa: E402

CASES = {"cylinder_m28_re200": dict(m=28, Re=200.0, Ustar=10.0, dt=0.02, seed=1, steps=3),
         # 3-D: the m = 3 section (97 quads) extruded into 4 periodic layers of the
         # 24-layer, 2 pi span case's thickness (388 hexahedra, 19,658 unknowns)
         "cylinder3d_m3_z4_re300": dict(m=3, layers=4, span=2.0 * np.pi * 4 / 24, Re=300.0, Ustar=8.0, dt=0.05,
                                        seed=1, steps=2)}


def make(name):
    c = CASES[name]
    if "layers" in c:
        mesh = I.viv_cylinder_mesh3d(c["m"], c["layers"], c["span"])
    else:
        mesh = I.viv_cylinder_mesh(c["m"])
    u0 = I.viv_initial_velocity(mesh, 1.0, 1e-3, c["seed"])
    if "layers" in c:
        oc = viv_oracle_case3d(mesh, c["Re"], c["Ustar"], c["dt"], u0)
    else:
        oc = viv_oracle_case(mesh, c["Re"], c["Ustar"], c["dt"], u0)
    deltas, forces, norms = [], [], []
    t0 = time.time()
    for s in range(c["steps"]):
        nr = oc.step()
        deltas.append(oc.delta.copy())
        forces.append(oc.force())
        norms.append(nr[-1])
        print(f"step {s + 1}: Newton norms {['%.2e' % v for v in nr]}  ({time.time() - t0:.0f} s)", flush=True)
    out = os.path.join(HERE, name + ".npz")
    np.savez_compressed(out, u=oc.u, p_vertex=oc.p[oc.is_vertex], x_minus_X=oc.x - oc.X,
                        lam_gamma=oc.lam[oc.cyl], delta=np.array(deltas), force=np.array(forces),
                        final_norm=np.array(norms), **{k: np.array(v) for k, v in c.items()})
    print("wrote", out)


if __name__ == "__main__":
    for name in (sys.argv[1:] or CASES):
        make(name)
