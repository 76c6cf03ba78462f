"""Parity at the sizes where the kernels change path, and at the headline
38,800-quad case.

8,556-quad cylinder (O-grid refinement 28, 145,850 unknowns, Re 200, U* 10,
dt 0.02): its largest front has 1,763 rows, so
  * threshold pivoting on the mixed path factors the big fronts' panels with
    the 8-CTA cluster kernel (panel_smem_kernel<float, 8, 256>: rows split over
    the cluster's shared memory, pivot maxima exchanged through DSMEM) and
    applies their interchanges with laswp_kernel (one CTA holds 1,600 FP32
    panel rows);
  * threshold pivoting on the FP64 path does the same above 800 rows
    (panel_smem_kernel<double, 8, 256>);
  * front assembly runs with 512 threads per item at the levels whose fronts
    reach order 1,024;
  * the windowed bench configuration (FP32 volume Jacobians, extrapolated
    Newton start) runs its 128-column outer blocks on the tensor cores.
Each is compared after three steps with the oracle's own run of the case
(tests/golden/cylinder_m28_re200.npz, written by make_cylinder_golden.py from
oracle/ alone): fields to 1e-9 relative L2, delta to 1e-8.

38,800-quad case (the benchmark's): the oracle's factorisation takes too
long, so two pins hold there - the oracle's residual evaluated at the GPU's
converged state (with the GPU's own BDF history) sits at the Newton
tolerance, and the mixed path agrees with the plain FP64 path to 1e-9."""
import os

import numpy as np
import pytest

from paper_2609_31477_b300 import inputs as I
from oracle.solver import viv_oracle_case

from gpu_common import rel_l2

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cylinder_m28_re200.npz")


@pytest.fixture(scope="module")
def viv():
    import torch
    assert torch.cuda.is_available()
    from paper_2609_31477_b300 import build, viv as V
    build.build()
    V.load()
    return V


@pytest.fixture(scope="module")
def m28(viv):
    g = dict(np.load(GOLDEN))
    mesh = I.viv_cylinder_mesh(int(g["m"]))
    M = viv.Mesh(mesh)
    return g, mesh, M


def _vertex_mask(mesh):
    v = np.zeros(len(mesh["X"]), bool)
    v[np.asarray(mesh["conn"])[:, [0, 2, 6, 8]].ravel()] = True
    return v


@pytest.mark.parametrize("precision,pivoting,jac32,pred", [("mixed", "window", 1, 1), ("mixed", "threshold", 0, 0),
                                                           ("fp64", "threshold", 0, 0)])
def test_path_changing_sizes_match_oracle(viv, m28, precision, pivoting, jac32, pred):
    g, mesh, M = m28
    fr = M.fronts()
    assert fr["m"].max() > 1600                       # beyond one CTA's FP32 panel rows: cluster panels
    lv_max = np.zeros(fr["level"].max() + 1, int)
    np.maximum.at(lv_max, fr["level"], fr["m"])
    assert (lv_max >= 1024).any()                     # 512-thread assembly at those levels
    prec = viv.VIV_FP64 if precision == "fp64" else viv.VIV_MIXED
    piv = viv.VIV_PIVOT_THRESHOLD if pivoting == "threshold" else viv.VIV_PIVOT_WINDOW
    u0 = I.viv_initial_velocity(mesh, 1.0, 1e-3, int(g["seed"]))
    case = viv.viv_case(M, float(g["Re"]), float(g["Ustar"]), float(g["dt"]), u0, precision=prec, pivoting=piv,
                        jacobian_fp32=jac32, predictor=pred)
    misses = perturbed = 0
    for s in range(int(g["steps"])):
        info = case.step()
        assert info["res_norm"] <= 1e-10
        assert np.abs(np.array(info["delta"]) - g["delta"][s]).max() <= 1e-8
        misses += info["threshold_misses"]
        perturbed += info["perturbed_pivots"]
    st = case.get_state()
    case.close()
    X = np.asarray(mesh["X"])
    cyl = (np.asarray(mesh["tags"]) & I.CYL) != 0
    errs = dict(u=rel_l2(st["u"], g["u"]), p=rel_l2(st["p"][_vertex_mask(mesh)], g["p_vertex"]),
                x=rel_l2(st["x"], g["x_minus_X"] + X), lam=rel_l2(st["lam"][cyl], g["lam_gamma"]),
                displacement=rel_l2(st["x"] - X, g["x_minus_X"]),
                delta=np.abs(st["delta"] - g["delta"][-1]).max())
    print(precision, pivoting, errs, "threshold misses", misses, "perturbed", perturbed)
    for k in ("u", "p", "x", "lam"):
        assert errs[k] <= 1e-9, errs
    assert errs["delta"] <= 1e-8, errs
    assert errs["displacement"] <= 1e-7, errs        # the mesh motion itself, not only x = X + motion
    assert perturbed == 0


def test_headline_case_oracle_residual_and_fp64_agreement(viv):
    """38,800 quads, Re 200, U* 10, dt 0.02, the benchmark's configuration."""
    mesh = I.viv_cylinder_mesh(60)
    u0 = I.viv_initial_velocity(mesh, 1.0, 1e-3, 1)
    M = viv.Mesh(mesh)
    mixed = viv.viv_case(M, 200.0, 10.0, 0.02, u0, precision=viv.VIV_MIXED, pivoting=viv.VIV_PIVOT_WINDOW,
                         jacobian_fp32=1, predictor=1)
    states = []
    for s in range(3):
        info = mixed.step()
        assert info["res_norm"] <= 1e-10
        states.append(mixed.get_state())
    mixed.close()
    # (ii) the oracle's residual at the GPU state, with the GPU's own history
    oc = viv_oracle_case(mesh, 200.0, 10.0, 0.02, u0)
    oc.u_n, oc.x_n = states[1]["u"], states[1]["x"]
    oc.hist = (states[0]["u"], states[0]["x"])
    for k in ("u", "p", "x", "lam", "delta"):
        setattr(oc, k, states[2][k].copy())
    c0, hu, hx = oc.bdf_coefficients()
    R = oc.residual(c0, hu, hx, states[2]["t"])
    print("oracle residual at the GPU state:", np.linalg.norm(R))
    assert np.linalg.norm(R) <= 1e-10
    # (iii) mixed path vs plain FP64 path (threshold pivoting, FP64 Jacobians, Newton from U^n)
    f64 = viv.viv_case(M, 200.0, 10.0, 0.02, u0, precision=viv.VIV_FP64)
    for s in range(3):
        f64.step()
    s64 = f64.get_state()
    f64.close()
    verts = _vertex_mask(mesh)
    errs = dict(u=rel_l2(states[2]["u"], s64["u"]), p=rel_l2(states[2]["p"][verts], s64["p"][verts]),
                x=rel_l2(states[2]["x"], s64["x"]), delta=np.abs(states[2]["delta"] - s64["delta"]).max())
    print("mixed vs FP64:", errs)
    assert max(errs["u"], errs["p"], errs["x"]) <= 1e-9 and errs["delta"] <= 1e-8, errs
    M.close()
