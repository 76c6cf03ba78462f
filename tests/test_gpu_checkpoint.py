"""Checkpoint / resume through the C ABI (viv_case_save, viv_case_load) and
the library's conversion of Re and U* into mu and k (vivParams)."""
import math

import numpy as np
import pytest

from paper_2609_31477_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def viv():
    import torch
    assert torch.cuda.is_available()
    from paper_2609_31477_b300 import build, viv as V
    build.build()
    V.load()
    return V


def test_library_derives_mu_and_k_from_re_and_ustar(viv):
    """mu = rho U D / Re and the stiffness whose reduced velocity
    U_r = pi U sqrt(pi rho L / k) (Section 1) equals U*: pi^3/64 for U* = 8."""
    mesh = I.viv_cylinder_mesh(4)
    M = viv.Mesh(mesh)
    case = viv.viv_case(M, 100.0, 8.0, 0.1, I.viv_initial_velocity(mesh, 1.0, 1e-3, 1))
    p = case.resolved_params()
    assert abs(p["k"] - 0.48447307) < 5e-9 and abs(p["mu"] - 0.01) < 1e-16
    assert abs(math.pi * math.sqrt(math.pi / p["k"]) - 8.0) < 1e-12
    case.close()
    # given k and mu win over Re and U*
    c2 = viv.Case(M, I.viv_initial_velocity(mesh, 1.0, 1e-3, 1), 1.0, 0.02, 0.7, 0.1, Re=100.0, Ustar=8.0)
    p2 = c2.resolved_params()
    assert p2["k"] == 0.7 and p2["mu"] == 0.02
    c2.close()


@pytest.mark.parametrize("precision,pivoting,jac32,pred,cfl", [("mixed", 1, 1, 1, 0.0), ("fp64", 0, 0, 0, 0.0),
                                                               ("mixed", 1, 1, 1, 1.0)])
def test_resumed_case_steps_bit_for_bit(viv, precision, pivoting, jac32, pred, cfl):
    """A case saved after two steps and loaded into a fresh case of the same
    mesh takes a third step identical in every bit to the uninterrupted run
    (with adaptive steps too: the saved step sizes carry over)."""
    mesh = I.viv_cylinder_mesh(6)
    u0 = I.viv_initial_velocity(mesh, 1.0, 1e-3, 4)
    M = viv.Mesh(mesh)
    prec = viv.VIV_MIXED if precision == "mixed" else viv.VIV_FP64
    kw = dict(precision=prec, pivoting=pivoting, jacobian_fp32=jac32, predictor=pred, cfl_target=cfl)
    a = viv.viv_case(M, 150.0, 6.0, 0.05, u0, **kw)
    a.step()
    a.step()
    ckpt = a.save()
    info_a = a.step()
    sa = a.get_state()
    b = viv.viv_case(M, 150.0, 6.0, 0.05, np.zeros_like(u0), **kw)
    b.load(ckpt)
    info_b = b.step()
    sb = b.get_state()
    for k in ("u", "p", "x", "lam", "delta"):
        assert np.array_equal(sa[k], sb[k]), k
    assert sa["t"] == sb["t"] and info_a["newton_iters"] == info_b["newton_iters"]
    assert info_a["res_norm"] == info_b["res_norm"] and info_a["dt"] == info_b["dt"]
    # a checkpoint of another mesh, or a different dt, is refused
    other = viv.Mesh(I.viv_cylinder_mesh(4))
    c = viv.viv_case(other, 150.0, 6.0, 0.05, I.viv_initial_velocity(other.mesh, 1.0, 1e-3, 4), **kw)
    with pytest.raises(viv.VivError):
        c.load(ckpt)
    d = viv.viv_case(M, 150.0, 6.0, 0.04, u0, **kw)
    if cfl == 0:
        with pytest.raises(viv.VivError):
            d.load(ckpt)
    for x in (a, b, c, d):
        x.close()
