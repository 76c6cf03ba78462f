"""The serving loop and checkpoints across the three element families: a Q2
quad case, a periodic hexahedral (3-D) case and a P2-P1 triangle case served
together give the states each gives alone, and a case of each family resumed
from a checkpoint steps bit for bit like the uninterrupted run."""
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


def _meshes():
    return {"quad": I.viv_cylinder_mesh(4),
            "hex": I.viv_cylinder_mesh3d(2, 2, 0.7),
            "tri": I.triangulate_q2(I.viv_cylinder_mesh(4))}


def test_families_alone_and_in_the_mix_match(viv):
    meshes = _meshes()
    dev = {k: viv.Mesh(m) for k, m in meshes.items()}
    u0 = {k: I.viv_initial_velocity(m, 1.0, 1e-3, 3) for k, m in meshes.items()}
    alone = {}
    for k in meshes:
        srv = viv.Server(8 << 30, max_active=1)
        rid = srv.submit(dev[k], u0[k], Re=150.0, Ustar=6.0, dt=0.05, n_steps=3)
        res = srv.wait_all(1)
        assert res[0]["status"] == "OK", res
        alone[k] = srv.state(rid, len(meshes[k]["X"]), dev[k].dim)
        srv.close()
    mix = viv.Server(8 << 30, max_active=3)
    ids = {k: mix.submit(dev[k], u0[k], Re=150.0, Ustar=6.0, dt=0.05, n_steps=3) for k in meshes}
    res = mix.wait_all(3)
    assert all(r["status"] == "OK" for r in res), res
    for k, rid in ids.items():
        got = mix.state(rid, len(meshes[k]["X"]), dev[k].dim)
        for f in ("u", "p", "x", "lam", "delta"):
            assert np.abs(got[f] - alone[k][f]).max() <= 1e-12 * max(1.0, np.abs(alone[k][f]).max()), (k, f)
    mix.close()


@pytest.mark.parametrize("family", ["hex", "tri"])
def test_resumed_case_steps_bit_for_bit(viv, family):
    mesh = _meshes()[family]
    u0 = I.viv_initial_velocity(mesh, 1.0, 1e-3, 4)
    M = viv.Mesh(mesh)
    kw = dict(precision=viv.VIV_MIXED, pivoting=viv.VIV_PIVOT_WINDOW, jacobian_fp32=1, predictor=1)
    a = viv.viv_case(M, 150.0, 6.0, 0.05, u0, **kw)
    a.step()
    a.step()
    ckpt = a.save()
    a.step()
    sa = a.get_state()
    b = viv.viv_case(M, 150.0, 6.0, 0.05, np.zeros_like(u0), **kw)
    b.load(ckpt)
    b.step()
    sb = b.get_state()
    for f in ("u", "p", "x", "lam", "delta"):
        assert np.array_equal(sa[f], sb[f]), f
    assert sa["t"] == sb["t"]
