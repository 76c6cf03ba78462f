"""Allocation-free solve.

Callers that cannot allocate device memory while they run - a framework whose
memory pool is already committed, or a latency-bound loop that cannot take the
device-wide synchronisation of cudaMalloc - use viv_lu_solve_noalloc, whose
workspace is a fixed array inside the library.  This checks, through the C
ABI, that it returns the same solution as the regular viv_solve_rhs, on two
calls in a row (the shared workspace keeps the previous call's contents)."""
import numpy as np
import pytest

from paper_2609_31477_b300 import inputs as I

pytestmark = pytest.mark.gpu


def test_noalloc_solve_matches_regular_solve_on_two_calls():
    import torch
    from paper_2609_31477_b300 import build, viv
    build.build()
    viv.load()
    mesh = I.viv_cylinder_mesh(4)
    u0 = I.viv_initial_velocity(mesh, 1.0, 1e-3, 1)
    M = viv.Mesh(mesh)
    case = viv.viv_case(M, 100.0, 8.0, 0.1, u0, precision=viv.VIV_FP64)
    case.begin_step()
    case.assemble(viv.VIV_RES | viv.VIV_JAC)
    case.factor()
    rng = np.random.default_rng(7)
    for _ in range(2):
        b = rng.standard_normal(M.n_dofs)
        ref, _ = case.solve_rhs(b)
        bd = torch.tensor(b, device="cuda")
        xd = torch.full_like(bd, float("nan"))
        torch.cuda.synchronize()          # inputs ready before the case stream reads them
        case.lu_solve_noalloc(bd, xd)
        torch.cuda.synchronize()          # the solve ran on the case's own stream
        x = xd.cpu().numpy()
        assert np.all(np.isfinite(x))
        assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)
    case.close()
    M.close()
