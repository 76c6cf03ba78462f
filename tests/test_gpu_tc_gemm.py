"""tcgen05 3xTF32 Schur-complement update against an FP64 reference of the
same operation (C - A B), on tile-aligned and ragged shapes."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (200, 300, 128), (257, 129, 20), (64, 64, 8), (300, 1100, 200),
                                   (1000, 777, 96), (129, 1, 33)])
def test_tc_schur_update_matches_reference(M, N, K):
    import torch
    from paper_2609_31477_b300 import build, viv
    build.build()
    viv.load()
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g, dtype=torch.float64).float()
    B = torch.randn(K, N, generator=g, dtype=torch.float64).float()
    C0 = torch.randn(M, N, generator=g, dtype=torch.float64).float()
    ref = C0.double() - A.double() @ B.double()
    col = lambda t: t.t().contiguous().t().cuda()          # column-major device storage
    Ad, Bd, Cd = col(A), col(B), col(C0)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    viv.tc_schur_update(Ad, Bd, Cd, err)
    torch.cuda.synchronize()
    assert err.item() == 0
    got = Cd.double().cpu()
    scale = (A.double().abs() @ B.double().abs()).max() + C0.double().abs().max()
    rel = ((got - ref).abs().max() / scale).item()
    # 3xTF32 keeps FP32-level accuracy; a single TF32 product would be ~1e-3
    assert rel < 4e-6, rel
