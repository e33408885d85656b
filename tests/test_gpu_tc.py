"""The tcgen05 3xTF32 GEMM tile (the nonlocal step's building block) against an
FP64 numpy product: 3xTF32 keeps ~21 significant bits, so the relative error
must be FP32-like (< 1e-5 of the largest entry at K = 513), far below
single-pass TF32 (~1e-3)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 16, 32), (300, 48, 77), (129, 256, 100), (64, 64, 1),
                                   (1000, 128, 513)])
def test_tc_gemm_nt_matches_fp64(M, N, K):
    import __graft_entry__ as ge
    ge.build()
    from paper_2410_02754_gb300.gbchfsi import tc_gemm_nt
    rng = np.random.default_rng(M + N + K)
    A = rng.normal(size=(M, K)).astype(np.float32)
    B = rng.normal(size=(N, K)).astype(np.float32)
    D = tc_gemm_nt(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy()
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    err = np.abs(D - ref).max() / np.abs(ref).max()
    assert err < 1e-5, err
