"""Pins of the FP64 batched-GEMM reference (oracle/gemm.py): the library
product against the written-out triple loop, the identity, a hand product,
and the FP32 error bound against an FP32 evaluation done in numpy."""
import numpy as np

from oracle import gemm


def test_matmul_matches_written_out_sum():
    rng = np.random.default_rng(1)
    for m, n, k in [(2, 2, 2), (3, 5, 7), (4, 1, 6)]:
        A = rng.standard_normal((3, m, k))
        B = rng.standard_normal((3, k, n))
        assert np.allclose(gemm.bgemm(A, B), gemm.bgemm_loops(A, B), rtol=0, atol=1e-13)


def test_identity_and_hand_product():
    I = np.eye(4)[None]
    B = np.arange(16.0).reshape(1, 4, 4)
    assert np.array_equal(gemm.bgemm(I, B), B)
    A = np.array([[[1.0, 2.0], [3.0, 4.0]]])
    Bm = np.array([[[5.0, 6.0], [7.0, 8.0]]])
    assert np.array_equal(gemm.bgemm(A, Bm), np.array([[[19.0, 22.0], [43.0, 50.0]]]))


def test_fp32_bound_covers_fp32_sequential_sums():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((50, 8, 32)).astype(np.float32)
    B = rng.standard_normal((50, 32, 8)).astype(np.float32)
    C32 = np.zeros((50, 8, 8), np.float32)
    for p in range(32):  # sequential FP32 accumulation, one rounding per step
        C32 = (C32 + A[:, :, p:p + 1] * B[:, p:p + 1, :]).astype(np.float32)
    err = np.abs(C32.astype(np.float64) - gemm.bgemm(A, B))
    assert np.all(err <= 2 * gemm.fp32_error_bound(A, B))
