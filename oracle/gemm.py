"""FP64 reference of the batched small-matrix multiplication (the batched
GEMM of Sec. 4.2.5, the workload of the dynamic-tuning study of Sec. 5.2) --
TEST INFRASTRUCTURE ONLY.

C[b] = A[b] B[b], A[b] m x k, B[b] k x n; numpy's matmul in float64 is the
definition's product (a library primitive standing for the sum over the
inner index), and bgemm_loops writes the sum out for tiny pins."""
from __future__ import annotations

import numpy as np


def bgemm(A, B):
    return np.matmul(np.asarray(A, np.float64), np.asarray(B, np.float64))


def bgemm_loops(A, B):
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    nb, m, k = A.shape
    n = B.shape[2]
    C = np.zeros((nb, m, n))
    for b in range(nb):
        for i in range(m):
            for j in range(n):
                s = 0.0
                for p in range(k):
                    s += A[b, i, p] * B[b, p, j]
                C[b, i, j] = s
    return C


def fp32_error_bound(A, B):
    """Elementwise bound on |C_fp32 - C| for FP32 inputs and any FP32
    evaluation of the inner sum (FMA chain or not): gamma_k sum_p |a_ip b_pj|
    with gamma_k = k u / (1 - k u), u = 2^-24 (Higham, Accuracy and Stability
    of Numerical Algorithms, 2002, Sec. 3.1)."""
    A = np.abs(np.asarray(A, np.float64))
    B = np.abs(np.asarray(B, np.float64))
    k = A.shape[2]
    u = 2.0 ** -24
    g = k * u / (1 - k * u)
    return g * np.matmul(A, B)
