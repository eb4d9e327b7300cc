"""The block algebra of the mixed path's tensor-core M~ inverse, replayed in
NumPy FP64 on the CPU (the GPU kernels are checked against FP64 products in
tests/test_gpu_tc_gemm.py; this checks the algorithm they implement): the
matrix padded to a multiple of 128 with a scaled identity, a right-looking
Cholesky by 128-blocks (panel A_ik L_kk^-T, trailing A_ij -= L_ik L_jk^T),
X = L^-1 by the recursive 2 x 2 block formula with the products in the
library's orientation (TT = XT11 L21^T, X21 = -X22 TT^T, XT12 = X21^T), and
M^-1 = X^T X restricted to the original n x n corner."""
import numpy as np
import pytest

P = 128


def _trtri(L, X, XT, b0, b1):
    if b1 - b0 <= 1:
        return
    m = b0 + (b1 - b0) // 2
    _trtri(L, X, XT, b0, m)
    _trtri(L, X, XT, m, b1)
    r1, r2 = slice(b0 * P, m * P), slice(m * P, b1 * P)
    TT = XT[r1, r1] @ L[r2, r1].T            # (L21 X11)^T
    X[r2, r1] = -X[r2, r2] @ TT.T            # -X22 L21 X11
    XT[r1, r2] = X[r2, r1].T


def spd_inverse_blocked(M, pad):
    n = M.shape[0]
    npad = -(-n // P) * P
    nb = npad // P
    A = np.eye(npad) * pad
    A[:n, :n] = M
    Dinv = []
    for k in range(nb):
        kk = slice(k * P, (k + 1) * P)
        Lkk = np.linalg.cholesky(A[kk, kk])
        A[kk, kk] = Lkk
        Dk = np.linalg.inv(Lkk)
        Dinv.append(Dk)
        rest = slice((k + 1) * P, npad)
        if (k + 1) * P < npad:
            A[rest, kk] = A[rest, kk] @ Dk.T                   # panel
            A[rest, rest] -= np.tril(A[rest, kk] @ A[rest, kk].T)  # trailing (lower part used)
    L = np.tril(A)
    X = np.zeros((npad, npad))
    XT = np.zeros((npad, npad))
    for k in range(nb):
        kk = slice(k * P, (k + 1) * P)
        X[kk, kk] = Dinv[k]
        XT[kk, kk] = Dinv[k].T
    _trtri(L, X, XT, 0, nb)
    Minv = XT @ XT.T
    return Minv[:n, :n], L, X


@pytest.mark.parametrize("n", [40, 128, 300, 700, 1000])
def test_blocked_inverse_equals_dense_inverse(n):
    rng = np.random.default_rng(n)
    B = rng.standard_normal((n, n))
    M = B @ B.T / n + 0.5 * np.eye(n)
    Minv, L, X = spd_inverse_blocked(M, pad=1.0)
    assert np.allclose(X @ L, np.eye(L.shape[0]), atol=1e-10)   # X = L^-1
    ref = np.linalg.inv(M)
    assert np.abs(Minv - ref).max() < 1e-10 * np.abs(ref).max()
    assert np.allclose(Minv, Minv.T, atol=1e-12 * np.abs(ref).max())
