"""The test matrices of Sec. 4.1 and Cross-DEIM on them (oracle pins)."""
import numpy as np
import pytest
import scipy.linalg

import lrp_inputs as li
from oracle import cross_deim as cd
from oracle import matrices as om


def test_hilbert_is_the_standard_hilbert_matrix():
    n = 40
    H = om.HilbertMatrix(n)
    assert np.array_equal(H.dense(), scipy.linalg.hilbert(n))
    J = [3, 0, 17]
    assert np.array_equal(H.cols(J), scipy.linalg.hilbert(n)[:, J])
    assert np.array_equal(H.rows(J), scipy.linalg.hilbert(n)[J, :])


def test_k_matrix_closed_forms():
    n = 101
    K = om.KMatrix(n).dense()
    assert K[0, 0] == 1.0 and K[-1, -1] == 1.0          # |(-1) + (-1)| / 2 = 1
    assert np.all(np.abs(np.diag(K[:, ::-1])) < 1e-30)  # x_i + y_{n-1-i} = 0: the kink
    assert np.allclose(K, K.T)                          # same grid on both axes
    i, j = 10, 70
    x = -1 + 2 * i / (n - 1)
    y = -1 + 2 * j / (n - 1)
    assert K[i, j] == pytest.approx((abs(x + y) / 2) ** 5, rel=1e-15)
    # C^4 but not smooth: slow singular value decay compared with H
    sk = np.linalg.svd(K, compute_uv=False)
    sh = np.linalg.svd(om.HilbertMatrix(n).dense(), compute_uv=False)
    assert sk[20] / sk[0] > 1e3 * sh[20] / sh[0]


@pytest.mark.parametrize("kind,tol", [("hilbert", 1e-9), ("k", 1e-6)])
def test_cross_deim_qdeim_on_test_matrices(kind, tol):
    # QDEIM (the paper's preferred selector on these matrices, Sec. 4.1)
    # converges in a few iterations to within 10 tol of the matrix, and within a
    # modest factor of the best approximation of the same rank (Eckart-Young).
    n = 300
    x0 = li.initial_bases(n, 4, 7)
    U, S, V, info, G = om.matrix_solve(kind, x0.U, x0.V, tol, 128, selector="qdeim", seed=7)
    A = G.dense()
    err = np.linalg.norm(A - (U * S) @ V.T) / np.linalg.norm(A)
    s = np.linalg.svd(A, compute_uv=False)
    best = np.sqrt(np.sum(s[S.shape[0]:] ** 2)) / np.linalg.norm(s)
    assert info.converged and info.iterations <= 8, info.iterations
    assert err < 10 * tol, (err, info.iterations, S.shape[0])
    assert err < 100 * max(best, 1e-15) + 10 * tol
    assert np.abs(U.T @ U - np.eye(S.shape[0])).max() < 1e-10


def test_cross_deim_leverage_on_test_matrices_is_weaker():
    # The top-c leverage selector grows the index sets more slowly (Sec. 4.1 finds
    # LS clearly worse on both matrices): on H its change drops to rounding level
    # while the eta S_min term keeps the stop test open; the iterate is still a
    # close approximation.
    n = 300
    x0 = li.initial_bases(n, 4, 7)
    U, S, V, info, G = om.matrix_solve("hilbert", x0.U, x0.V, 1e-9, 128, selector="ls", seed=7)
    A = G.dense()
    err = np.linalg.norm(A - (U * S) @ V.T) / np.linalg.norm(A)
    assert min(info.rho) < 1e-12
    assert err < 1e-5
    _, _, _, info_q, _ = om.matrix_solve("hilbert", x0.U, x0.V, 1e-9, 128, selector="qdeim", seed=7)
    assert info.iterations > info_q.iterations
