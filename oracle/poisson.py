"""Poisson model problem, DST-I and exact solution (CPU, FP64; test infrastructure).

Paper Sec. 3: the 5-point Laplacian on the unit square with zero Dirichlet data
and ``n`` interior points per dimension gives ``T W + W T^T = h^2 F``
(Eq. matrix_poisson), ``h = 1/(n+1)``, ``T = tridiag(-1, 2, -1)``.
``T = Z Lambda Z^T`` with ``lambda_k = 2(1 - cos(pi k/(n+1)))`` and
``z_k(i) = sqrt(2/(n+1)) sin(i k pi/(n+1))``.  ``Z`` is symmetric and
orthogonal, so it is its own inverse (the normalised DST with DST(DST(I)) = I,
Sec. 3.2).  In the transformed variables the equation decouples
(Eq. g_for_p): ``What(i,j) = h^2 Fhat(i,j) / (lambda_i + lambda_j)``.

Pins (tests/test_oracle_poisson.py): Z against the direct O(n^2) sine sum and
Z @ Z = I; lambda against numpy.linalg.eigh(T); the full-grid solve against a
dense Kronecker LU solve (n <= 31) and the 5-point residual; the eigenfunction
right-hand side against its closed-form rank-1 solution.
"""
from __future__ import annotations

import numpy as np
import scipy.fft


def eigenvalues(n: int) -> np.ndarray:
    """lambda_k, k = 1..n, in the cancellation-free form 4 sin^2(pi k / (2(n+1))).

    Equal to the paper's 2(1 - cos(pi k/(n+1))) (half-angle identity); the sine
    form keeps full relative accuracy for small k at large n.
    """
    k = np.arange(1, n + 1, dtype=np.float64)
    return 4.0 * np.sin(np.pi * k / (2.0 * (n + 1))) ** 2


def eigenvalues_printed(n: int) -> np.ndarray:
    """lambda_k exactly as printed in Sec. 3: 2(1 - cos(pi k/(n+1)))."""
    k = np.arange(1, n + 1, dtype=np.float64)
    return 2.0 * (1.0 - np.cos(np.pi * k / (n + 1)))


def tridiag(n: int) -> np.ndarray:
    """Dense T = tridiag(-1, 2, -1) (n x n), Sec. 3."""
    return 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)


def dst_matrix(n: int) -> np.ndarray:
    """Dense Z with Z[i-1, k-1] = sqrt(2/(n+1)) sin(i k pi/(n+1)), Sec. 3."""
    i = np.arange(1, n + 1, dtype=np.float64)
    return np.sqrt(2.0 / (n + 1)) * np.sin(np.pi * np.outer(i, i) / (n + 1))


def dst1_direct(X: np.ndarray) -> np.ndarray:
    """Z @ X by the O(n^2) definition (for pins only)."""
    return dst_matrix(X.shape[0]) @ X


def dst1(X: np.ndarray) -> np.ndarray:
    """Z @ X along axis 0 via scipy's orthonormal DST-I (O(n log n) per column)."""
    return scipy.fft.dst(np.asarray(X, dtype=np.float64), type=1, norm="ortho", axis=0)


def apply_T(X: np.ndarray) -> np.ndarray:
    """T @ X by the 1-D 3-point stencil with zero Dirichlet ends."""
    Y = 2.0 * X
    Y[1:] -= X[:-1]
    Y[:-1] -= X[1:]
    return Y


def residual_5pt(W: np.ndarray, F: np.ndarray) -> np.ndarray:
    """T W + W T - h^2 F on the full grid (Eq. matrix_poisson)."""
    n = W.shape[0]
    h = 1.0 / (n + 1)
    return apply_T(W) + apply_T(W.T).T - h * h * F


def full_grid_solve(F: np.ndarray) -> np.ndarray:
    """Full-rank DST solver of Sec. 3.1: Fhat = Z F Z, divide, W = Z What Z."""
    n = F.shape[0]
    h = 1.0 / (n + 1)
    lam = eigenvalues(n)
    Fh = dst1(dst1(F).T).T
    Wh = h * h * Fh / (lam[:, None] + lam[None, :])
    return dst1(dst1(Wh).T).T


def kron_solve(F: np.ndarray) -> np.ndarray:
    """Dense (I (x) T + T (x) I) vec(W) = h^2 vec(F) by LU (n <= 31 only)."""
    n = F.shape[0]
    h = 1.0 / (n + 1)
    T = tridiag(n)
    I = np.eye(n)
    A = np.kron(I, T) + np.kron(T, I)
    # column-major vec: vec(T W + W T) = (I (x) T + T^T (x) I) vec(W)
    w = np.linalg.solve(A, h * h * F.reshape(-1, order="F"))
    return w.reshape(n, n, order="F")


class SpectralSolution:
    """Entry access to the exact transformed solution What (Eq. g_for_p).

    With F = U_f diag(s_f) V_f^T, Fhat = Uh diag(s_f) Vh^T where Uh = Z U_f and
    Vh = Z V_f (Sec. 3.2), so What(i,j) = h^2 sum_k Uh(i,k) s_k Vh(j,k) /
    (lambda_i + lambda_j) costs O(r_f) per entry (Sec. 2.1, entries at O(r)).
    """

    def __init__(self, U: np.ndarray, s: np.ndarray, V: np.ndarray, transformed: bool = False):
        self.n = U.shape[0]
        self.h = 1.0 / (self.n + 1)
        self.lam = eigenvalues(self.n)
        self.Uh = np.array(U, dtype=np.float64) if transformed else dst1(U)
        self.Vh = np.array(V, dtype=np.float64) if transformed else dst1(V)
        self.s = np.asarray(s, dtype=np.float64)

    @property
    def shape(self):
        return (self.n, self.n)

    def cols(self, J) -> np.ndarray:
        """What(:, J), n x |J|."""
        J = np.asarray(J, dtype=np.int64)
        num = (self.Uh * self.s) @ self.Vh[J].T
        return self.h * self.h * num / (self.lam[:, None] + self.lam[None, J])

    def rows(self, I) -> np.ndarray:
        """What(I, :), |I| x n."""
        I = np.asarray(I, dtype=np.int64)
        num = (self.Uh[I] * self.s) @ self.Vh.T
        return self.h * self.h * num / (self.lam[I, None] + self.lam[None, :])

    def dense(self) -> np.ndarray:
        return self.rows(np.arange(self.n))


def lowrank_rel_diff(U1, S1, V1, U2, S2, V2) -> float:
    """||U1 S1 V1^T - U2 S2 V2^T||_F / ||U2 S2 V2^T||_F without forming n x n.

    Householder QR of the stacked factors moves the cancellation into a small
    core, so the result is accurate even when the difference is ~1e-14.
    """
    U = np.concatenate([U1, U2], axis=1)
    V = np.concatenate([V1, V2], axis=1)
    D = np.concatenate([np.asarray(S1, float), -np.asarray(S2, float)])
    _, RU = np.linalg.qr(U)
    _, RV = np.linalg.qr(V)
    diff = np.linalg.norm((RU * D) @ RV.T)
    _, R2u = np.linalg.qr(U2)
    _, R2v = np.linalg.qr(V2)
    ref = np.linalg.norm((R2u * np.asarray(S2, float)) @ R2v.T)
    return float(diff / ref)


def rel_error_vs_exact(U, S, V, exact: SpectralSolution, block: int = 1024,
                       rows=None) -> float:
    """||W - W_ex||_F / ||W_ex||_F for a physical-space result W = U diag(S) V^T.

    Z is orthogonal, so the error equals ||Z U S (Z V)^T - What_ex||_F; it is
    summed exactly over row blocks of the transformed grid (or over the given
    rows only, which yields the error restricted to those rows).
    """
    Uh = dst1(U) * np.asarray(S, float)
    Vh = dst1(V)
    n = exact.n
    idx = np.arange(n) if rows is None else np.asarray(rows)
    num = 0.0
    den = 0.0
    for b in range(0, idx.shape[0], block):
        I = idx[b:b + block]
        E = exact.rows(I)
        num += float(np.sum((E - Uh[I] @ Vh.T) ** 2))
        den += float(np.sum(E ** 2))
    return float(np.sqrt(num / den))


def rel_error_sampled(U, S, V, exact: SpectralSolution, n_low: int = 256, per_stratum: int = 32,
                      seed: int = 0, block: int = 16):
    """Stratified estimate of ||W - W_ex||_F / ||W_ex||_F for grids too large to sum.

    Transformed space as in rel_error_vs_exact (Z orthogonal).  The transformed
    rows are split by frequency: rows [0, n_low) (the low frequencies, which
    hold most of the mass) are summed exactly; then geometric strata
    [L, 2L), [2L, 4L), ... up to n, from each of which per_stratum rows are
    drawn uniformly without replacement (all of it when smaller), each row's sums
    exact and scaled by the stratum size over the sample size.  Returns
    (estimate, standard error): the variance of each stratum's scaled sum from
    its sample variance with the finite-population correction, carried through
    rel = sqrt(num / den) to first order.  When every stratum is taken whole
    the estimate is exact and the standard error 0.
    """
    Uh = dst1(U) * np.asarray(S, float)
    Vh = dst1(V)
    n = exact.n
    L = max(1, min(n_low, n))

    def row_sums(I):
        e = np.empty(len(I))
        d = np.empty(len(I))
        for b in range(0, len(I), block):
            Ib = np.asarray(I[b:b + block])
            E = exact.rows(Ib)
            e[b:b + len(Ib)] = np.sum((E - Uh[Ib] @ Vh.T) ** 2, axis=1)
            d[b:b + len(Ib)] = np.sum(E ** 2, axis=1)
        return e, d

    e1, d1 = row_sums(np.arange(L))
    num, den = float(e1.sum()), float(d1.sum())
    var_num = var_den = cov = 0.0
    rng = np.random.default_rng(seed)
    lo = L
    while lo < n:
        hi = min(2 * lo, n)
        size = hi - lo
        m = min(per_stratum, size)
        I = lo + (np.arange(size) if m == size else rng.choice(size, size=m, replace=False))
        e2, d2 = row_sums(I)
        scale = size / m
        num += scale * float(e2.sum())
        den += scale * float(d2.sum())
        if 1 < m < size:
            f = size * size / m * (1.0 - m / size)
            var_num += f * float(np.var(e2, ddof=1))
            var_den += f * float(np.var(d2, ddof=1))
            cov += f * float(np.cov(e2, d2, ddof=1)[0, 1])
        lo = hi
    q = num / den
    var_q = (var_num - 2 * q * cov + q * q * var_den) / (den * den)
    rel = float(np.sqrt(q))
    se = float(np.sqrt(max(var_q, 0.0)) / (2 * rel)) if rel > 0 else 0.0
    return rel, se
