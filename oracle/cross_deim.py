"""CPU Cross-DEIM (FP64; test infrastructure).

Follows the paper's Algorithm "scross" (stabilised cross approximation,
Sec. 2.1), the index selectors of Algorithm "(Q)DEIM" and Algorithm
"LeverageScores" (Sec. 2.2), and the adaptive loop of Algorithm "Cross-DEIM"
(Sec. 2.2.3), applied to the transformed Poisson solution of Sec. 3.2.
Library primitives serve as single steps (Householder QR, SVD, pinv, pivoted
QR); nothing is blocked, fused or reordered.

Readings where the paper is silent or garbled:
  * initial guess U_{-1}, V_{-1}: orthonormal bases of the numerical range of
    the transformed RHS factors (the paper only says "warm started"), columns
    whose Householder |R(l,l)| falls below 1e-12 max|diag R| dropped;
  * leverage scores: Algorithm LeverageScores as printed, Bernoulli sampling
    (the default selector "bernoulli"), c = sample_factor x columns, draws from
    Philox4x32-10; the selector "ls" takes the top-c rows deterministically
    instead (c = columns of the input basis), ties to the lower index;
  * new indices are appended after the previous ones in descending score;
  * the growth safeguard adds one index to I_k (not to I_k^*), drawn from the
    SplitMix64 generator (Steele, Lea, Flood 2014) keyed by (seed, k, side),
    then linear-probed to the first index not yet in the set;
  * the scross branch is |J| <= |I| (the paper's k <= l with k = |J|), and the
    mirror system uses Z(J, :);
  * the interpolatory solve always uses the SVD pseudoinverse with cutoff
    max(|I|,|J|) * eps * sigma_max;
  * the in-loop "truncated SVD" drops only numerically zero singular values,
    below max(|I|,|J|) * eps * sigma_1 (the pseudoinverse cutoff); a tail rule
    at tol here would keep S_min near tol and the stop test could never pass;
  * rho, S_min, the redundancy threshold and the final truncation are relative
    (to ||S_k||_F, ||S_k||_F, max|diag R| and ||S||_F);
  * eta_1 = ||U_k(I_k,:)^+||_2 and eta_2 = ||V_k(J_k,:)^+||_2 (the DEIM
    constants), with I_k, J_k after the redundancy removal.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

MASK64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014)."""
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def growth_index(seed: int, k: int, side: int, n: int, present) -> int:
    """Deterministic stand-in for i_rand in the complement of the index set."""
    i = splitmix64((seed + 2 * k + side) & MASK64) % n
    present = set(int(v) for v in present)
    if len(present) >= n:
        return -1
    while i in present:
        i = (i + 1) % n
    return int(i)


M32 = (1 << 32) - 1
PHILOX_M = (0xD2511F53, 0xCD9E8D57)   # multipliers of the Philox-4x32 S-box
PHILOX_W = (0x9E3779B9, 0xBB67AE85)   # Weyl increments of the key schedule


def philox4x32_10(ctr, key):
    """Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
    easy as 1, 2, 3", SC 2011): ten rounds of the 4x32 S-box on the counter
    (c0, c1, c2, c3), the 2x32 key advanced by the Weyl increments before every
    round but the first.  Counter words may be NumPy uint64 arrays holding
    32-bit values (vectorised over rows); returns the four output words."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & np.uint64(M32) for c in ctr)
    k0, k1 = int(key[0]) & M32, int(key[1]) & M32
    m0, m1 = np.uint64(PHILOX_M[0]), np.uint64(PHILOX_M[1])
    mask, sh = np.uint64(M32), np.uint64(32)
    for r in range(10):
        if r:
            k0 = (k0 + PHILOX_W[0]) & M32
            k1 = (k1 + PHILOX_W[1]) & M32
        p0 = m0 * c0  # exact: 32 x 32 -> 64 bits
        p1 = m1 * c2
        c0, c1, c2, c3 = ((p1 >> sh) ^ c1 ^ np.uint64(k0)) & mask, p1 & mask, \
            ((p0 >> sh) ^ c3 ^ np.uint64(k1)) & mask, p0 & mask
    return c0, c1, c2, c3


def philox_uniform(seed: int, k: int, side: int, rows) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits, one per row: Philox4x32-10
    with counter (row, k, side, 0) and key (low, high 32 bits of seed); the
    double is (x0 >> 5) 2^26 + (x1 >> 6), scaled by 2^-53 (exact)."""
    rows = np.asarray(rows, dtype=np.uint64)
    z = np.zeros_like(rows)
    x0, x1, _, _ = philox4x32_10((rows, z + np.uint64(k & M32), z + np.uint64(side & M32), z),
                                 (seed & M32, (seed >> 32) & M32))
    a = (x0 >> np.uint64(5)).astype(np.float64)
    b = (x1 >> np.uint64(6)).astype(np.float64)
    return (a * 67108864.0 + b) / 9007199254740992.0


def select_bernoulli(U: np.ndarray, seed: int, k: int, side: int, factor: float = 1.0) -> np.ndarray:
    """Algorithm LeverageScores as printed: row i is sampled independently with
    probability p_i = min(1, c pi_i), c = factor x (columns of U), pi the
    leverage scores; c pi_i is evaluated as factor x sum_eta U(i, eta)^2.  The
    draws are Philox uniforms (philox_uniform); sampled rows in descending score,
    ties to the lower index."""
    s = np.sum(U * U, axis=1)
    p = np.minimum(1.0, factor * s)
    u = philox_uniform(seed, k, side, np.arange(U.shape[0]))
    keep = np.nonzero(u < p)[0]
    order = np.lexsort((keep, -s[keep]))
    return keep[order]


def leverage_scores(U: np.ndarray) -> np.ndarray:
    """pi_i = (1/c) sum_eta U(i, eta)^2 for an n x c basis (Algorithm LeverageScores)."""
    return np.sum(U * U, axis=1) / U.shape[1]


def select_leverage(U: np.ndarray, c: int | None = None) -> np.ndarray:
    """Top-c rows by leverage score, descending, ties to the lower index."""
    c = U.shape[1] if c is None else c
    pi = leverage_scores(U)
    order = np.lexsort((np.arange(pi.shape[0]), -pi))
    return order[:c]


def select_qdeim(U: np.ndarray) -> np.ndarray:
    """QDEIM: the first c column pivots of a pivoted QR of U^T (Algorithm (Q)DEIM)."""
    _, _, piv = scipy.linalg.qr(U.T, mode="economic", pivoting=True)
    return piv[:U.shape[1]]


def select_deim(U: np.ndarray) -> np.ndarray:
    """DEIM: greedy interpolation points (Chaturantabut-Sorensen), rows of U."""
    n, c = U.shape
    idx = [int(np.argmax(np.abs(U[:, 0])))]
    for l in range(1, c):
        coef = np.linalg.solve(U[idx, :l], U[idx, l])
        res = U[:, l] - U[:, :l] @ coef
        idx.append(int(np.argmax(np.abs(res))))
    return np.array(idx)


SELECTORS = {"ls": select_leverage, "qdeim": select_qdeim, "deim": select_deim}


def union_ordered(prev, new, cap: int | None):
    """prev (kept order) followed by the entries of `new` not already present."""
    out = list(int(v) for v in prev)
    seen = set(out)
    for v in new:
        v = int(v)
        if v in seen:
            continue
        if cap is not None and len(out) >= cap:
            break
        out.append(v)
        seen.add(v)
    return out


@dataclass
class ScrossResult:
    U: np.ndarray
    S: np.ndarray
    V: np.ndarray
    rC: np.ndarray
    rR: np.ndarray


def scross(G, I, J, drop_rel: float) -> ScrossResult:
    """Algorithm scross: SVD of C G(I,J)^+ R from C = G(:,J), R = G(I,:).

    QR of C and R^T; if |J| <= |I| solve Q(I,:) W = R, else Z(J,:) W = C^T;
    SVD of the small core; the result is truncated to singular values
    >= drop_rel * sigma_1.
    """
    I = np.asarray(I, dtype=np.int64)
    J = np.asarray(J, dtype=np.int64)
    C = G.cols(J)
    Rt = G.rows(I).T
    Q, RC = np.linalg.qr(C)
    Z, RR = np.linalg.qr(Rt)
    p, q = J.shape[0], I.shape[0]
    eps = np.finfo(np.float64).eps
    if p <= q:
        core = np.linalg.pinv(Q[I, :], rtol=max(p, q) * eps) @ RR.T      # p x q
    else:
        core = RC @ np.linalg.pinv(Z[J, :], rtol=max(p, q) * eps).T      # p x q
    Ut, s, Vt = np.linalg.svd(core, full_matrices=False)
    if drop_rel is None:
        drop_rel = max(p, q) * eps
    r = int(np.sum(s >= drop_rel * s[0])) if s[0] > 0 else 1
    r = max(r, 1)
    return ScrossResult(Q @ Ut[:, :r], s[:r], Z @ Vt[:r].T, np.diag(RC).copy(),
                        np.diag(RR).copy())


def diff_norm(A, B) -> float:
    """||U_a S_a V_a^T - U_b S_b V_b^T||_F via QR of stacked factors."""
    if B is None:
        return float(np.linalg.norm(A[1]))
    U = np.concatenate([A[0], B[0]], axis=1)
    V = np.concatenate([A[2], B[2]], axis=1)
    D = np.concatenate([A[1], -B[1]])
    _, RU = np.linalg.qr(U)
    _, RV = np.linalg.qr(V)
    return float(np.linalg.norm((RU * D) @ RV.T))


def inv_smin(M: np.ndarray) -> float:
    """||M^+||_2 = 1 / sigma_min(M) (inf for a rank-deficient M)."""
    s = np.linalg.svd(M, compute_uv=False)
    if s.size == 0 or s[-1] <= 0:
        return float("inf")
    return float(1.0 / s[-1])


def tail_rank(s: np.ndarray, tol: float) -> int:
    """Smallest r with sum_{l > r} s_l^2 < tol^2 sum_l s_l^2 (final truncation)."""
    s2 = np.asarray(s, float) ** 2
    total = s2.sum()
    if total <= 0:
        return 1
    tail = np.concatenate([np.cumsum(s2[::-1])[::-1], [0.0]])  # tail[r] = sum_{l>=r}
    for r in range(0, s2.shape[0] + 1):
        if tail[r] < tol * tol * total:
            return max(r, 1)
    return s2.shape[0]


@dataclass
class CrossDEIMInfo:
    iterations: int = 0
    converged: bool = False
    rank_capped: bool = False
    r_star: int = 0
    rho: list = field(default_factory=list)
    eta_smin: list = field(default_factory=list)
    sizes: list = field(default_factory=list)
    ranks: list = field(default_factory=list)
    I: list = field(default_factory=list)
    J: list = field(default_factory=list)


def cross_deim(G, U0, V0, tol: float, r_max: int, maxiter: int = 30,
               selector: str = "bernoulli", seed: int = 0, m_cap: int | None = None,
               inloop_rel: float | None = None, redundancy: float = 1e-12,
               I0=None, J0=None, A0=None, sample_factor: float = 1.0):
    """Algorithm Cross-DEIM on a matrix given by entry access (G.cols / G.rows).

    Returns (U, S, V, info): the first r = max(min(r*, r_max), 1) singular
    triplets of the last cross approximation.
    """
    n_rows, n_cols = G.shape

    def sel(Ub, k, side):
        if selector == "bernoulli":
            return select_bernoulli(Ub, seed, k, side, sample_factor)
        return SELECTORS[selector](Ub)

    U_prev, V_prev = U0, V0
    I = list(I0) if I0 is not None else []
    J = list(J0) if J0 is not None else []
    A_prev = A0
    info = CrossDEIMInfo()
    drop_rel = None if inloop_rel is None else inloop_rel * tol
    res = None
    for k in range(maxiter):
        Istar = sel(U_prev, k, 0)
        Jstar = sel(V_prev, k, 1)
        I_new = union_ordered(I, Istar, m_cap)
        if (len(I_new) == len(I) or k == 0) and (m_cap is None or len(I_new) < m_cap):
            g = growth_index(seed, k, 0, n_rows, I_new)
            if g >= 0:
                I_new.append(g)
        J_new = union_ordered(J, Jstar, m_cap)
        if (len(J_new) == len(J) or k == 0) and (m_cap is None or len(J_new) < m_cap):
            g = growth_index(seed, k, 1, n_cols, J_new)
            if g >= 0:
                J_new.append(g)
        I, J = I_new, J_new
        info.sizes.append((len(I), len(J)))
        res = scross(G, I, J, drop_rel)
        # Remove redundant rows / columns (relative reading of |r| < 1e-12).
        aR = np.abs(res.rR)
        aC = np.abs(res.rC)
        I = [I[l] for l in range(len(I)) if aR[l] >= redundancy * aR.max()]
        J = [J[l] for l in range(len(J)) if aC[l] >= redundancy * aC.max()]
        A_k = (res.U, res.S, res.V)
        nrm = float(np.linalg.norm(res.S))
        rho = diff_norm(A_k, A_prev) / nrm
        smin = float(res.S[-1]) / nrm
        eta1 = inv_smin(res.U[np.asarray(I), :])
        eta2 = inv_smin(res.V[np.asarray(J), :])
        eta_s = min(eta1 * (1 + eta2), eta2 * (1 + eta1)) * smin
        info.rho.append(rho)
        info.eta_smin.append(eta_s)
        info.ranks.append(res.S.shape[0])
        info.iterations = k + 1
        A_prev = A_k
        U_prev, V_prev = res.U, res.V
        if max(rho, eta_s) < tol:
            info.converged = True
            break
    r_star = tail_rank(res.S, tol)
    r = max(min(r_star, r_max), 1)
    info.r_star = r_star
    info.rank_capped = r_star > r_max
    info.I, info.J = I, J
    info.last = (res.U, res.S, res.V)  # the last iterate before the final truncation
    return res.U[:, :r], res.S[:r], res.V[:, :r], info


def orth(X: np.ndarray, tau: float = 1e-12) -> np.ndarray:
    """Orthonormal basis of the numerical range of X: Householder QR, keeping
    the columns l of Q with |R(l,l)| >= tau max|diag R| (the relative reading of
    the paper's numerical-zero threshold 1e-12, the test of the redundancy
    removal).  A numerically dependent column of X (say, two equal terms of the
    right-hand side) would otherwise add a direction of pure rounding noise to
    the initial basis and to its leverage scores.  At least one column is kept."""
    Q, R = np.linalg.qr(X)
    d = np.abs(np.diag(R))
    if d.size == 0 or d.max() <= 0:
        return Q[:, :1]
    return Q[:, d >= tau * d.max()]


def poisson_solve(U_f, s_f, V_f, tol: float, r_max: int, maxiter: int = 30,
                  selector: str = "bernoulli", seed: int = 0, m_cap: int | None = None,
                  inloop_rel: float | None = None, warm=None, sample_factor: float = 1.0):
    """Low-rank Poisson solve of Sec. 3.2.

    Fhat = DST(U_f) S_f DST(V_f)^T, Cross-DEIM on What (Eq. g_for_p), then
    W = DST(Uhat) S DST(Vhat)^T.  `warm` = (I, J, (Uh, S, Vh)) from an earlier
    solve (its info.I, info.J and info.last) replaces the initial bases and the
    empty index sets; the first iteration's change rho is still measured from
    zero, as in a cold start.  Returns (U, S, V, info, G).
    """
    from .poisson import SpectralSolution, dst1

    G = SpectralSolution(U_f, s_f, V_f)
    if warm is None:
        U0, V0, I0, J0, A0 = orth(G.Uh), orth(G.Vh), None, None, None
    else:
        I0, J0, last = warm
        U0, V0, A0 = last[0], last[2], None
    Uh, S, Vh, info = cross_deim(G, U0, V0, tol, r_max, maxiter, selector, seed,
                                 m_cap, inloop_rel, I0=I0, J0=J0, A0=A0, sample_factor=sample_factor)
    info.spectral = (Uh, S, Vh)
    return dst1(Uh), S, dst1(Vh), info, G
