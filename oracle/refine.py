"""Low-rank residual and one step of iterative refinement (CPU FP64; test infrastructure).

Not in the paper: the mixed-precision path adds one refinement step.  Its
arithmetic is plain: for a trial solution W0 = U0 diag(S0) V0^T of
T W + W T = h^2 F (Eq. matrix_poisson) the residual

    R = h^2 F - (T W0 + W0 T)
      = [U_f, T U0, U0] diag(h^2 s_f, -S0, -S0) [V_f, V0, T V0]^T

has rank at most r_f + 2 r0.  Because T = Z Lambda Z (Sec. 3) the same residual
in transformed variables is Rhat = Z R Z with factors
[Uh_f, Lambda Uh0, Uh0] and [Vh_f, Vh0, Lambda Vh0].  The correction dW solves
T dW + dW T = R, i.e. dWhat(i,j) = Rhat(i,j) / (lambda_i + lambda_j)
(Eq. g_for_p with h^2 F replaced by R), and W1 = W0 + dW.

Pins (tests/test_oracle_refine.py): the factor form equals the dense 5-point
residual and its transform; one step from a perturbed trial solution reduces
the error against the exact solution by orders of magnitude.
"""
from __future__ import annotations

import numpy as np

from .poisson import SpectralSolution, apply_T, eigenvalues
from .cross_deim import cross_deim, orth, tail_rank


def physical_residual_factors(U_f, s_f, V_f, U0, S0, V0):
    """(X, d, Y) with X diag(d) Y^T = h^2 F - (T W0 + W0 T)."""
    n = U_f.shape[0]
    h = 1.0 / (n + 1)
    X = np.concatenate([U_f, apply_T(U0), U0], axis=1)
    Y = np.concatenate([V_f, V0, apply_T(V0)], axis=1)
    d = np.concatenate([h * h * np.asarray(s_f, float), -np.asarray(S0, float),
                        -np.asarray(S0, float)])
    return X, d, Y


def spectral_residual_factors(Uh_f, s_f, Vh_f, Uh0, S0, Vh0):
    """(X, d, Y) with X diag(d) Y^T = h^2 Fhat - (Lambda What0 + What0 Lambda)."""
    n = Uh_f.shape[0]
    h = 1.0 / (n + 1)
    lam = eigenvalues(n)
    X = np.concatenate([Uh_f, lam[:, None] * Uh0, Uh0], axis=1)
    Y = np.concatenate([Vh_f, Vh0, lam[:, None] * Vh0], axis=1)
    d = np.concatenate([h * h * np.asarray(s_f, float), -np.asarray(S0, float),
                        -np.asarray(S0, float)])
    return X, d, Y


def recompress(X, d, Y, rel: float, r_max: int | None = None):
    """Truncated SVD of X diag(d) Y^T via Householder QR of X and Y and an SVD
    of the small core R_X diag(d) R_Y^T; keeps the tail-rule rank at `rel`."""
    QX, RX = np.linalg.qr(X)
    QY, RY = np.linalg.qr(Y)
    Ut, s, Vt = np.linalg.svd((RX * d) @ RY.T)
    r = tail_rank(s, rel)
    if r_max is not None:
        r = max(min(r, r_max), 1)
    return QX @ Ut[:, :r], s[:r], QY @ Vt[:r].T


def refine_once(G: SpectralSolution, Uh0, S0, Vh0, tol: float, r_max: int,
                maxiter: int = 30, seed: int = 0, m_cap: int | None = None,
                residual_rel: float = 1e-14):
    """One refinement step in transformed variables; returns (Uh1, S1, Vh1, info)."""
    X, d, Y = spectral_residual_factors(G.Uh, G.s, G.Vh, Uh0, S0, Vh0)
    Ur, sr, Vr = recompress(X, d, Y, residual_rel)
    h = G.h
    Gd = SpectralSolution(Ur, sr / (h * h), Vr, transformed=True)
    dU, dS, dV, info = cross_deim(Gd, orth(Ur), orth(Vr), tol, m_cap or 10**9,
                                  maxiter, "ls", seed, m_cap)
    U = np.concatenate([Uh0, dU], axis=1)
    V = np.concatenate([Vh0, dV], axis=1)
    s = np.concatenate([np.asarray(S0, float), dS])
    U1, S1, V1 = recompress(U, s, V, tol, r_max)
    return U1, S1, V1, info
