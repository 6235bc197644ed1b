"""Test matrices of the paper's Sec. 4.1 given by their entries (test
infrastructure; FP64).  Each exposes shape, cols(J) = G(:, J) and rows(I) =
G(I, :), the access Algorithm scross needs, and dense() for small sizes.

  H(i, j) = 1 / (1 + i + j)                  (Hilbert; indices from 0, so H is
                                              the standard Hilbert matrix)
  K(i, j) = (|x_i + y_j| / 2)^5,  x_i = -1 + 2 i/(m-1),  y_j = -1 + 2 j/(n-1)
                                             (i, j from 0: the paper's grid with
                                              indices from 1 shifted by one)
"""
from __future__ import annotations

import numpy as np


class HilbertMatrix:
    def __init__(self, n: int):
        self.n = n

    @property
    def shape(self):
        return (self.n, self.n)

    def _entries(self, i, j) -> np.ndarray:
        return 1.0 / (1.0 + i[:, None].astype(np.float64) + j[None, :].astype(np.float64))

    def cols(self, J) -> np.ndarray:
        return self._entries(np.arange(self.n), np.asarray(J, dtype=np.int64))

    def rows(self, I) -> np.ndarray:
        return self._entries(np.asarray(I, dtype=np.int64), np.arange(self.n))

    def dense(self) -> np.ndarray:
        return self.rows(np.arange(self.n))


class KMatrix:
    def __init__(self, n: int):
        self.n = n
        self.x = -1.0 + 2.0 * np.arange(n) / (n - 1)
        self.y = -1.0 + 2.0 * np.arange(n) / (n - 1)

    @property
    def shape(self):
        return (self.n, self.n)

    def _entries(self, i, j) -> np.ndarray:
        t = np.abs(self.x[i][:, None] + self.y[j][None, :]) / 2.0
        return t ** 5

    def cols(self, J) -> np.ndarray:
        return self._entries(np.arange(self.n), np.asarray(J, dtype=np.int64))

    def rows(self, I) -> np.ndarray:
        return self._entries(np.asarray(I, dtype=np.int64), np.arange(self.n))

    def dense(self) -> np.ndarray:
        return self.rows(np.arange(self.n))


MATRICES = {"hilbert": HilbertMatrix, "k": KMatrix}


def matrix_solve(kind: str, U0, V0, tol: float, r_max: int, **kw):
    """Algorithm Cross-DEIM on the n x n test matrix `kind` from initial guesses
    U0, V0 (orthonormalised first).  Returns (U, S, V, info, G)."""
    from .cross_deim import cross_deim, orth

    G = MATRICES[kind](U0.shape[0])
    U, S, V, info = cross_deim(G, orth(U0), orth(V0), tol, r_max, **kw)
    return U, S, V, info, G
