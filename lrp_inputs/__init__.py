"""Seeded synthetic right-hand sides for the low-rank Poisson workloads.

This module only draws and tabulates inputs.  It holds none of the solver's
arithmetic (no sine transform, no eigenvalues, no cross approximation), so both
the CPU oracle and the GPU path may take their inputs from here.

Every right-hand side is returned as FP64 factors ``F = U_f diag(s_f) V_f^T``
sampled on the interior grid ``x_i = i*h``, ``i = 1..n``, ``h = 1/(n+1)``
(the grid of the paper's Sec. 3, 5-point Laplacian on the unit square).

Draw order (fixed, so a seed names one input):
  Gaussians:  a ~ N(0,1) [K], x_c ~ U[0.2,0.8] [K], y_c ~ U[0.2,0.8] [K],
              s ~ U[s_lo, s_hi] [K]
  eigenfunctions (after the Gaussians): p ~ U{1..pmax} [E], q ~ U{1..pmax} [E],
              a ~ N(0,1) [E]
A Gaussian term k contributes the separable product
  a_k * exp(-(x-x_k)^2/(2 s_k^2)) * exp(-(y-y_k)^2/(2 s_k^2)),
an eigenfunction term the product a * sin(p pi x) * sin(q pi y).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class LowRankRHS:
    n: int
    U: np.ndarray  # n x r_f, FP64, column-major friendly (Fortran order)
    s: np.ndarray  # r_f weights
    V: np.ndarray  # n x r_f

    @property
    def rank(self) -> int:
        return int(self.s.shape[0])

    @property
    def h(self) -> float:
        return 1.0 / (self.n + 1)

    def dense(self) -> np.ndarray:
        """The n x n grid function F (only for small n)."""
        return (self.U * self.s) @ self.V.T


def grid(n: int) -> np.ndarray:
    """Interior grid points x_i = i/(n+1), i = 1..n."""
    return np.arange(1, n + 1, dtype=np.float64) / (n + 1)


def gaussian_eigen_rhs(n: int, seed: int, n_gauss: int, n_eigen: int = 0,
                       s_lo: float = 0.05, s_hi: float = 0.15,
                       pmax: int = 64) -> LowRankRHS:
    """Sum of seeded separable Gaussians plus discrete eigenfunctions."""
    rng = np.random.default_rng(seed)
    x = grid(n)
    a = rng.standard_normal(n_gauss)
    xc = rng.uniform(0.2, 0.8, n_gauss)
    yc = rng.uniform(0.2, 0.8, n_gauss)
    sg = rng.uniform(s_lo, s_hi, n_gauss)
    U = np.exp(-((x[:, None] - xc[None, :]) ** 2) / (2.0 * sg[None, :] ** 2))
    V = np.exp(-((x[:, None] - yc[None, :]) ** 2) / (2.0 * sg[None, :] ** 2))
    s = a.copy()
    if n_eigen > 0:
        p = rng.integers(1, pmax + 1, n_eigen)
        q = rng.integers(1, pmax + 1, n_eigen)
        ae = rng.standard_normal(n_eigen)
        Ue = np.sin(np.pi * x[:, None] * p[None, :])
        Ve = np.sin(np.pi * x[:, None] * q[None, :])
        U = np.concatenate([U, Ue], axis=1)
        V = np.concatenate([V, Ve], axis=1)
        s = np.concatenate([s, ae])
    return LowRankRHS(n, np.asfortranarray(U), s, np.asfortranarray(V))


def eigenfunction_rhs(n: int, p: int, q: int, a: float = 1.0) -> LowRankRHS:
    """Rank-1 right-hand side a*sin(p pi x) sin(q pi y) (a discrete eigenfunction)."""
    x = grid(n)
    U = np.sin(np.pi * p * x)[:, None]
    V = np.sin(np.pi * q * x)[:, None]
    return LowRankRHS(n, np.asfortranarray(U), np.array([a]), np.asfortranarray(V))


# --- The five synthetic workloads (sizes, ranks, tolerances) -----------------

def workload_single_small(seed: int = 0) -> LowRankRHS:
    """n = 255 (h = 1/256), 4 Gaussians, tol 1e-10, max rank 32, FP64."""
    return gaussian_eigen_rhs(255, seed, 4)


def workload_n4095(seed: int = 0) -> LowRankRHS:
    """n = 4095, 16 Gaussians + 4 eigenfunctions (p, q in 1..64)."""
    return gaussian_eigen_rhs(4095, seed, 16, 4)


def workload_large(seed: int = 0, n: int = (1 << 20) - 1) -> LowRankRHS:
    """n = 2^20 - 1, 32 narrow Gaussians (s in [0.005, 0.05])."""
    return gaussian_eigen_rhs(n, seed, 32, 0, s_lo=0.005, s_hi=0.05)


def perturb_amplitudes(rhs: LowRankRHS, seed: int, rel: float = 0.01) -> LowRankRHS:
    """Warm re-solve input: a_k * (1 + rel * N(0,1))."""
    rng = np.random.default_rng(seed)
    s = rhs.s * (1.0 + rel * rng.standard_normal(rhs.s.shape[0]))
    return LowRankRHS(rhs.n, rhs.U, s, rhs.V)


def batch_mixed_sizes(count: int, seed: int = 0,
                      sizes=(511, 1023, 2047, 4095, 8191),
                      rank_lo: int = 2, rank_hi: int = 24):
    """Batched workload: n uniform over `sizes`, Gaussian rank uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=count)
    rs = rng.integers(rank_lo, rank_hi + 1, size=count)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    return [gaussian_eigen_rhs(int(n), int(sd), int(r)) for n, r, sd in zip(ns, rs, seeds)]


@dataclass
class Request:
    t_arrival: float
    rhs: LowRankRHS
    mixed: bool
    tol: float
    repeat_of: int  # -1, or index of an earlier request this perturbs


def serving_stream(count: int, rate: float, seed: int = 0, kmin: int = 8, kmax: int = 18,
                   rank_lo: int = 2, rank_hi: int = 48, frac_fp64: float = 0.2,
                   frac_repeat: float = 0.1):
    """Poisson-process arrivals; n = 2^k - 1; 20% FP64 at 1e-10, 80% mixed at 1e-6;
    10% are perturbed repeats of an earlier request."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    out = []
    for i in range(count):
        if i > 0 and rng.uniform() < frac_repeat:
            j = int(rng.integers(0, i))
            base = out[j]
            rhs = perturb_amplitudes(base.rhs, int(rng.integers(0, 2**31 - 1)))
            out.append(Request(float(t[i]), rhs, base.mixed, base.tol, j))
            continue
        k = int(rng.integers(kmin, kmax + 1))
        r = int(rng.integers(rank_lo, rank_hi + 1))
        fp64 = rng.uniform() < frac_fp64
        rhs = gaussian_eigen_rhs((1 << k) - 1, int(rng.integers(0, 2**31 - 1)), r)
        out.append(Request(float(t[i]), rhs, not fp64, 1e-10 if fp64 else 1e-6, -1))
    return out


def initial_bases(n: int, r: int, seed: int) -> LowRankRHS:
    """Seeded initial guesses U_0, V_0 (n x r, standard normal entries, U drawn
    before V) for Cross-DEIM on a matrix given by its entries (the test matrices
    of Sec. 4.1); s is all ones.  The method orthonormalises them itself."""
    rng = np.random.default_rng(seed)
    U = np.asfortranarray(rng.standard_normal((n, r)))
    V = np.asfortranarray(rng.standard_normal((n, r)))
    return LowRankRHS(n, U, np.ones(r), V)


def paper_gaussian_rhs(n: int) -> LowRankRHS:
    """The right-hand side of the paper's Poisson experiment (Sec. 4.2), read as
    the Gaussian exp(-36((x-0.1)^2 + (y-0.55)^2)) on [-1, 1]^2 (the printed
    exponent has a sign error that makes it grow without bound), mapped to this
    grid's unit square by x = 2x' - 1: exp(-144((x'-0.55)^2 + (y'-0.775)^2)),
    one separable term (rank 1)."""
    x = grid(n)
    U = np.asfortranarray(np.exp(-144.0 * (x - 0.55) ** 2)[:, None])
    V = np.asfortranarray(np.exp(-144.0 * (x - 0.775) ** 2)[:, None])
    return LowRankRHS(n, U, np.ones(1), V)
