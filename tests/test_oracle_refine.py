"""Pins for oracle/refine.py: the factor form of the residual equals the dense
5-point residual; one refinement step reduces the error by orders of magnitude."""
import numpy as np

import lrp_inputs as li
from oracle import cross_deim as cd
from oracle import poisson as po
from oracle import refine as rf


def test_physical_residual_factors_equal_dense_5pt_residual():
    n = 63
    rhs = li.gaussian_eigen_rhs(n, 1, 3, 1)
    rng = np.random.default_rng(0)
    U0, _ = np.linalg.qr(rng.standard_normal((n, 4)))
    V0, _ = np.linalg.qr(rng.standard_normal((n, 4)))
    S0 = np.array([1.0, 0.5, 0.1, 0.01])
    X, d, Y = rf.physical_residual_factors(rhs.U, rhs.s, rhs.V, U0, S0, V0)
    W0 = (U0 * S0) @ V0.T
    dense = -po.residual_5pt(W0, rhs.dense())
    assert np.abs((X * d) @ Y.T - dense).max() < 1e-13 * np.abs(dense).max()


def test_spectral_residual_is_transform_of_physical():
    n = 63
    rhs = li.gaussian_eigen_rhs(n, 2, 2, 1)
    rng = np.random.default_rng(1)
    U0, V0 = rng.standard_normal((n, 3)), rng.standard_normal((n, 3))
    S0 = np.array([2.0, 1.0, 0.3])
    Xp, dp, Yp = rf.physical_residual_factors(rhs.U, rhs.s, rhs.V, U0, S0, V0)
    Xs, ds, Ys = rf.spectral_residual_factors(po.dst1(rhs.U), rhs.s, po.dst1(rhs.V),
                                              po.dst1(U0), S0, po.dst1(V0))
    Rp = (Xp * dp) @ Yp.T
    Rs = (Xs * ds) @ Ys.T
    Z = po.dst_matrix(n)
    assert np.abs(Z @ Rp @ Z - Rs).max() < 1e-12 * np.abs(Rs).max()


def test_recompress_matches_dense_svd():
    rng = np.random.default_rng(2)
    X, Y = rng.standard_normal((50, 6)), rng.standard_normal((50, 6))
    d = np.array([1, -1, 2, 1e-3, -1e-6, 3.0])
    U, s, V = rf.recompress(X, d, Y, 1e-15)
    ref = np.linalg.svd((X * d) @ Y.T, compute_uv=False)
    assert np.abs(s - ref[:s.shape[0]]).max() < 1e-12 * ref[0]


def test_one_refinement_step_reduces_error():
    rhs = li.workload_single_small(2)
    G = po.SpectralSolution(rhs.U, rhs.s, rhs.V)
    Uh, S, Vh, info = cd.cross_deim(G, cd.orth(G.Uh), cd.orth(G.Vh), 1e-10, 32)
    # trial solution spoiled at the FP32 level (what a single-precision solve leaves)
    rng = np.random.default_rng(3)
    Uh0 = (Uh + 3e-7 * rng.standard_normal(Uh.shape)).astype(np.float32).astype(np.float64)
    Vh0 = (Vh + 3e-7 * rng.standard_normal(Vh.shape)).astype(np.float32).astype(np.float64)
    S0 = S.astype(np.float32).astype(np.float64)
    e0 = po.rel_error_vs_exact(po.dst1(Uh0), S0, po.dst1(Vh0), G)
    U1, S1, V1, _ = rf.refine_once(G, Uh0, S0, Vh0, 1e-10, 32)
    e1 = po.rel_error_vs_exact(po.dst1(U1), S1, po.dst1(V1), G)
    assert e0 > 1e-7
    assert e1 < 1e-9 and e1 < e0 / 100
