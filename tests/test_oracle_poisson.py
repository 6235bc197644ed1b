"""Pins for oracle/poisson.py: closed forms, textbook routines, brute force."""
import numpy as np
import pytest

import lrp_inputs as li
from oracle import cross_deim as cd
from oracle import poisson as po


@pytest.mark.parametrize("n", [1, 3, 7, 64, 255, 1023])
def test_dst1_matches_direct_sine_sum(n):
    # Sec. 3: z_k(i) = sqrt(2/(n+1)) sin(i k pi/(n+1)); scipy's fast DST vs the O(n^2) sum.
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, 3))
    # brute-force sum written element by element (independent of dst_matrix)
    ref = np.zeros_like(X)
    i = np.arange(1, n + 1)
    for k in range(1, n + 1):
        ref[k - 1] = np.sqrt(2.0 / (n + 1)) * np.sum(np.sin(np.pi * i * k / (n + 1))[:, None] * X, axis=0)
    assert np.allclose(po.dst1(X), ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))
    assert np.allclose(po.dst1_direct(X), ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))


@pytest.mark.parametrize("n", [3, 255, 4095])
def test_dst1_self_inverse(n):
    # Sec. 3.2: the DST normalised so that DST(DST(I)) = I.
    rng = np.random.default_rng(1)
    X = rng.standard_normal((n, 4))
    assert np.abs(po.dst1(po.dst1(X)) - X).max() < 1e-13 * np.sqrt(n)
    if n <= 255:
        Z = po.dst_matrix(n)
        assert np.abs(Z - Z.T).max() == 0.0
        assert np.abs(Z @ Z - np.eye(n)).max() < 1e-13


@pytest.mark.parametrize("n,p", [(7, 3), (255, 17), (4095, 64)])
def test_dst_of_eigenfunction_is_scaled_unit_vector(n, p):
    # Z sin(p pi x) = sqrt((n+1)/2) e_p (orthogonality of the sine basis).
    x = li.grid(n)
    y = po.dst1(np.sin(np.pi * p * x)[:, None])[:, 0]
    e = np.zeros(n)
    e[p - 1] = np.sqrt((n + 1) / 2.0)
    assert np.abs(y - e).max() < 1e-12 * np.sqrt(n)


@pytest.mark.parametrize("n", [1, 2, 5, 64, 200])
def test_eigenvalues_match_eigh(n):
    # Textbook routine: eigenvalues of the dense tridiagonal T.
    w = np.linalg.eigvalsh(po.tridiag(n))
    assert np.abs(np.sort(po.eigenvalues(n)) - w).max() < 1e-13


def test_eigenpairs_residual():
    n = 63
    T = po.tridiag(n)
    Z = po.dst_matrix(n)
    lam = po.eigenvalues(n)
    assert np.abs(T @ Z - Z * lam[None, :]).max() < 1e-13


def test_eigenvalue_forms_agree_and_small_k_series():
    # Half-angle identity with the printed form; and the Taylor series at large n
    # where the printed 2(1-cos) form cancels: lambda ~ t^2 - t^4/12, t = pi k/(n+1).
    n = 1023
    assert np.abs(po.eigenvalues(n) - po.eigenvalues_printed(n)).max() < 1e-14
    n = (1 << 20) - 1
    lam = po.eigenvalues(n)
    k = np.arange(1, 6)
    t = np.pi * k / (n + 1)
    series = t ** 2 - t ** 4 / 12.0 + t ** 6 / 360.0
    assert np.abs(lam[:5] / series - 1).max() < 1e-14


@pytest.mark.parametrize("n", [3, 7, 15, 31])
def test_full_grid_solve_matches_kronecker_lu(n):
    rng = np.random.default_rng(n)
    F = rng.standard_normal((n, n))
    W = po.full_grid_solve(F)
    Wk = po.kron_solve(F)
    assert np.abs(W - Wk).max() < 1e-13 * np.abs(Wk).max()


@pytest.mark.parametrize("n", [255, 1023])
def test_full_grid_solve_5pt_residual(n):
    rhs = li.gaussian_eigen_rhs(n, 3, 4, 2)
    F = rhs.dense()
    W = po.full_grid_solve(F)
    h = 1.0 / (n + 1)
    res = po.residual_5pt(W, F)
    # backward-error form: rounding in W (~eps ||W||) is amplified by ||T|| <= 4
    # in each term, while ||h^2 F|| ~ ||W|| / (n+1)^2 is far smaller.
    eps = np.finfo(float).eps
    assert np.linalg.norm(res) < 50 * eps * (8 * np.linalg.norm(W) + np.linalg.norm(h * h * F))


@pytest.mark.parametrize("n,p,q", [(31, 2, 5), (255, 7, 64), (4095, 1, 33)])
def test_eigenfunction_rhs_exact_rank_one_solution(n, p, q):
    # W = a h^2 / (lambda_p + lambda_q) sin(p pi x) sin(q pi y) solves T W + W T = h^2 F.
    a = -1.7
    rhs = li.eigenfunction_rhs(n, p, q, a)
    G = po.SpectralSolution(rhs.U, rhs.s, rhs.V)
    h = 1.0 / (n + 1)
    lp = 4 * np.sin(np.pi * p / (2 * (n + 1))) ** 2
    lq = 4 * np.sin(np.pi * q / (2 * (n + 1))) ** 2
    coef = a * h * h / (lp + lq)
    # exact spectral solution: coef * (n+1)/2 at (p, q), zero elsewhere
    col = G.cols([q - 1])[:, 0]
    e = np.zeros(n)
    e[p - 1] = coef * (n + 1) / 2.0
    assert np.abs(col - e).max() < 1e-12 * abs(e[p - 1])
    x = li.grid(n)
    U = np.sin(np.pi * p * x)[:, None]
    V = np.sin(np.pi * q * x)[:, None]
    assert po.rel_error_vs_exact(U, np.array([coef]), V, G) < 1e-12


def test_spectral_entries_match_full_grid_transform():
    n = 127
    rhs = li.gaussian_eigen_rhs(n, 5, 3, 1)
    G = po.SpectralSolution(rhs.U, rhs.s, rhs.V)
    W = po.full_grid_solve(rhs.dense())
    Wh = po.dst1(po.dst1(W).T).T
    assert np.abs(G.dense() - Wh).max() < 1e-13 * np.abs(Wh).max()
    J = [0, 5, 126]
    assert np.abs(G.cols(J) - Wh[:, J]).max() < 1e-13 * np.abs(Wh).max()
    assert np.abs(G.rows(J) - Wh[J, :]).max() < 1e-13 * np.abs(Wh).max()


def test_error_measures_against_dense():
    n = 63
    rng = np.random.default_rng(0)
    U1, V1 = rng.standard_normal((n, 3)), rng.standard_normal((n, 3))
    U2, V2 = U1 + 1e-9 * rng.standard_normal((n, 3)), V1.copy()
    S1, S2 = np.array([3.0, 2.0, 1.0]), np.array([3.0, 2.0, 1.0 + 1e-11])
    A = (U1 * S1) @ V1.T
    B = (U2 * S2) @ V2.T
    ref = np.linalg.norm(A - B) / np.linalg.norm(B)
    got = po.lowrank_rel_diff(U1, S1, V1, U2, S2, V2)
    assert abs(got - ref) < 1e-6 * ref
    rhs = li.gaussian_eigen_rhs(n, 1, 2)
    G = po.SpectralSolution(rhs.U, rhs.s, rhs.V)
    W = po.full_grid_solve(rhs.dense())
    Uw, Sw, Vtw = np.linalg.svd(W)
    err = po.rel_error_vs_exact(Uw[:, :2], Sw[:2], Vtw[:2].T, G)
    ref = np.linalg.norm(W - (Uw[:, :2] * Sw[:2]) @ Vtw[:2]) / np.linalg.norm(W)
    assert abs(err - ref) < 1e-10 * max(ref, 1e-300) + 1e-15


def test_sampled_error_exact_when_all_rows_low():
    rhs = li.gaussian_eigen_rhs(255, 3, 4)
    U, S, V, info, G = cd.poisson_solve(rhs.U, rhs.s, rhs.V, 1e-4, 8)
    exact = po.rel_error_vs_exact(U, S, V, G)
    est, se = po.rel_error_sampled(U, S, V, G, n_low=255)
    assert se == 0.0
    assert abs(est - exact) <= 1e-12 * exact


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_sampled_error_within_standard_errors(seed):
    # Narrow Gaussians (the large-grid recipe) on n = 4095, a loose solve so the
    # error sits well above rounding: the stratified estimate from 16 exact
    # rows + 32 rows per geometric stratum lands within four of its standard
    # errors of the exact full sum, and that standard error is below 0.1%.
    rhs = li.gaussian_eigen_rhs(4095, seed, 8, 0, s_lo=0.005, s_hi=0.05)
    U, S, V, info, G = cd.poisson_solve(rhs.U, rhs.s, rhs.V, 1e-3, 24)
    exact = po.rel_error_vs_exact(U, S, V, G)
    est, se = po.rel_error_sampled(U, S, V, G, n_low=16, per_stratum=32, seed=seed)
    assert abs(est - exact) <= 4 * se + 1e-9 * exact, (est, se, exact)
    assert se < 1e-3 * exact
