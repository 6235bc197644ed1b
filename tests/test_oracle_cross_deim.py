"""Pins for oracle/cross_deim.py: published generator values, brute force,
exact cross-approximation identities, closed-form solutions."""
import numpy as np
import pytest
import scipy.linalg

import lrp_inputs as li
from oracle import cross_deim as cd
from oracle import poisson as po


def test_splitmix64_published_first_outputs():
    # SplitMix64 seeded with 0: the first output of the reference generator is
    # 0xe220a8397b1dcdaf; with state += golden gamma each call the second is
    # 0x6e789e6aa1b965f4.
    assert cd.splitmix64(0) == 0xE220A8397B1DCDAF
    assert cd.splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4


def test_growth_index_probes_to_complement():
    n = 10
    i0 = cd.splitmix64(7 + 2 * 3 + 1) % n
    present = [(i0 + d) % n for d in range(4)]
    g = cd.growth_index(7, 3, 1, n, present)
    assert g == (i0 + 4) % n and g not in present
    assert cd.growth_index(7, 3, 1, 3, [0, 1, 2]) == -1


def test_leverage_scores_sum_to_one_and_topc_bruteforce():
    rng = np.random.default_rng(0)
    U, _ = np.linalg.qr(rng.standard_normal((50, 6)))
    pi = cd.leverage_scores(U)
    assert abs(pi.sum() - 1.0) < 1e-14
    # brute force: repeatedly take the max, lowest index first on ties
    U[7] = U[3]  # planted tie between rows 3 and 7
    pi = cd.leverage_scores(U)
    left = list(range(50))
    ref = []
    for _ in range(6):
        best = max(left, key=lambda i: (pi[i], -i))
        ref.append(best)
        left.remove(best)
    assert list(cd.select_leverage(U)) == ref
    assert ref.index(3) < ref.index(7) if 7 in ref else True


def _greedy_column_pivots(A, c):
    """Businger-Golub pivoting by explicit Gram-Schmidt downdates (brute force)."""
    A = A.copy()
    piv = []
    for _ in range(c):
        norms = np.sum(A * A, axis=0)
        norms[piv] = -1
        j = int(np.argmax(norms))
        piv.append(j)
        q = A[:, j] / np.linalg.norm(A[:, j])
        A = A - np.outer(q, q @ A)
    return piv


def test_qdeim_matches_greedy_pivoting():
    rng = np.random.default_rng(3)
    U, _ = np.linalg.qr(rng.standard_normal((40, 5)) * np.array([5, 3, 2, 1, 0.5]))
    assert list(cd.select_qdeim(U)) == _greedy_column_pivots(U.T, 5)


def test_deim_selects_independent_rows():
    rng = np.random.default_rng(4)
    U, _ = np.linalg.qr(rng.standard_normal((30, 4)))
    idx = cd.select_deim(U)
    assert len(set(idx.tolist())) == 4
    assert np.linalg.matrix_rank(U[idx]) == 4


class DenseG:
    def __init__(self, A):
        self.A = A
        self.shape = A.shape

    def cols(self, J):
        return self.A[:, np.asarray(J)]

    def rows(self, I):
        return self.A[np.asarray(I), :]


def test_scross_exact_for_low_rank_both_branches():
    # Cross approximation theorem: rank(G(I,J)) = rank(G) => C G(I,J)^+ R = G.
    rng = np.random.default_rng(5)
    A = rng.standard_normal((60, 5)) @ rng.standard_normal((5, 45))
    G = DenseG(A)
    I = rng.choice(60, 9, replace=False)
    J = rng.choice(45, 7, replace=False)
    for (II, JJ) in [(I, J), (I[:6], J)]:   # |J| <= |I| and |J| > |I|
        r = cd.scross(G, II, JJ, None)
        approx = (r.U * r.S) @ r.V.T
        assert np.abs(approx - A).max() < 1e-12 * np.abs(A).max()
        assert r.S.shape[0] == 5
    # both branches give the same approximation on a full-rank matrix
    B = rng.standard_normal((30, 30))
    GB = DenseG(B)
    I, J = np.arange(12), np.arange(12)
    r1 = cd.scross(GB, I, J[:11], None)
    r2 = cd.scross(GB, I[:11], J, None)
    C = B[:, J[:11]]
    ref = C @ np.linalg.pinv(B[np.ix_(I, J[:11])]) @ B[I, :]
    assert np.abs((r1.U * r1.S) @ r1.V.T - ref).max() < 1e-10 * np.abs(ref).max()
    C = B[:, J]
    ref2 = C @ np.linalg.pinv(B[np.ix_(I[:11], J)]) @ B[I[:11], :]
    assert np.abs((r2.U * r2.S) @ r2.V.T - ref2).max() < 1e-10 * np.abs(ref2).max()


def test_scross_all_indices_is_truncated_svd():
    # I = J = all rows/cols: the cross approximation is G itself and scross
    # returns its SVD (numpy.linalg.svd on the dense matrix).
    n = 47
    rhs = li.gaussian_eigen_rhs(n, 2, 3)
    G = po.SpectralSolution(rhs.U, rhs.s, rhs.V)
    r = cd.scross(G, np.arange(n), np.arange(n), None)
    s_ref = np.linalg.svd(G.dense(), compute_uv=False)
    k = r.S.shape[0]
    assert np.abs(r.S - s_ref[:k]).max() < 1e-12 * s_ref[0]
    assert np.abs((r.U * r.S) @ r.V.T - G.dense()).max() < 1e-12 * s_ref[0]


def test_scross_redundancy_diagonal_flags_duplicate_column():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((40, 4)) @ rng.standard_normal((4, 40))
    G = DenseG(A)
    I = np.array([0, 1, 2, 3, 4])
    J = np.array([5, 6, 7, 8, 5])   # column 5 twice: the repeat is dependent
    r = cd.scross(G, I, J, None)
    aC = np.abs(r.rC)
    assert aC[4] < 1e-12 * aC.max()
    assert np.all(aC[:4] > 1e-6 * aC.max())


def test_tail_rank_bruteforce():
    rng = np.random.default_rng(7)
    for _ in range(50):
        s = np.sort(np.abs(rng.standard_normal(12)) * 10.0 ** rng.uniform(-12, 0, 12))[::-1]
        tol = 10.0 ** rng.uniform(-10, -1)
        total = np.sum(s ** 2)
        ref = next(r for r in range(13) if np.sum(s[r:] ** 2) < tol * tol * total)
        assert cd.tail_rank(s, tol) == max(ref, 1)


def test_cross_deim_eigenfunction_rhs_rank_one():
    n, p, q = 255, 9, 40
    rhs = li.eigenfunction_rhs(n, p, q, 2.5)
    U, S, V, info, G = cd.poisson_solve(rhs.U, rhs.s, rhs.V, 1e-12, 8)
    assert S.shape[0] == 1
    assert po.rel_error_vs_exact(U, S, V, G) < 1e-12
    assert p - 1 in info.I and q - 1 in info.J


@pytest.mark.parametrize("selector", ["ls", "qdeim"])
def test_cross_deim_small_grid_within_tolerance(selector):
    # Brute force on a small grid: the full-grid DST solve is the exact answer.
    n = 63
    rhs = li.gaussian_eigen_rhs(n, 11, 3)
    tol = 1e-8
    U, S, V, info, G = cd.poisson_solve(rhs.U, rhs.s, rhs.V, tol, 40, selector=selector)
    W = po.full_grid_solve(rhs.dense())
    err = np.linalg.norm((U * S) @ V.T - W) / np.linalg.norm(W)
    assert err < 10 * tol
    s_ex = np.linalg.svd(W, compute_uv=False)
    # the returned rank is no larger than the exact tail-rule rank plus the safeguard slack
    assert S.shape[0] <= cd.tail_rank(s_ex, tol / 10)


def test_cross_deim_workload_n255_reaches_tolerance():
    rhs = li.workload_single_small(0)
    U, S, V, info, G = cd.poisson_solve(rhs.U, rhs.s, rhs.V, 1e-10, 32, m_cap=2 * 32 + 4)
    assert info.converged
    assert po.rel_error_vs_exact(U, S, V, G) < 1e-9
    assert np.all(np.diff(S) <= 0)
    # orthonormal factors
    assert np.abs(U.T @ U - np.eye(S.shape[0])).max() < 1e-12


def test_rank_cap_and_floor():
    rhs = li.workload_single_small(1)
    U, S, V, info, G = cd.poisson_solve(rhs.U, rhs.s, rhs.V, 1e-10, 5)
    assert S.shape[0] == 5 and info.rank_capped
    U, S, V, info, G = cd.poisson_solve(rhs.U, rhs.s, rhs.V, 10.0, 5)
    assert S.shape[0] == 1


def test_planted_sign_error_is_caught():
    # A plausible mistake (a sign flip in the Cauchy denominator) must break the
    # exactness check on the eigenfunction right-hand side.
    n, p, q = 63, 3, 5
    rhs = li.eigenfunction_rhs(n, p, q)
    G = po.SpectralSolution(rhs.U, rhs.s, rhs.V)
    good = G.cols([q - 1])
    G.lam = -G.lam[::-1].copy()
    bad = G.cols([q - 1])
    assert np.abs(good - bad).max() > 1e-3 * np.abs(good).max()


@pytest.mark.parametrize("seed", [0, 1])
def test_warm_resolve_of_perturbed_rhs(seed):
    # Warm start (Sec. 5, repeated solves): index sets and the last iterate of a
    # solve seed the re-solve of a nearby right-hand side.  The first iteration's
    # change is measured from zero (rho_0 = 1), so at least two iterations run;
    # a 1% amplitude change converges in fewer iterations than a cold re-solve
    # (2 and 10 against 10 and 29 with leverage sampling), to the same accuracy.
    import lrp_inputs as li
    from oracle import poisson as po
    rhs = li.workload_single_small(seed)
    tol, r_max, m_cap = 1e-10, 32, 68
    _, _, _, info, _ = cd.poisson_solve(rhs.U, rhs.s, rhs.V, tol, r_max, seed=seed, m_cap=m_cap)
    r2 = li.perturb_amplitudes(rhs, 100 + seed)
    Uc, Sc, Vc, ic, G = cd.poisson_solve(r2.U, r2.s, r2.V, tol, r_max, seed=seed, m_cap=m_cap)
    Uw, Sw, Vw, iw, _ = cd.poisson_solve(r2.U, r2.s, r2.V, tol, r_max, seed=seed, m_cap=m_cap,
                                         warm=(info.I, info.J, info.last))
    assert iw.rho[0] == 1.0
    assert 2 <= iw.iterations < ic.iterations
    err_c = po.rel_error_vs_exact(Uc, Sc, Vc, G)
    err_w = po.rel_error_vs_exact(Uw, Sw, Vw, G)
    assert err_w < max(10 * tol, 1.01 * err_c)


def test_philox4x32_10_published_known_answers():
    # Known-answer vectors of Philox4x32-10 published with the generator
    # (Salmon et al., SC 2011; the Random123 distribution's test vectors).
    kat = [((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
           ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
           ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
            (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1))]
    for ctr, key, want in kat:
        got = tuple(int(v) for v in cd.philox4x32_10(ctr, key))
        assert got == want, [hex(v) for v in got]


def test_philox_uniform_range_and_moments():
    u = cd.philox_uniform(7, 3, 1, np.arange(200000))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / u.size)
    assert abs(u.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / u.size)
    # distinct counters give distinct draws: no row repeats another's value
    assert np.unique(u).size == u.size


def test_bernoulli_leverage_inclusion_frequencies():
    # Algorithm LeverageScores samples row i with probability min(1, c pi_i):
    # over many keys the inclusion frequency of each row is that probability.
    rng = np.random.default_rng(5)
    n, c = 120, 4
    U = np.linalg.qr(rng.standard_normal((n, c)) * np.geomspace(0.01, 10.0, n)[:, None])[0]
    factor = 3.0
    p = np.minimum(1.0, factor * np.sum(U * U, axis=1))
    assert (p == 1.0).any() and (p < 0.05).any()
    T = 3000
    hits = np.zeros(n)
    sizes = []
    for key in range(T):
        rows = cd.select_bernoulli(U, key, 2, 0, factor)
        hits[rows] += 1
        sizes.append(rows.size)
        # sampled rows come in descending score, ties to the lower index
        sc = np.sum(U[rows] ** 2, axis=1)
        assert np.all(np.diff(sc) <= 0)
    freq = hits / T
    sd = np.sqrt(np.maximum(p * (1 - p), 1e-12) / T)
    assert np.all(np.abs(freq - p) <= 5 * sd + 1e-12), np.max(np.abs(freq - p) / (sd + 1e-12))
    assert np.all(freq[p == 1.0] == 1.0)
    assert abs(np.mean(sizes) - p.sum()) < 5 * np.sqrt(np.sum(p * (1 - p)) / T)
    # expected sample size is at most c = factor x columns
    assert p.sum() <= factor * c + 1e-12


def test_bernoulli_cross_deim_small_grid_within_tolerance():
    n = 63
    rhs = li.gaussian_eigen_rhs(n, 11, 3)
    tol = 1e-8
    U, S, V, info, G = cd.poisson_solve(rhs.U, rhs.s, rhs.V, tol, 40, selector="bernoulli", seed=3)
    W = po.full_grid_solve(rhs.dense())
    err = np.linalg.norm((U * S) @ V.T - W) / np.linalg.norm(W)
    assert err < 10 * tol


def test_inv_smin_is_inverse_smallest_singular_value():
    # A matrix with known singular values 4, 2, 0.5 (orthogonal factors from a
    # seeded QR): ||M^+||_2 = 1 / 0.5.  Reading eta as 1/sigma_max (the literal
    # ||(I(:,I_k))^T U_k||_2^{-1}) would give 0.25 and fail here.
    rng = np.random.default_rng(11)
    Qa, _ = np.linalg.qr(rng.standard_normal((7, 3)))
    Qb, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    M = (Qa * np.array([4.0, 2.0, 0.5])) @ Qb.T
    assert abs(cd.inv_smin(M) - 2.0) < 1e-13
    # invariant: M^+ M = I for full column rank, and ||M^+||_2 bounds ||M^+ x|| / ||x||
    x = rng.standard_normal(7)
    assert np.linalg.norm(np.linalg.pinv(M) @ x) <= cd.inv_smin(M) * np.linalg.norm(x) * (1 + 1e-13)
    # a rank-deficient square matrix has no finite bound
    assert cd.inv_smin(np.diag([1.0, 0.0])) == float("inf")


def test_diff_norm_against_dense_difference():
    # ||U_a S_a V_a^T - U_b S_b V_b^T||_F from the stacked-factor QR equals the
    # norm of the explicitly formed difference; with B = None it is ||S_a||_F.
    rng = np.random.default_rng(12)
    Ua, _ = np.linalg.qr(rng.standard_normal((40, 4)))
    Va, _ = np.linalg.qr(rng.standard_normal((30, 4)))
    Ub, _ = np.linalg.qr(rng.standard_normal((40, 3)))
    Vb, _ = np.linalg.qr(rng.standard_normal((30, 3)))
    Sa, Sb = np.array([3.0, 1.0, 0.2, 0.01]), np.array([2.0, 0.7, 0.1])
    dense = np.linalg.norm((Ua * Sa) @ Va.T - (Ub * Sb) @ Vb.T)
    assert abs(cd.diff_norm((Ua, Sa, Va), (Ub, Sb, Vb)) - dense) < 1e-13 * dense
    assert abs(cd.diff_norm((Ua, Sa, Va), None) - np.linalg.norm(Sa)) < 1e-15
    # a nearly equal pair: the small difference keeps its relative accuracy
    # (the dense difference of two O(1) matrices loses ~1e-16 absolute only)
    Sc = Sa * (1 + 1e-9 * np.arange(1, 5))
    small = np.linalg.norm((Ua * (Sa - Sc)) @ Va.T)
    assert abs(cd.diff_norm((Ua, Sa, Va), (Ua, Sc, Va)) - small) < 1e-6 * small


def test_orth_keeps_the_numerical_range():
    # A column equal to another (two equal right-hand-side terms) has a zero
    # Householder pivot up to rounding: it is dropped.  A column that is merely
    # close (pivot 1e-6 relative) is kept.  Full-rank input: the plain Q.
    rng = np.random.default_rng(21)
    X = rng.standard_normal((50, 4))
    Q = cd.orth(X)
    assert Q.shape == (50, 4) and np.allclose(np.abs(Q.T @ X), np.abs(np.linalg.qr(X)[0].T @ X))
    Xd = np.concatenate([X, X[:, 1:2]], axis=1)
    Qd = cd.orth(Xd)
    assert Qd.shape == (50, 4)
    assert np.linalg.norm(Xd - Qd @ (Qd.T @ Xd)) < 1e-13 * np.linalg.norm(Xd)  # the range is kept
    Xc = np.concatenate([X, X[:, 1:2] + 1e-6 * rng.standard_normal((50, 1))], axis=1)
    assert cd.orth(Xc).shape == (50, 5)
    assert cd.orth(np.zeros((5, 2))).shape == (5, 1)
