"""The oracle's Cross-DEIM on the paper's own Poisson right-hand side (Sec. 4.2,
one Gaussian; its garbled exponent read with the sign as +, R14) with the
printed Algorithm LeverageScores (Bernoulli sampling): three growth/draw seeds
at n = 1023 and 4095 stop by the stop test, and the result lies within 10 tol
of the exact solution of Eq. g_for_p (exact sums).  The same right-hand side
is held to the same bar on the GPU (test_gpu_paper_rhs.py)."""
import pytest

import lrp_inputs as li
from oracle import cross_deim as cd
from oracle import poisson as po

TOL = 1e-6


@pytest.mark.parametrize("n", [1023, 4095])
def test_oracle_meets_the_bar_on_the_paper_rhs(n):
    rhs = li.paper_gaussian_rhs(n)
    ranks = set()
    for seed in range(3):
        U, S, V, info, G = cd.poisson_solve(rhs.U, rhs.s, rhs.V, TOL, 64, seed=seed)
        assert info.converged, (n, seed)
        err = po.rel_error_vs_exact(U, S, V, G)
        assert err <= 10 * TOL, (n, seed, err)
        ranks.add(len(S))
    # the rank the tolerance asks for does not depend on the draws
    assert len(ranks) == 1
