"""Bernoulli leverage-score selection (Algorithm LeverageScores as printed,
Sec. 2.2.2): row i is sampled with probability min(1, c pi_i).  The GPU draws
the same Philox4x32-10 numbers as the oracle (counter (row, iteration, side, 0),
key = seed) and takes the same decisions, so the FP64 iteration trace (|I_k|,
|J_k|, in-loop rank, rho) equals the oracle's iteration by iteration; the mixed
path meets the 1e-6 error bar with it."""
import numpy as np
import pytest

import lrp_inputs as li
from oracle import cross_deim as cd
from oracle import poisson as po

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _gpu(rhs, tol, r_max, **kw):
    import paper_2607_06021_gb300 as lrp
    from tests.gpu_util import rhs_dev, to_np
    plan = lrp.Plan(rhs.n, tol, r_max, max_rhs_rank=rhs.rank, selector="bernoulli", **kw)
    plan.set_trace(True)
    U, S, V, info = plan.solve(*rhs_dev(rhs))
    tr = plan.trace(0)
    plan.close()
    return to_np(U), to_np(S), to_np(V), info, tr


@pytest.mark.parametrize("seed,factor", [(0, 1.0), (1, 2.0), (2, 0.5)])
def test_bernoulli_fp64_trace_matches_oracle(seed, factor):
    rhs = li.workload_single_small(seed)
    tol, r_max, m_cap, key = 1e-10, 32, 68, 11 + seed
    U, S, V, info, tr = _gpu(rhs, tol, r_max, m_cap=m_cap, seed=key, sample_factor=factor)
    Uo, So, Vo, oinfo, G = cd.poisson_solve(rhs.U, rhs.s, rhs.V, tol, r_max, selector="bernoulli", seed=key,
                                            m_cap=m_cap, sample_factor=factor)
    assert len(tr) == oinfo.iterations, (len(tr), oinfo.iterations)
    for k, row in enumerate(tr):
        assert (row["size_I"], row["size_J"]) == tuple(oinfo.sizes[k]), (k, row, oinfo.sizes[k])
        assert row["rank"] == oinfo.ranks[k], (k, row)
        assert abs(row["rho"] - oinfo.rho[k]) <= 1e-6 * oinfo.rho[k] + 1e-13, (k, row["rho"], oinfo.rho[k])
    assert po.lowrank_rel_diff(U, S, V, Uo, So, Vo) <= 1e-10
    assert po.rel_error_vs_exact(U, S, V, G) < 1e-9


def test_bernoulli_n4095_fp64_and_mixed():
    rhs = li.workload_n4095(3)
    tol, r_max, m_cap, key = 1e-8, 64, 148, 5
    G = po.SpectralSolution(rhs.U, rhs.s, rhs.V)
    U, S, V, info, tr = _gpu(rhs, tol, r_max, m_cap=m_cap, seed=key, sample_factor=1.5)
    Uo, So, Vo, oinfo, _ = cd.poisson_solve(rhs.U, rhs.s, rhs.V, tol, r_max, selector="bernoulli", seed=key,
                                            m_cap=m_cap, sample_factor=1.5)
    assert info["iterations"] == oinfo.iterations
    assert [(r["size_I"], r["size_J"]) for r in tr] == [tuple(s) for s in oinfo.sizes]
    assert po.rel_error_vs_exact(U, S, V, G) < 10 * tol
    assert po.lowrank_rel_diff(U, S, V, Uo, So, Vo) <= 1e-10
    Um, Sm, Vm, infom, _ = _gpu(rhs, tol, r_max, m_cap=64, seed=key, sample_factor=1.5, precision="mixed")
    assert po.rel_error_vs_exact(Um, Sm, Vm, G) <= 1e-6, infom
