"""QDEIM index selection on the GPU (Algorithm IS, Sec. 2.2.1; the paper's
comparison selector): the same pivots as the oracle's column-pivoted QR of U^T,
iteration by iteration, and the same solution."""
import pytest

import lrp_inputs as li
from oracle import cross_deim as cd
from oracle import poisson as po

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _gpu(rhs, tol, r_max, m_cap, seed, precision="fp64"):
    import paper_2607_06021_gb300 as lrp
    from tests.gpu_util import rhs_dev, to_np
    plan = lrp.Plan(rhs.n, tol, r_max, max_rhs_rank=rhs.rank, m_cap=m_cap, seed=seed, selector="qdeim",
                    precision=precision)
    plan.set_trace(True)
    U, S, V, info = plan.solve(*rhs_dev(rhs))
    tr = plan.trace(0)
    plan.close()
    return to_np(U), to_np(S), to_np(V), info, tr


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_qdeim_fp64_matches_oracle(seed):
    rhs = li.workload_single_small(seed)
    tol, r_max, m_cap = 1e-10, 32, 68
    U, S, V, info, tr = _gpu(rhs, tol, r_max, m_cap, seed)
    Uo, So, Vo, oinfo, G = cd.poisson_solve(rhs.U, rhs.s, rhs.V, tol, r_max, seed=seed, m_cap=m_cap,
                                            selector="qdeim")
    assert info["iterations"] == oinfo.iterations, (info, oinfo.iterations)
    for k, row in enumerate(tr):
        assert (row["size_I"], row["size_J"]) == tuple(oinfo.sizes[k]), (k, row, oinfo.sizes[k])
    assert po.lowrank_rel_diff(U, S, V, Uo, So, Vo) <= 1e-10
    assert po.rel_error_vs_exact(U, S, V, G) < 10 * tol


@pytest.mark.parametrize("n", [1, 7, 31, 1023])
def test_qdeim_edge_sizes(n):
    rhs = li.gaussian_eigen_rhs(n, 3, 1 if n < 7 else 4)
    tol, r_max = 1e-10, 16
    U, S, V, info, _ = _gpu(rhs, tol, r_max, 0, 0)
    Uo, So, Vo, oinfo, G = cd.poisson_solve(rhs.U, rhs.s, rhs.V, tol, r_max, m_cap=2 * r_max + rhs.rank,
                                            selector="qdeim")
    assert info["iterations"] == oinfo.iterations
    assert po.lowrank_rel_diff(U, S, V, Uo, So, Vo) <= 1e-10


def test_qdeim_mixed_n4095_accuracy():
    rhs = li.workload_n4095(1)
    U, S, V, info, _ = _gpu(rhs, 1e-8, 64, 64, 0, precision="mixed")
    G = po.SpectralSolution(rhs.U, rhs.s, rhs.V)
    assert po.rel_error_vs_exact(U, S, V, G) <= 1e-6, info
