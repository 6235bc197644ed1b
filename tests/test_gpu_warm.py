"""Warm start on the GPU (Sec. 5, repeated solves): a solve stores its index
sets and last iterate in a warm record; the re-solve of a perturbed right-hand
side starts from them.  Parity against the oracle's warm re-solve on the same
record contents (the two sides' cold solves agree index for index)."""
import numpy as np
import pytest

import lrp_inputs as li
from oracle import cross_deim as cd
from oracle import poisson as po

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cases():
    return [(li.workload_single_small, 0, 1e-10, 32, 68), (li.workload_single_small, 1, 1e-10, 32, 68),
            (li.workload_n4095, 1, 1e-8, 64, 148)]


@pytest.mark.parametrize("case", range(3))
@pytest.mark.parametrize("precision", ["fp64"])
def test_warm_resolve_matches_oracle(case, precision):
    import paper_2607_06021_gb300 as lrp
    from tests.gpu_util import rhs_dev, to_np
    mk, seed, tol, r_max, m_cap = _cases()[case]
    rhs = mk(seed)
    r2 = li.perturb_amplitudes(rhs, 100 + seed)
    plan = lrp.Plan(rhs.n, tol, r_max, max_rhs_rank=rhs.rank, m_cap=m_cap, seed=seed, precision=precision)
    warm = plan.warm_record()
    _, _, _, info0 = plan.solve(*rhs_dev(rhs), warm=warm)
    U, S, V, info = plan.solve(*rhs_dev(r2), warm=warm)
    U, S, V = to_np(U), to_np(S), to_np(V)
    Uc, Sc, Vc, infoc = plan.solve(*rhs_dev(r2))  # cold: the record is not touched
    warm.close()
    plan.close()
    _, _, _, o0, _ = cd.poisson_solve(rhs.U, rhs.s, rhs.V, tol, r_max, seed=seed, m_cap=m_cap)
    Uo, So, Vo, ow, G = cd.poisson_solve(r2.U, r2.s, r2.V, tol, r_max, seed=seed, m_cap=m_cap,
                                         warm=(o0.I, o0.J, o0.last))
    assert info0["iterations"] == o0.iterations
    assert info["iterations"] == ow.iterations, (info, ow.iterations, ow.rho)
    assert info["iterations"] <= infoc["iterations"] + 1
    diff = po.lowrank_rel_diff(U, S, V, Uo, So, Vo)
    assert diff < 10 * tol, (diff, info)
    assert po.rel_error_vs_exact(U, S, V, G) < 10 * tol


def test_warm_reset_gives_cold_solve():
    import paper_2607_06021_gb300 as lrp
    from tests.gpu_util import rhs_dev, to_np
    rhs = li.workload_single_small(2)
    plan = lrp.Plan(rhs.n, 1e-10, 32, max_rhs_rank=rhs.rank, m_cap=68, seed=2)
    warm = plan.warm_record()
    plan.solve(*rhs_dev(rhs), warm=warm)
    warm.reset()
    U, S, V, info = plan.solve(*rhs_dev(rhs), warm=warm)
    Uc, Sc, Vc, infoc = plan.solve(*rhs_dev(rhs))
    assert info["iterations"] == infoc["iterations"]
    assert po.lowrank_rel_diff(to_np(U), to_np(S), to_np(V), to_np(Uc), to_np(Sc), to_np(Vc)) < 1e-13
    warm.close()
    plan.close()


def test_warm_mixed_precision_resolve():
    # Mixed precision: the record is written by the FP32 first solve and seeds the
    # FP32 first solve of the next call; the result keeps the refined accuracy.
    import paper_2607_06021_gb300 as lrp
    from tests.gpu_util import rhs_dev, to_np
    rhs = li.workload_n4095(0)
    r2 = li.perturb_amplitudes(rhs, 7)
    tol = 1e-8
    plan = lrp.Plan(rhs.n, tol, 64, max_rhs_rank=rhs.rank, m_cap=64, precision="mixed")
    warm = plan.warm_record()
    plan.solve(*rhs_dev(rhs), warm=warm)
    U, S, V, info = plan.solve(*rhs_dev(r2), warm=warm)
    warm.close()
    plan.close()
    G = po.SpectralSolution(r2.U, r2.s, r2.V)
    err = po.rel_error_vs_exact(to_np(U), to_np(S), to_np(V), G)
    assert err < 1e-6, (err, info)
