"""Mixed grid sizes in one launch (lrp_multi_*): a batch of problems of several
n is solved as one CUDA graph launch whose per-size branches run their
Cross-DEIM loops on the device.  Each problem's result equals the solve of the
same problem by a plan of its size alone, bit for bit (no workspace is shared
between branches, and the per-problem arithmetic does not depend on the batch);
a second call with other problems of the same sizes reuses the captured graph."""
import numpy as np
import pytest

import lrp_inputs as li

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _np(res):
    from tests.gpu_util import to_np
    return [(to_np(U), to_np(S), to_np(V), info) for U, S, V, info in res]


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_multi_size_one_launch_equals_standalone(precision):
    import paper_2607_06021_gb300 as lrp
    from tests.gpu_util import rhs_dev
    sizes = (511, 1023, 2047, 4095)
    tol, r_max, rf_cap = (1e-6, 64, 24) if precision == "mixed" else (1e-8, 48, 24)
    m_cap = 64
    rhss = li.batch_mixed_sizes(20, seed=5, sizes=sizes, rank_lo=2, rank_hi=rf_cap)
    counts = [sum(1 for r in rhss if r.n == n) for n in sizes]
    multi = lrp.Multi(sizes, [max(c, 1) for c in counts], tol, r_max, precision=precision, max_rhs_rank=rf_cap,
                      m_cap=m_cap)  # refine_steps = 2 (the default) in mixed precision
    got = _np(multi.solve_batch([rhs_dev(r) for r in rhss]))
    # a second call: the same sizes, other problems (reversed order), same graph
    got2 = _np(multi.solve_batch([rhs_dev(r) for r in rhss[::-1]]))
    multi.close()
    for rhs, (U, S, V, info), (U2, S2, V2, info2) in zip(rhss, got, got2[::-1]):
        plan = lrp.Plan(rhs.n, tol, r_max, precision=precision, max_rhs_rank=rf_cap, m_cap=m_cap)
        (Ua, Sa, Va, ia), = _np([plan.solve(*rhs_dev(rhs))])
        plan.close()
        assert info == ia == info2
        for a, b, c in ((U, Ua, U2), (S, Sa, S2), (V, Va, V2)):
            assert np.array_equal(a, b) and np.array_equal(a, c)


def test_multi_rejects_sizes_outside_the_set():
    import paper_2607_06021_gb300 as lrp
    from tests.gpu_util import rhs_dev
    multi = lrp.Multi((255, 511), [2, 2], 1e-6, 32, max_rhs_rank=8, m_cap=48)
    rhs = li.gaussian_eigen_rhs(1023, 1, 3)
    with pytest.raises(lrp.LrpError) as e:
        multi.solve_batch([rhs_dev(rhs)])
    assert e.value.status == lrp.LRP_EINVAL
    multi.close()
