"""The bench workload in the launch configuration the bench times: 1024 seeded
n = 4095 problems (rank-20 right-hand sides, tol 1e-8, rank cap 64, index-set
capacity 64) as 4 concurrent lanes of 256, mixed precision with one refinement
step.  Every problem of the batch is checked against the oracle's exact
discrete solution (Eq. g_for_p, evaluated spectrally) within the 1e-6 relative
error of the solves/s metric; every problem returns a result status and a rank
within the cap."""
import numpy as np
import pytest

import lrp_inputs as li

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bench_configuration_every_problem_against_oracle():
    import paper_2607_06021_gb300 as lrp
    from tests.gpu_util import exact_errors_n4095, rhs_dev
    B, n, tol, r_max = 1024, 4095, 1e-8, 64
    rhss = [li.workload_n4095(seed=sd) for sd in range(B)]
    grp = lrp.Group(n, tol, r_max, lanes=4, precision="mixed", batch=B, max_rhs_rank=20, m_cap=64)
    res = grp.solve_batch([rhs_dev(r) for r in rhss])
    grp.close()
    statuses = {info["status"] for *_, info in res}
    assert statuses <= {0, 5, 6}, statuses  # LRP_OK, LRP_NOT_CONVERGED, LRP_RANK_CAPPED
    assert all(1 <= info["rank"] <= r_max for *_, info in res)
    errs = exact_errors_n4095(range(B), [(U, S, V) for U, S, V, _ in res])
    worst = np.argsort(errs)[-5:]
    assert errs.max() <= 1e-6, [(int(b), float(errs[b])) for b in worst]
