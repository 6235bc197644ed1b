"""The bench workload in the launch configuration the bench times: 1024 seeded
n = 4095 problems (rank-20 right-hand sides, tol 1e-8, rank cap 64, index-set
capacity 64) as 4 concurrent lanes of 256, mixed precision with one refinement
step.  Sixteen problems spread over the batch are checked against the oracle's
exact discrete solution (Eq. g_for_p, evaluated spectrally) within the 1e-6
relative error of the solves/s metric; every problem returns a result status
and a rank within the cap."""
import numpy as np
import pytest

import lrp_inputs as li
from oracle import poisson as po

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bench_configuration_sampled_against_oracle():
    import paper_2607_06021_gb300 as lrp
    from tests.gpu_util import rhs_dev, to_np
    B, n, tol, r_max = 1024, 4095, 1e-8, 64
    rhss = [li.workload_n4095(seed=sd) for sd in range(B)]
    grp = lrp.Group(n, tol, r_max, lanes=4, precision="mixed", batch=B, max_rhs_rank=20, m_cap=64)
    res = grp.solve_batch([rhs_dev(r) for r in rhss])
    grp.close()
    statuses = {info["status"] for *_, info in res}
    assert statuses <= {0, 5, 6}, statuses  # LRP_OK, LRP_NOT_CONVERGED, LRP_RANK_CAPPED
    assert all(1 <= info["rank"] <= r_max for *_, info in res)
    picks = sorted({int(b) for b in np.linspace(0, B - 1, 16)})
    errs = []
    for b in picks:
        U, S, V, _ = res[b]
        G = po.SpectralSolution(rhss[b].U, rhss[b].s, rhss[b].V)
        errs.append(po.rel_error_vs_exact(to_np(U), to_np(S), to_np(V), G))
    assert max(errs) <= 1e-6, list(zip(picks, errs))
