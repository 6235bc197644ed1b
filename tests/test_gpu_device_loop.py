"""Device-side iteration loops (lrp_opts.loop_on_device): the whole solve is one
captured CUDA graph whose Cross-DEIM loops are conditional while-nodes.  The
arithmetic is the host-driven loop's, so every output equals it bit for bit;
consecutive solves through one plan reuse the captured graph with new inputs."""
import numpy as np
import pytest

import lrp_inputs as li

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _solve(rhss, n, tol, r_max, rf_cap, device_loop, **kw):
    import paper_2607_06021_gb300 as lrp
    from tests.gpu_util import rhs_dev, to_np
    plan = lrp.Plan(n, tol, r_max, batch=len(rhss), max_rhs_rank=rf_cap, loop_on_device=device_loop, **kw)
    out = []
    for batch in (rhss, rhss[::-1]):  # a second call with the problems in another order
        res = plan.solve_batch([rhs_dev(r) for r in batch])
        out.append([(to_np(U), to_np(S), to_np(V), info) for U, S, V, info in res])
    plan.close()
    return out


def _same(a, b):
    for (U1, S1, V1, i1), (U2, S2, V2, i2) in zip(a, b):
        assert i1 == i2
        assert np.array_equal(S1, S2) and np.array_equal(U1, U2) and np.array_equal(V1, V2)


@pytest.mark.parametrize("precision,n,tol,r_max,steps", [("fp64", 255, 1e-10, 32, 2), ("mixed", 4095, 1e-8, 64, 1),
                                                         ("mixed", 4095, 1e-8, 64, 2), ("fp64", 4095, 1e-8, 64, 2)])
def test_device_loop_equals_host_loop(precision, n, tol, r_max, steps):
    # mixed precision with refine_steps = 2: the second step is a conditional
    # if-node of the graph, a host decision in the host-driven solve
    rhss = [li.gaussian_eigen_rhs(n, 40 + s, 4 + 3 * s, 1 if s % 2 else 0) for s in range(6)]
    kw = dict(precision=precision, m_cap=min(2 * r_max + 24, 64) if precision == "mixed" else 2 * r_max + 24,
              refine_steps=steps)
    host = _solve(rhss, n, tol, r_max, 24, False, **kw)
    dev = _solve(rhss, n, tol, r_max, 24, True, **kw)
    for h, d in zip(host, dev):
        _same(h, d)
    # the second call solved the same problems in reverse order
    _same(host[0], host[1][::-1])


@pytest.mark.parametrize("max_iter", [1, 2, 3])
def test_device_loop_iteration_cap(max_iter):
    # the loop bound: max_iter = 1 captures no loop node; 2 and 3 one and two trips
    rhss = [li.workload_single_small(s) for s in range(3)]
    host = _solve(rhss, 255, 1e-10, 32, 4, False, max_iter=max_iter)
    dev = _solve(rhss, 255, 1e-10, 32, 4, True, max_iter=max_iter)
    _same(host[0], dev[0])
    assert all(i["iterations"] == max_iter and i["status"] == 5 for *_, i in dev[0])
    # LRP_NOT_CONVERGED still writes a valid result: orthonormal factors,
    # singular values positive and descending
    for U, S, V, i in dev[0]:
        assert i["rank"] >= 1 and np.all(np.isfinite(U)) and np.all(S > 0) and np.all(np.diff(S) <= 0)
        assert np.abs(U.T @ U - np.eye(S.shape[0])).max() < 1e-10
        assert np.abs(V.T @ V - np.eye(S.shape[0])).max() < 1e-10
