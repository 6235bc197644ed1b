"""Request server: continuous batching of mixed sizes and precisions gives the
same result for every request as a standalone solve of it; warm-start keys;
admission by footprint; latency statistics."""
import numpy as np
import pytest

import lrp_inputs as li
from oracle import poisson as po

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bucket_plan(lrp, n, r_f, tol, max_rank, precision):
    # the server's plan for this request's bucket: r_f rounded up to a multiple
    # of 16; m_cap = min(2 max_rank + that, 256) in FP64, 64 in mixed precision
    # while r_f' + 16 <= 64
    rfc = (r_f + 15) // 16 * 16
    m64 = min(2 * max_rank + rfc, 256)
    m_cap = m64 if precision == "fp64" else min(max(64, rfc + 16), max(m64, rfc + 2))
    return lrp.Plan(n, tol, max_rank, max_rhs_rank=rfc, m_cap=m_cap, precision=precision)


def test_mixed_stream_equals_standalone_solves():
    import paper_2607_06021_gb300 as lrp
    from tests.gpu_util import rhs_dev, to_np
    rng = np.random.default_rng(5)
    reqs = []
    for i in range(24):
        n = int(rng.choice([255, 1023, 4095]))
        r_f = int(rng.integers(2, 13))
        prec = "fp64" if i % 4 == 0 else "mixed"
        tol = 1e-10 if prec == "fp64" else 1e-6
        reqs.append((li.gaussian_eigen_rhs(n, 100 + i, r_f), prec, tol))
    sv = lrp.Server(lanes=2, max_batch=8)
    rmax = {"fp64": 64, "mixed": 32}
    tickets = [sv.submit(r.U, r.s, r.V, tol, rmax[prec], prec) for r, prec, tol in reqs]
    assert all(t is not None for t in tickets)
    results = [sv.wait(t, 120.0) for t in tickets]
    stats = sv.stats()
    sv.close()
    assert stats["completed"] == len(reqs) and stats["p99_us"] >= stats["p50_us"] > 0
    for (rhs, prec, tol), (U, S, V, res) in zip(reqs, results):
        assert res["status"] in (0, 5), res
        plan = _bucket_plan(lrp, rhs.n, rhs.rank, tol, rmax[prec], prec)
        Ua, Sa, Va, info = plan.solve(*rhs_dev(rhs))
        plan.close()
        Ua, Sa, Va = to_np(Ua), to_np(Sa), to_np(Va)
        # same plan shape, per-slot kernels: the batch neighbours change nothing
        assert res["rank"] == info["rank"]
        assert po.lowrank_rel_diff(U, S, V, Ua, Sa, Va) <= 1e-14, (rhs.n, prec)
        if res["status"] == 0:
            G = po.SpectralSolution(rhs.U, rhs.s, rhs.V)
            err = po.rel_error_vs_exact(U, S, V, G)
            assert err <= max(10 * tol, 1e-6 if prec == "mixed" else 0.0), (rhs.n, prec, err)


def test_warm_key_reuses_record():
    import paper_2607_06021_gb300 as lrp
    rhs = li.workload_n4095(1)
    r2 = li.perturb_amplitudes(rhs, 3)
    sv = lrp.Server(lanes=1)
    a = sv.wait(sv.submit(rhs.U, rhs.s, rhs.V, 1e-8, 64, "fp64", warm_key=42), 60.0)
    b = sv.wait(sv.submit(r2.U, r2.s, r2.V, 1e-8, 64, "fp64", warm_key=42), 60.0)
    c = sv.wait(sv.submit(r2.U, r2.s, r2.V, 1e-8, 64, "fp64"), 60.0)
    sv.close()
    assert a[3]["warm_used"] == 0 and b[3]["warm_used"] == 1 and c[3]["warm_used"] == 0
    G = po.SpectralSolution(r2.U, r2.s, r2.V)
    assert po.rel_error_vs_exact(*b[:3], G) < 10 * 1e-8


def test_admission_by_footprint_and_queue():
    import paper_2607_06021_gb300 as lrp
    rhs = li.gaussian_eigen_rhs(4095, 1, 8)
    small = lrp.Server(memory_cap_bytes=1 << 20)
    with pytest.raises(lrp.LrpError) as e:
        small.submit(rhs.U, rhs.s, rhs.V, 1e-6, 32)
    assert e.value.status == lrp.LRP_ECAPACITY
    small.close()
    big = li.gaussian_eigen_rhs(65535, 2, 16)
    sv = lrp.Server(lanes=1, max_queue=1)
    t0 = sv.submit(big.U, big.s, big.V, 1e-10, 64, "fp64")
    t1 = sv.submit(rhs.U, rhs.s, rhs.V, 1e-6, 32)
    t2 = sv.submit(rhs.U, rhs.s, rhs.V, 1e-6, 32)
    assert t0 is not None and (t1 is None or t2 is None)
    for t in (t0, t1, t2):
        if t is not None:
            assert sv.wait(t, 120.0) is not None
    assert sv.stats()["rejected"] >= 1
    sv.close()
