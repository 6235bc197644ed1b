"""Launch shapes (lrp_opts.gemm_rows_per_thread, dst_cta_threads) change only
how the work is spread over threads and CTAs: every problem's result must be
the same bits under every allowed value, in both precisions, at a grid whose
DST packs several columns per CTA (n = 1023) and at the bench workload's
n = 4095; the autotuner relies on this."""
import numpy as np
import pytest

import lrp_inputs as li

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [dict(gemm_rows_per_thread=1, dst_cta_threads=1024), dict(gemm_rows_per_thread=2, dst_cta_threads=512),
          dict(gemm_rows_per_thread=1, dst_cta_threads=256)]


@pytest.mark.parametrize("n,precision", [(1023, "mixed"), (1023, "fp64"), (4095, "mixed"), (4095, "fp64")])
def test_results_do_not_depend_on_launch_shapes(n, precision):
    import paper_2607_06021_gb300 as lrp
    from tests.gpu_util import rhs_dev, to_np
    rhss = [li.gaussian_eigen_rhs(n, 70 + i, 4 + i % 12, 2) for i in range(8)]
    kw = dict(batch=8, max_rhs_rank=16, m_cap=64, precision=precision)
    tol = 1e-8
    base = lrp.Plan(n, tol, 32, **kw)
    ref = base.solve_batch([rhs_dev(r) for r in rhss])
    base.close()
    for shp in SHAPES:
        plan = lrp.Plan(n, tol, 32, **kw, **shp)
        res = plan.solve_batch([rhs_dev(r) for r in rhss])
        plan.close()
        for (U, S, V, info), (Ur, Sr, Vr, ir) in zip(res, ref):
            assert info == ir, shp
            assert np.array_equal(to_np(U), to_np(Ur)) and np.array_equal(to_np(S), to_np(Sr)), shp
            assert np.array_equal(to_np(V), to_np(Vr)), shp
