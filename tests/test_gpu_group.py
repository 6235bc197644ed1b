"""lrp_group_*: a batch solved as concurrent sub-batches on several lanes gives
each problem exactly the result of a single plan; the compact pack chains the
lanes' results."""
import numpy as np
import pytest

import lrp_inputs as li

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_group_equals_single_plan(precision):
    import paper_2607_06021_gb300 as lrp
    from tests.gpu_util import rhs_dev, to_np
    n = 1023
    rhss = [li.gaussian_eigen_rhs(n, 40 + i, 3 + i % 9) for i in range(11)]
    kw = dict(max_rhs_rank=16, m_cap=48, precision=precision)
    grp = lrp.Group(n, 1e-8, 16, lanes=3, batch=12, **kw)
    res_g = grp.solve_batch([rhs_dev(r) for r in rhss])
    plan = lrp.Plan(n, 1e-8, 16, batch=12, **kw)
    res_p = plan.solve_batch([rhs_dev(r) for r in rhss])
    for (Ug, Sg, Vg, ig), (Up, Sp, Vp, ip) in zip(res_g, res_p):
        assert ig["rank"] == ip["rank"] and ig["total_iterations"] == ip["total_iterations"]
        assert np.array_equal(to_np(Ug), to_np(Up)) and np.array_equal(to_np(Sg), to_np(Sp))
        assert np.array_equal(to_np(Vg), to_np(Vp))
    # compact results of all lanes, back to back in problem order
    cap = 11 * (2 * n + 1) * 16
    packed = torch.zeros(cap, dtype=torch.float64, device="cuda")
    offs = torch.zeros(12, dtype=torch.int64, device="cuda")
    grp.pack(packed, offs)
    torch.cuda.synchronize()
    o, pk = offs.cpu().numpy(), packed.cpu().numpy()
    for i, (U, S, V, info) in enumerate(res_g):
        r = info["rank"]
        assert np.array_equal(pk[o[i]:o[i] + n * r].reshape(r, n).T, to_np(U))
        assert np.array_equal(pk[o[i] + n * r:o[i] + n * r + r], to_np(S))
    assert o[11] == sum((2 * n + 1) * info["rank"] for *_, info in res_g)
    grp.close()
    plan.close()
