"""lrp_plan_pack: the compact copy of a batch's results holds exactly the first
rank columns of U and V and the rank singular values of every problem."""
import numpy as np
import pytest

import lrp_inputs as li

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_pack_matches_outputs_and_respects_capacity():
    import paper_2607_06021_gb300 as lrp
    from tests.gpu_util import rhs_dev, to_np
    n = 1023
    rhss = [li.gaussian_eigen_rhs(n, s, r) for s, r in [(1, 3), (2, 9), (3, 14)]]
    plan = lrp.Plan(n, 1e-8, 32, max_rhs_rank=16, batch=3, precision="mixed")
    res = plan.solve_batch([rhs_dev(r) for r in rhss])
    cap = 3 * (2 * n + 1) * 32
    packed = torch.full((cap,), -7.0, dtype=torch.float64, device="cuda")
    offs = torch.zeros(4, dtype=torch.int64, device="cuda")
    plan.pack(packed, offs)
    torch.cuda.synchronize()
    o = offs.cpu().numpy()
    pk = packed.cpu().numpy()
    for i, (U, S, V, info) in enumerate(res):
        r = info["rank"]
        blk = pk[o[i]:o[i] + (2 * n + 1) * r]
        assert np.array_equal(blk[:n * r].reshape(r, n).T, to_np(U)[:, :r])
        assert np.array_equal(blk[n * r:n * r + r], to_np(S)[:r])
        assert np.array_equal(blk[n * r + r:].reshape(r, n).T, to_np(V)[:, :r])
    assert o[3] == sum((2 * n + 1) * info["rank"] for *_, info in res)
    assert np.all(pk[o[3]:] == -7.0)
    # too small a buffer: nothing beyond capacity is written, the total says so
    small = torch.full((10,), -7.0, dtype=torch.float64, device="cuda")
    plan.pack(small, offs)
    torch.cuda.synchronize()
    assert offs[3].item() > 10 and torch.all(small == -7.0).item()
    plan.close()
