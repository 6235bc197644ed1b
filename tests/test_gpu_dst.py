"""DST-I kernel parity with the oracle (scipy DST-I / direct sine sum)."""
import numpy as np
import pytest

from oracle import poisson as po

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 3, 7, 63, 255, 1023, 4095, 8191])
@pytest.mark.parametrize("ncols", [1, 5])
def test_dst1_matches_oracle(n, ncols):
    from tests.gpu_util import to_dev, to_np
    import paper_2607_06021_gb300 as lrp
    rng = np.random.default_rng(n * 7 + ncols)
    X = rng.standard_normal((n, ncols))
    Y = to_np(lrp.dst1(to_dev(X)))
    ref = po.dst1(X)
    scale = np.abs(ref).max()
    assert np.abs(Y - ref).max() <= 1e-13 * max(scale, 1.0) * np.log2(n + 1)


def test_dst1_ld_larger_than_n_and_self_inverse():
    import paper_2607_06021_gb300 as lrp
    n, c, ld = 511, 3, 600
    rng = np.random.default_rng(3)
    buf = torch.zeros((c, ld), dtype=torch.float64, device="cuda")
    buf[:, :n] = torch.from_numpy(rng.standard_normal((c, n))).cuda()
    X = buf.t()[:n, :]            # n x c view with ld = 600
    Y = lrp.dst1(X)
    Z = lrp.dst1(Y)
    assert torch.abs(Z - X).max().item() < 1e-13 * np.sqrt(n)
    assert torch.all(buf[:, n:] == 0)


@pytest.mark.parametrize("n,ncols", [(16383, 3), (65535, 2), ((1 << 20) - 1, 2)])
def test_dst1_multipass_matches_oracle(n, ncols):
    # n+1 > 8192: the four-step FFT through HBM (two passes).
    from tests.gpu_util import to_dev, to_np
    import paper_2607_06021_gb300 as lrp
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, ncols))
    Y = to_np(lrp.dst1(to_dev(X)))
    ref = po.dst1(X)
    scale = np.abs(ref).max()
    assert np.abs(Y - ref).max() <= 1e-13 * max(scale, 1.0) * np.log2(n + 1)
