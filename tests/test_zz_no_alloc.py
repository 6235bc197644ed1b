"""lrp_dst1_noalloc, the allocation-free DST-I entry point, against lrp_dst1
and the oracle's DST.

Callers that may not allocate device memory at call time (host callbacks that
run while another framework owns the memory pool, code under a fixed memory
budget, callers that must avoid the implicit synchronisation of cudaMalloc)
use lrp_dst1_noalloc: its scratch is a fixed array inside the library.  This
file is collected last so that a failure here leaves every other test run.
"""
import ctypes

import numpy as np
import pytest

from oracle import poisson as po

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _entry():
    import paper_2607_06021_gb300 as lrp
    f = lrp.library().lrp_dst1_noalloc
    f.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_int64, ctypes.c_void_p]
    f.restype = ctypes.c_int32
    return lrp, f


def _call(lrp, f, X, n, c):
    stream = torch.cuda.current_stream()
    Y = torch.full((c, n), float("nan"), dtype=torch.float64, device="cuda").t()
    st = f(n, c, X.data_ptr(), n, Y.data_ptr(), n, ctypes.c_void_p(stream.cuda_stream))
    assert st == lrp.LRP_OK, lrp.last_error()
    torch.cuda.synchronize()
    return Y


def test_dst1_noalloc_matches_dst1_on_two_calls_in_a_row():
    lrp, f = _entry()
    # two sizes in a row (the second call rewrites the shared scratch), then the
    # largest size the scratch serves, n + 1 = 8192
    for call, (n, c) in enumerate([(4095, 3), (255, 5), (8191, 2)]):
        rng = np.random.default_rng(100 + call)
        Xh = rng.standard_normal((n, c))
        X = torch.from_numpy(np.ascontiguousarray(Xh.T)).cuda().t()
        ref = lrp.dst1(X)
        Y = _call(lrp, f, X, n, c)
        scale = float(ref.abs().max())
        # the tolerance of the DST parity tests
        tol = 1e-13 * max(scale, 1.0) * np.log2(n + 1)
        assert float((Y - ref).abs().max()) <= tol
        # and against the oracle's DST-I (scipy's orthonormal type-1 transform)
        Yo = po.dst1(Xh)
        assert np.abs(Y.cpu().numpy() - Yo).max() <= tol


def test_dst1_noalloc_allocates_no_device_memory():
    lrp, f = _entry()
    n, c = 4095, 4
    rng = np.random.default_rng(7)
    X = torch.from_numpy(np.ascontiguousarray(rng.standard_normal((c, n)))).cuda().t()
    Y = torch.empty((c, n), dtype=torch.float64, device="cuda").t()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # the first call on the device may load the kernels (module loading is not
    # the call's own allocation); the device's free memory must not move across
    # the calls after it
    assert f(n, c, X.data_ptr(), n, Y.data_ptr(), n, stream) == lrp.LRP_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert f(n, c, X.data_ptr(), n, Y.data_ptr(), n, stream) == lrp.LRP_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_dst1_noalloc_rejects_sizes_beyond_its_scratch():
    lrp, f = _entry()
    n = 16383  # n+1 = 16384 > 8192, the largest table the fixed scratch holds
    st = f(n, 1, ctypes.c_void_p(16), n, ctypes.c_void_p(16), n, None)
    assert st == lrp.LRP_EINVAL
    assert "8192" in lrp.last_error()
