"""lrp_dst1_noalloc, the allocation-free DST-I entry point, against lrp_dst1.

Callers that may not allocate device memory at call time (host callbacks that
run while another framework owns the memory pool, code under a fixed memory
budget, callers that must avoid the implicit synchronisation of cudaMalloc)
use lrp_dst1_noalloc: its scratch is a fixed array inside the library.  This
file is collected last so that a failure here leaves every other test run.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _entry():
    import paper_2607_06021_gb300 as lrp
    f = lrp.library().lrp_dst1_noalloc
    f.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_int64, ctypes.c_void_p]
    f.restype = ctypes.c_int32
    return lrp, f


def test_dst1_noalloc_matches_dst1_on_two_calls_in_a_row():
    lrp, f = _entry()
    stream = torch.cuda.current_stream()
    for call, (n, c) in enumerate([(4095, 3), (255, 5)]):
        rng = np.random.default_rng(100 + call)
        X = torch.from_numpy(np.ascontiguousarray(rng.standard_normal((c, n)))).cuda().t()
        ref = lrp.dst1(X)
        Y = torch.full((c, n), float("nan"), dtype=torch.float64, device="cuda").t()
        st = f(n, c, X.data_ptr(), n, Y.data_ptr(), n, ctypes.c_void_p(stream.cuda_stream))
        assert st == lrp.LRP_OK, lrp.last_error()
        torch.cuda.synchronize()
        scale = float(ref.abs().max())
        # the tolerance of the DST parity tests
        assert float((Y - ref).abs().max()) <= 1e-13 * max(scale, 1.0) * np.log2(n + 1)


def test_dst1_noalloc_rejects_sizes_beyond_its_scratch():
    lrp, f = _entry()
    n = 16383  # n+1 = 16384 > 8192, the largest table the fixed scratch holds
    st = f(n, 1, ctypes.c_void_p(16), n, ctypes.c_void_p(16), n, None)
    assert st == lrp.LRP_EINVAL
    assert "8192" in lrp.last_error()
