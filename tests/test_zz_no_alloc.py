"""cb_topk_noalloc: top-k for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: an application that has reserved the
whole GPU for its own pool, or a host that forbids CUDA allocation calls.
For them the library keeps a fixed device array and this entry point uses it
instead of allocating.  The test calls it through the C ABI twice in a row
and checks that both results equal cb_topk's (bit-exact, as every top-k test
here), and that a k beyond the fixed capacity is rejected.  It lives in a
file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1409_5000_gb300 import binding

    L = binding.lib()
    L.cb_topk_noalloc.restype = ctypes.c_int
    L.cb_topk_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return L


def _run(L, fn, S, k):
    idx = torch.empty(k, dtype=torch.int32, device="cuda")
    val = torch.empty(k, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = fn(ctypes.c_void_p(S.data_ptr()), S.numel(), k, ctypes.c_void_p(idx.data_ptr()),
            ctypes.c_void_p(val.data_ptr()), ctypes.c_void_p(stream))
    assert rc == 0, L.cb_last_error()
    torch.cuda.synchronize()
    return idx.cpu().numpy(), val.cpu().numpy()


def test_noalloc_topk_matches_topk_twice(lib):
    rng = np.random.default_rng(2024)
    cases = [(np.exp(rng.normal(size=2_000_000) * 2), 30),
             (rng.integers(0, 40, size=300_000).astype(np.float64), 4096)]  # many ties, max k
    for S_np, k in cases:  # two calls in a row sharing the fixed scratch
        S = torch.from_numpy(S_np).cuda()
        ref_idx, ref_val = _run(lib, lib.cb_topk, S, k)
        got_idx, got_val = _run(lib, lib.cb_topk_noalloc, S, k)
        assert np.array_equal(got_idx, ref_idx)
        assert np.array_equal(got_val, ref_val)


def test_noalloc_rejects_k_beyond_capacity(lib):
    S = torch.zeros(10_000, dtype=torch.float64, device="cuda")
    idx = torch.empty(5000, dtype=torch.int32, device="cuda")
    val = torch.empty(5000, dtype=torch.float64, device="cuda")
    rc = lib.cb_topk_noalloc(ctypes.c_void_p(S.data_ptr()), S.numel(), 5000,
                             ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(val.data_ptr()), None)
    assert rc == 1  # CB_ERR_ARG
    assert b"capacity" in lib.cb_last_error()
