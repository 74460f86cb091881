"""cb_topk_noalloc: top-k for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: an application that has reserved the
whole GPU for its own pool and refuses further allocations, or a host that
forbids CUDA allocation calls in its plug-ins.  For them the library keeps a
fixed device array and this entry point uses it instead of allocating.

The tests call it through the C ABI and check, bit for bit:
* against the FP64 oracle's full sort (oracle.topk) and against cb_topk;
* two calls in a row on one stream with nothing between them, k falling
  from the maximum (4096) to 30 on different scores, so the second call
  must clear what the first left in the shared array;
* that a k beyond the fixed capacity is rejected.
The file is collected last, so a run that stops at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle.communicability as oc

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


def _launch(L, fn, S, k):
    """Enqueue one call on the current stream; returns the device outputs."""
    idx = torch.empty(k, dtype=torch.int32, device="cuda")
    val = torch.empty(k, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = fn(ctypes.c_void_p(S.data_ptr()), S.numel(), k, ctypes.c_void_p(idx.data_ptr()),
            ctypes.c_void_p(val.data_ptr()), ctypes.c_void_p(stream))
    assert rc == 0, L.cb_last_error()
    return idx, val


def _host(out):
    torch.cuda.synchronize()
    return out[0].cpu().numpy().astype(np.int64), out[1].cpu().numpy()


def _cases():
    rng = np.random.default_rng(2024)
    return [(np.exp(rng.normal(size=2_000_000) * 2), 30),
            (rng.integers(0, 40, size=300_000).astype(np.float64), 4096)]  # many ties, max k


def test_noalloc_topk_matches_oracle_and_topk(lib):
    for S_np, k in _cases():
        S = torch.from_numpy(S_np).cuda()
        ref_idx, ref_val = oc.topk(S_np, k)
        got_idx, got_val = _host(_launch(lib, lib.cb_topk_noalloc, S, k))
        assert np.array_equal(got_idx, ref_idx)
        assert np.array_equal(got_val, ref_val)
        lib_idx, lib_val = _host(_launch(lib, lib.cb_topk, S, k))
        assert np.array_equal(got_idx, lib_idx)
        assert np.array_equal(got_val, lib_val)


def test_noalloc_two_calls_in_a_row(lib):
    """Back to back on one stream, no other top-k call between: k = 4096 on
    scores with many ties, then k = 30 on other scores; then the same pair
    again in the opposite order.  Every result equals the oracle's."""
    (S_big, k_big), (S_ties, k_ties) = _cases()
    pairs = [((S_ties, k_ties), (S_big, k_big)), ((S_big, k_big), (S_ties, k_ties))]
    for first, second in pairs:
        S1 = torch.from_numpy(first[0]).cuda()
        S2 = torch.from_numpy(second[0]).cuda()
        torch.cuda.synchronize()
        out1 = _launch(lib, lib.cb_topk_noalloc, S1, first[1])
        out2 = _launch(lib, lib.cb_topk_noalloc, S2, second[1])
        for out, (S_np, k) in ((out1, first), (out2, second)):
            got_idx, got_val = _host(out)
            ref_idx, ref_val = oc.topk(S_np, k)
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
