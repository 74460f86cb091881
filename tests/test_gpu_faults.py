"""Host-made faults on the GPU path (needs a GB300; no GPU fault, trap or hang).

* A bounded wait that runs out: the test hook cb_debug_stall_tile makes one
  tile of the column-blocked SpMV expect a column block that is never
  copied.  Its mbarrier wait gives up after 1 s of global time; that
  realisation reports CB_ERR_TIMEOUT, the others are unaffected, and the
  context stays usable (the same handle gives the reference scores again
  once the hook is off, through direct launches and captured graphs).
* Out of memory: cb_set_memory_limit caps the library's device memory, so
  allocations fail as on a full device.  Uploads, workspaces and the restart
  buffers then return CB_ERR_OOM and free what they took.
"""
import math
import time

import numpy as np
import pytest

from paper_1409_5000_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K_BTILE_ROWS = 16384  # rows per column-blocked tile


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1409_5000_gb300 import binding

    binding.lib()
    return binding


@pytest.fixture(scope="module")
def ens():
    return synth.er_ensemble([20_000, 40_000, 9_000], 10.0, 10, 4, config=501)


def _run(B, gs, m, prec, report):
    S = torch.empty(gs.n_max, dtype=torch.float64, device="cuda")
    ls = torch.empty(1, dtype=torch.float64, device="cuda")
    rep = (B.InstReport * len(gs.n))() if report else None
    err = None
    try:
        B.cb_ensemble_scores(gs.h, m, prec, gs.n_max, S.data_ptr(), ls.data_ptr(), rep,
                             torch.cuda.current_stream().cuda_stream)
    except B.CBError as e:
        err = e
    torch.cuda.synchronize()
    return err, float(ls.item()), S.cpu().numpy(), rep


def test_bounded_wait_times_out(B, ens):
    first = [sum(math.ceil(g.n / K_BTILE_ROWS) for g in ens.graphs[:r]) for r in range(3)]
    with B.GraphSet(ens.graphs) as gs:
        err, ls_ref, S_ref, _ = _run(B, gs, 12, B.CB_FP32, True)
        assert err is None
        _, ls_ref0, S_ref0, _ = _run(B, gs, 12, B.CB_FP32, False)
        assert ls_ref0 == ls_ref and np.array_equal(S_ref0, S_ref)
        B.cb_debug_stall_tile(gs.h, first[1] + 1)  # second tile of realisation 1
        t0 = time.perf_counter()
        err, ls, S, rep = _run(B, gs, 12, B.CB_FP32, True)
        dt = time.perf_counter() - t0
        assert err is not None and err.code == B.CB_ERR_TIMEOUT, err
        assert [r.status for r in rep] == [B.CB_OK, B.CB_ERR_TIMEOUT, B.CB_OK]
        assert rep[1].m_eff == 0 and rep[0].m_eff == 12 and rep[2].m_eff == 12
        assert math.isnan(ls) and np.all(np.isnan(S))
        assert 0.5 < dt < 30.0, dt  # one bounded (1 s) wait, not a hang
        # FP64 runs the tiled-CSR kernel (no bulk copies): unaffected
        err, _, _, _ = _run(B, gs, 12, B.CB_FP64, True)
        assert err is None
        # off again: the same handle, direct launches, then captured and replayed
        B.cb_debug_stall_tile(gs.h, 0xFFFFFFFF)
        for rep_on in (True, False, False, False):
            err, ls, S, _ = _run(B, gs, 12, B.CB_FP32, rep_on)
            assert err is None and ls == ls_ref and np.array_equal(S, S_ref)


def test_stall_drops_captured_graphs(B, ens):
    """A pass captured before the hook is set must not replay without it."""
    with B.GraphSet(ens.graphs) as gs:
        S = torch.empty(gs.n_max, dtype=torch.float64, device="cuda")
        ls = torch.empty(1, dtype=torch.float64, device="cuda")
        for _ in range(3):
            B.ensemble_scores(gs, 10, B.CB_FP32, out=(S, ls))
        B.cb_debug_stall_tile(gs.h, 0)
        B.ensemble_scores(gs, 10, B.CB_FP32, out=(S, ls))
        torch.cuda.synchronize()
        assert math.isnan(float(ls.item()))
        B.cb_debug_stall_tile(gs.h, 0xFFFFFFFF)
        with pytest.raises(B.CBError):
            B.cb_debug_stall_tile(gs.h, 10_000)


def test_memory_limit_oom(B, ens):
    torch.cuda.synchronize()
    base = B.cb_memory_in_use()
    try:
        B.cb_set_memory_limit(base + (1 << 20))  # 1 MiB: far too little for the upload
        with pytest.raises(B.CBError) as ei:
            B.GraphSet(ens.graphs)
        assert ei.value.code == B.CB_ERR_OOM
        assert B.cb_memory_in_use() == base  # nothing kept by the failed upload
        B.cb_set_memory_limit(0)
        with B.GraphSet(ens.graphs) as gs:
            ref = B.ensemble_scores(gs, 10, B.CB_FP32)[1].cpu().numpy()
            held = B.cb_memory_in_use()
            # room for the handle and its workspace, not for the restart buffers
            B.cb_set_memory_limit(held + 4096)
            with pytest.raises(B.CBError) as ei:
                B.ensemble_scores_restarted(gs, 10, 2, B.CB_FP32)
            assert ei.value.code == B.CB_ERR_OOM
            assert B.cb_memory_in_use() == held
            # a larger workspace does not fit either; the handle still works
            with pytest.raises(B.CBError) as ei:
                B.ensemble_scores(gs, 40, B.CB_FP32)
            assert ei.value.code == B.CB_ERR_OOM
            B.cb_set_memory_limit(0)
            again = B.ensemble_scores(gs, 10, B.CB_FP32)[1].cpu().numpy()
            assert np.array_equal(ref, again)
        assert B.cb_memory_in_use() == base
    finally:
        B.cb_set_memory_limit(0)
