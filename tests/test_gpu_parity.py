"""CUDA path vs the FP64 oracle, element by element (needs a GB300).

Every case runs through the C ABI (via the ctypes binding) on seeded
synthetic graphs shaped like the paper's workloads, at sizes the oracle
finishes in seconds, spanning several SpMV tiles, reduction groups and a
ragged tail, plus the degenerate cases of the method.
"""
import math

import numpy as np
import pytest

import oracle.communicability as oc
from paper_1409_5000_gb300 import synth
from tests import parity, pins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PREC = {"fp32": 0, "fp64": 1}
# The FP32 cases here run the specialised formats wherever they are built
# (CB_PATH_FORMATS): the automatic choice would give these small handles to
# the tiled-CSR kernel, which the tune and CSR-only cases cover.
FORMATS = 1


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1409_5000_gb300 import binding

    binding.lib()  # raises if libcb.so is missing: no fallback
    return binding


def _single(B, g, m, prec, csr_only=False):
    with B.GraphSet([g], csr_only=csr_only, path=None if csr_only else FORMATS) as gs:
        ls, y, rep = B.communicability(gs, 0, m, PREC[prec], report=True)
        torch.cuda.synchronize()
        return float(ls.item()), y.cpu().numpy(), rep


class _G:
    def __init__(self, n, rp, col):
        self.n, self.row_ptr, self.col = n, rp, col


CLOSED = [(name, mk) for name, mk in pins.CLOSED]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CLOSED, ids=[c[0] for c in CLOSED])
def test_closed_forms(B, case, prec):
    name, mk = case
    (n, rp, col), ref, dim = mk()
    theta, y, rep = _single(B, _G(n, rp, col), 20, prec)
    s = np.exp(theta) * y
    tol = parity.TOL_FP64 if prec == "fp64" else 2e-6
    assert np.max(np.abs(s - ref) / ref) <= tol, (name, np.max(np.abs(s - ref) / ref))
    if prec == "fp64":
        assert rep.m_eff == dim


def test_single_isolated_node(B):
    g = synth.from_edges(1, np.zeros((0, 2), np.uint32))
    for prec in ("fp64", "fp32"):
        theta, y, rep = _single(B, g, 10, prec)
        assert rep.m_eff == 1 and abs(math.exp(theta) * y[0] - 1.0) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_er_ensemble_small(B, prec):
    """10 x ER(500, p=0.016) + 15-node sparse target, m = 20, top-15."""
    ens = synth.er_ensemble_small()
    m, k = ens.meta["m"], ens.meta["k"]
    gs_o = [(g.n, g.row_ptr, g.col) for g in ens.graphs]
    theta_o, S_o = oc.ensemble_scores(gs_o, m)
    with B.GraphSet(ens.graphs, path=FORMATS) as gs:
        ls, S, rep = B.ensemble_scores(gs, m, PREC[prec], report=True)
        idx, val = B.topk(S, k)
        torch.cuda.synchronize()
        e = parity.assert_scores(ls.item(), S.cpu().numpy(), theta_o, S_o, prec)
        tol = parity.TOL_FP64 if prec == "fp64" else parity.TOL_FP32
        parity.assert_topk(idx.cpu().numpy(), val.cpu().numpy(), S_o, k, tol)
        assert all(r.m_eff == m and r.status == 0 for r in rep)
    # each realisation alone through the plain per-graph call
    with B.GraphSet(ens.graphs, path=FORMATS) as gs:
        for r in (0, 9):
            ls, y = B.communicability(gs, r, m, PREC[prec])
            th_o, y_o, _ = oc.krylov_expv(*gs_o[r], m)
            parity.assert_scores(ls.item(), y.cpu().numpy(), th_o, y_o, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_uneven_ensemble(B, prec):
    """8 ER realisations, n ~ U[2e3, 4e4], dbar 20, 30-node target, m = 25:
    many tiles, several reduction groups, ragged tails, padding (eq. 5)."""
    ens = synth.er_ensemble_uneven(n_inst=8, n_lo=2_000, n_hi=40_000, config=303)
    m = ens.meta["m"]
    gs_o = [(g.n, g.row_ptr, g.col) for g in ens.graphs]
    theta_o, S_o = oc.ensemble_scores(gs_o, m)
    with B.GraphSet(ens.graphs, path=FORMATS) as gs:
        ls, S = B.ensemble_scores(gs, m, PREC[prec], n_out=ens.n_max + 37)
        S = S.cpu().numpy()
        assert np.all(S[ens.n_max:] == 0.0)
        parity.assert_scores(ls.item(), S[: ens.n_max], theta_o, S_o, prec)
        idx, val = B.topk(torch.from_numpy(S).cuda(), 30)
        tol = parity.TOL_FP64 if prec == "fp64" else parity.TOL_FP32
        parity.assert_topk(idx.cpu().numpy(), val.cpu().numpy(), S_o[: ens.n_max], 30, tol)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kind", ["er", "ba", "ws"])
def test_single_background_clique(B, kind, prec):
    """n = 1e5 ER / BA / WS + planted 12-clique, m = 30 (BA rows reach the
    warp and whole-CTA tiers)."""
    ens = synth.single_clique_100k(kind)
    g = ens.graphs[0]
    m = ens.meta["m"]
    th_o, y_o, _ = oc.krylov_expv(g.n, g.row_ptr, g.col, m)
    theta, y, rep = _single(B, g, m, prec)
    parity.assert_scores(theta, y, th_o, y_o, prec)
    tol = parity.TOL_FP64 if prec == "fp64" else parity.TOL_FP32
    with B.GraphSet([g], path=FORMATS) as gs:
        ls, yy = B.communicability(gs, 0, m, PREC[prec])
        idx, val = B.topk(yy, 12)
        parity.assert_topk(idx.cpu().numpy(), val.cpu().numpy(), y_o, 12, tol)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_heavy_rows(B, prec):
    """A hub of degree ~20000 (split across CTAs), rows of degree 1024-8192
    (whole-CTA tier) and ordinary ER rows."""
    n = 30_000
    rng = np.random.default_rng(11)
    hub = [(0, j) for j in range(1, 20_001)]
    mid = [(1, int(j)) for j in rng.choice(np.arange(2, n), 3000, replace=False)]
    mid += [(2, int(j)) for j in rng.choice(np.arange(3, n), 1500, replace=False)]
    g0 = synth.er(n, 6.0 / n, 5)
    src = np.repeat(np.arange(n), np.diff(g0.row_ptr.astype(np.int64)))
    base = [(int(a), int(b)) for a, b in zip(src, g0.col) if a < b]
    g = synth.from_edges(n, base + hub + mid)
    assert g.degrees().max() > 8192
    th_o, y_o, _ = oc.krylov_expv(g.n, g.row_ptr, g.col, 30)
    theta, y, _ = _single(B, g, 30, prec)
    parity.assert_scores(theta, y, th_o, y_o, prec)


@pytest.mark.parametrize("kind", ["er", "ws"])
def test_converged_every_score_fp64(B, kind):
    """Once m is large enough for the spectral width, the m-step result is
    e^A 1 itself, and every score (not only the head) is within 1e-10."""
    g = synth.er(20_000, 8.0 / 20_000, 3) if kind == "er" else synth.ws(20_000, 10, 0.1, 3)
    th_o, y_o, _ = oc.krylov_expv(g.n, g.row_ptr, g.col, 70)
    theta, y, _ = _single(B, g, 70, "fp64")
    parity.assert_scores_all(theta, y, th_o, y_o, parity.TOL_FP64)


def test_empty_and_complete_breakdown(B):
    g = synth.from_edges(5000, np.zeros((0, 2), np.uint32))
    theta, y, rep = _single(B, g, 30, "fp32")
    assert rep.m_eff == 1 and np.allclose(np.exp(theta) * y, 1.0, rtol=1e-7)
    g = synth.from_edges(40, np.array(pins.complete(40)))
    theta, y, rep = _single(B, g, 30, "fp32")
    # FP32: theta = alpha_1 = 39 carries ~1e-7 relative error, i.e. ~4e-6 in e^theta
    assert rep.m_eff == 1 and np.allclose(np.exp(theta) * y, math.exp(39), rtol=parity.TOL_FP32)


@pytest.mark.parametrize("n,k", [(1, 1), (7, 7), (1000, 1), (2049, 2000), (4096, 17), (4096, 4096),
                                 (4097, 30), (100_000, 64), (1_234_567, 20), (50_000, 4096)])
def test_topk_bit_exact(B, n, k):
    rng = np.random.default_rng(n + k)
    S = rng.integers(0, 50, size=n).astype(np.float64) * 0.25  # many exact ties
    S[rng.integers(0, n, size=max(1, n // 100))] = -0.0
    S[rng.integers(0, n, size=max(1, n // 100))] = np.nan
    if n > 10:
        S[3] = np.inf
        S[5] = -np.inf
    idx, val = B.topk(torch.from_numpy(S).cuda(), k)
    ref_idx, ref_val = oc.topk(S, k)
    assert np.array_equal(idx.cpu().numpy().astype(np.int64), ref_idx)
    assert np.array_equal(val.cpu().numpy(), ref_val, equal_nan=True)


def test_topk_distinct_values(B):
    rng = np.random.default_rng(1)
    S = np.exp(rng.normal(size=3_000_000) * 3)
    idx, val = B.topk(torch.from_numpy(S).cuda(), 100)
    ref_idx, ref_val = oc.topk(S, 100)
    assert np.array_equal(idx.cpu().numpy().astype(np.int64), ref_idx)
    assert np.array_equal(val.cpu().numpy(), ref_val)


def test_deterministic(B):
    ens = synth.er_ensemble_uneven(n_inst=6, n_lo=5_000, n_hi=60_000, config=304)
    with B.GraphSet(ens.graphs, path=FORMATS) as gs:
        a = B.ensemble_scores(gs, 25, 0)[1].cpu().numpy()
        b = B.ensemble_scores(gs, 25, 0)[1].cpu().numpy()
    assert np.array_equal(a, b)


def test_graph_replay(B, monkeypatch):
    """Repeated ensemble calls replay a captured CUDA graph: the first call
    launches directly, the second captures, later ones replay.  All must be
    bit-identical to direct launches, also after the workspace grows (a
    per-realisation call at larger m) and for a second output buffer."""
    ens = synth.er_ensemble_uneven(n_inst=5, n_lo=5_000, n_hi=40_000, config=305)
    with B.GraphSet(ens.graphs, path=FORMATS) as gs:
        monkeypatch.setenv("CB_NO_GRAPH", "1")
        ref = {m: B.ensemble_scores(gs, m, 0) for m in (12, 30)}
        ref = {m: (float(l.item()), S.cpu().numpy()) for m, (l, S) in ref.items()}
        monkeypatch.delenv("CB_NO_GRAPH")
        n = gs.n_max
        bufs = [(torch.full((n,), -1.0, dtype=torch.float64, device="cuda"),
                 torch.zeros(1, dtype=torch.float64, device="cuda")) for _ in range(2)]
        for rep in range(4):
            for m in (12, 30):
                S, ls = bufs[m == 30]
                S.fill_(float("nan"))
                B.ensemble_scores(gs, m, 0, out=(S, ls))
                assert float(ls.item()) == ref[m][0], (rep, m)
                assert np.array_equal(S.cpu().numpy(), ref[m][1]), (rep, m)
            if rep == 1:  # regrow the workspace under the captured graphs
                B.communicability(gs, 0, 60)
                ref30 = B.ensemble_scores(gs, 30, 0)
                assert np.array_equal(ref30[1].cpu().numpy(), ref[30][1])


def test_memory_pool_reuse_and_release(B):
    """Freed handles leave their memory in the library's pool; a second upload
    reuses it and computes the same scores; cb_release_cached_memory hands
    it back to the driver."""
    g = synth.er(200_000, 20.0 / 200_000, 5)
    with B.GraphSet([g], path=FORMATS) as gs:
        ref = B.ensemble_scores(gs, 10, 0)[1].cpu().numpy()
    torch.cuda.synchronize()
    held, _ = torch.cuda.mem_get_info()
    with B.GraphSet([g], path=FORMATS) as gs:
        again = B.ensemble_scores(gs, 10, 0)[1].cpu().numpy()
    assert np.array_equal(ref, again)
    torch.cuda.synchronize()
    B.cb_release_cached_memory()
    released, _ = torch.cuda.mem_get_info()
    # the handle held ~16 MB of columns, ~9 MB of basis, ~12 MB of streams
    assert released >= held + (20 << 20), (held, released)


def test_max_depth(B):
    g = synth.er(3000, 8.0 / 3000, 9)
    th_o, y_o, _ = oc.krylov_expv(g.n, g.row_ptr, g.col, 128)
    theta, y, rep = _single(B, g, 128, "fp64")
    parity.assert_scores(theta, y, th_o, y_o, "fp64")


def test_argument_errors(B):
    g = synth.er(100, 0.05, 1)
    with B.GraphSet([g], path=FORMATS) as gs:
        y = torch.empty(100, dtype=torch.float64, device="cuda")
        ls = torch.empty(1, dtype=torch.float64, device="cuda")
        with pytest.raises(B.CBError):  # realisation out of range
            B.cb_communicability(gs.h, 1, 10, 0, y.data_ptr(), ls.data_ptr(), None, 0)
        with pytest.raises(B.CBError):
            B.communicability(gs, 0, 0)
        with pytest.raises(B.CBError):
            B.communicability(gs, 0, B.CB_MAX_M + 1)
        with pytest.raises(B.CBError):
            B.ensemble_scores(gs, 10, n_out=50)
    S = torch.zeros(10, dtype=torch.float64, device="cuda")
    with pytest.raises(B.CBError):
        B.topk(S, 11)
    bad = _G(3, np.array([0, 1, 1, 1], np.uint32), np.array([2], np.uint32))  # not symmetric
    with pytest.raises(B.CBError):
        B.GraphSet([bad], validate=True)


def test_column_blocked_matches_tiled_csr(B):
    """The FP32 column-blocked SpMV (shared-memory gathers) and the tiled-CSR
    SpMV compute the same recurrence: results agree to FP32 rounding, and
    both agree with the oracle.  n = 70 000 spans 5 column blocks and a
    ragged last tile; a hub row takes the long-row tier."""
    n = 70_000
    g0 = synth.er(n, 12.0 / n, 41)
    src = np.repeat(np.arange(n), np.diff(g0.row_ptr.astype(np.int64)))
    base = [(int(a), int(b)) for a, b in zip(src, g0.col) if a < b]
    hub = [(7, int(j)) for j in range(20_000, 21_000)]
    g = synth.from_edges(n, base + hub)
    res = {}
    for mode in ("blocked", "csr"):
        res[mode] = _single(B, g, 30, "fp32", csr_only=mode == "csr")
    (tb, yb, _), (tc, yc, _) = res["blocked"], res["csr"]
    e = parity.errors(tb, yb, tc, yc)  # head + normwise: the tail is FP32 noise in both
    assert e["head_rel"] < 1e-5 and e["norm_rel"] < 1e-5, e
    th_o, y_o, _ = oc.krylov_expv(g.n, g.row_ptr, g.col, 30)
    parity.assert_scores(tb, yb, th_o, y_o, "fp32")


@pytest.mark.parametrize("n", [16_384, 16_385, 32_771, 49_152])
def test_column_block_boundaries(B, n):
    """n at and just past multiples of the 16384-entry column block: the last
    block's bulk copy is rounded up to whole 16-byte units (a 1-entry block
    copies 4 floats), and a tile's row range ends exactly on a block edge.
    Ensemble of the boundary size with a smaller realisation, FP32 vs oracle."""
    graphs = [synth.er(n, 10.0 / n, 60 + n % 97), synth.er(5_000, 0.002, 61)]
    th_o, S_o = oc.ensemble_scores([(g.n, g.row_ptr, g.col) for g in graphs], 20)
    with B.GraphSet(graphs, path=FORMATS) as gs:
        ls, S = B.ensemble_scores(gs, 20, B.CB_FP32)
        parity.assert_scores(float(ls.item()), S.cpu().numpy(), th_o, S_o, "fp32")


def test_unsorted_rows_rejected(B):
    """The column-blocked format needs each row sorted: an unsorted row is an
    argument error at upload, not a silent miscount."""
    g = synth.er(2000, 0.01, 3)
    col = g.col.copy()
    rp = g.row_ptr
    i = int(np.argmax(np.diff(rp.astype(np.int64))))
    col[rp[i]:rp[i + 1]] = col[rp[i]:rp[i + 1]][::-1].copy()
    with pytest.raises(B.CBError):
        B.GraphSet([_G(g.n, rp, col)])


def test_upload_from_device_arrays(B):
    """CSR arrays already on the device (CB_DEVICE_PTRS), still being copied
    there by work queued on the upload's stream: the handle gives
    bit-identical scores to the upload of the same graphs from host arrays."""
    ens = synth.er_ensemble_uneven(n_inst=7, n_lo=2_000, n_hi=40_000, config=313)
    with B.GraphSet(ens.graphs, path=FORMATS) as gh:
        ref = B.ensemble_scores(gh, 25, B.CB_FP32)[1].cpu().numpy()
    st = torch.cuda.Stream()
    host = [(torch.from_numpy(g.row_ptr.astype(np.uint32).view(np.int32)).pin_memory(),
             torch.from_numpy(g.col.astype(np.uint32).view(np.int32)).pin_memory())
            for g in ens.graphs]
    with torch.cuda.stream(st):
        torch.cuda._sleep(20_000_000)  # the copies below land well after the call returns
        dev = [_G(g.n, rp.to("cuda", non_blocking=True), cl.to("cuda", non_blocking=True))
               for g, (rp, cl) in zip(ens.graphs, host)]
    with B.GraphSet(dev, stream=st, path=FORMATS) as gd:
        got = B.ensemble_scores(gd, 25, B.CB_FP32, stream=st)[1]
        st.synchronize()
        assert np.array_equal(got.cpu().numpy(), ref)


def test_upload_concurrent_with_compute(B):
    """An upload on a second host thread and stream while this thread runs an
    ensemble (the double-buffered end-to-end pattern): both results are
    bit-identical to the same calls made one after the other."""
    from concurrent.futures import ThreadPoolExecutor

    ens_a = synth.er_ensemble_uneven(n_inst=6, n_lo=20_000, n_hi=120_000, config=311)
    ens_b = synth.er_ensemble_uneven(n_inst=5, n_lo=10_000, n_hi=90_000, config=312)
    with B.GraphSet(ens_a.graphs, path=FORMATS) as ga:
        ref_a = B.ensemble_scores(ga, 25, B.CB_FP32)[1].cpu().numpy()
    with B.GraphSet(ens_b.graphs, path=FORMATS) as gb:
        ref_b = B.ensemble_scores(gb, 25, B.CB_FP32)[1].cpu().numpy()
    up = torch.cuda.Stream()
    with B.GraphSet(ens_a.graphs, path=FORMATS) as ga, ThreadPoolExecutor(1) as ex:
        fut = ex.submit(lambda: B.GraphSet(ens_b.graphs, stream=up, path=FORMATS))
        for _ in range(3):
            got_a = B.ensemble_scores(ga, 25, B.CB_FP32)[1]
        torch.cuda.current_stream().synchronize()
        gb = fut.result()
        try:
            got_b = B.ensemble_scores(gb, 25, B.CB_FP32)[1].cpu().numpy()
        finally:
            gb.close()
        assert np.array_equal(got_a.cpu().numpy(), ref_a)
    assert np.array_equal(got_b, ref_b)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_small_path_single_launch(B, prec):
    """Realisations of at most 8192 nodes run all m steps in one launch (one
    CTA per realisation) on the automatic path: the scores meet the oracle bar,
    agree with the per-step tiled-CSR kernels (CB_PATH_CSR) to rounding, and
    the breakdowns (K_30, whose all-ones vector is an eigenvector, and an
    isolated-node realisation: m_eff = 1) stop where the per-step path stops.
    Uneven sizes up to the limit."""
    graphs = [synth.er(n, 10.0 / (n - 1), 40 + q) for q, n in enumerate([500, 8192, 3001, 64])]
    graphs.append(synth.from_edges(30, [(i, j) for i in range(30) for j in range(i + 1, 30)]))
    graphs.append(synth.from_edges(700, np.zeros((0, 2), np.uint32)))
    m = 20
    th_o, S_o = oc.ensemble_scores([(g.n, g.row_ptr, g.col) for g in graphs], m)
    out = {}
    for path in (0, 2):  # automatic (single launch), tiled CSR per step
        with B.GraphSet(graphs, path=path) as gs:
            ls, S, rep = B.ensemble_scores(gs, m, PREC[prec], report=True)
            torch.cuda.synchronize()
            out[path] = (float(ls.item()), S.cpu().numpy(), [(r.m_eff, r.status) for r in rep])
    parity.assert_scores(out[0][0], out[0][1], th_o, S_o, prec)
    assert out[0][2] == out[2][2], (out[0][2], out[2][2])
    assert out[0][2][4][0] == 1 and out[0][2][5][0] == 1 and out[0][2][0][0] == m
    e = parity.errors(out[0][0], out[0][1], out[2][0], out[2][1])
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert e["head_rel"] <= tol and e["norm_rel"] <= tol, e
