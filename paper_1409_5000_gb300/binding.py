"""Thin Python binding of libcb (argument marshalling only).

The functions ``cb_*`` mirror the C ABI declared in ``include/cb.h`` one to
one and take raw integers (device pointers, stream handles).  The helpers
below them (:class:`GraphSet`, :func:`ensemble_scores`, ...) only allocate
torch tensors for the outputs and pass their pointers; every step of the
computation runs in the CUDA library.

The library is loaded on first use.  If ``_lib/libcb.so`` has not been
built, loading raises :class:`RuntimeError`; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from ._build import cb_lib_path, INCLUDE

CB_OK, CB_ERR_ARG, CB_ERR_CUDA, CB_ERR_OOM, CB_ERR_TIMEOUT, CB_ERR_NONFINITE, CB_ERR_STATE = range(7)
CB_FP32, CB_FP64 = 0, 1
CB_REORTH = 0x100  # OR into prec: full reorthogonalisation (two Gram-Schmidt passes)
CB_VALIDATE, CB_DEVICE_PTRS, CB_CSR_ONLY, CB_TWO_PHASE = 1, 2, 4, 8
CB_MAX_M, CB_MAX_TOPK, CB_MAX_CYCLES = 128, 4096, 1024
CB_PATH_AUTO, CB_PATH_FORMATS, CB_PATH_CSR = 0, 1, 2


class CBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libcb error {code}: {msg}")
        self.code = code


class InstReport(ctypes.Structure):
    _fields_ = [("m_eff", ctypes.c_uint32), ("status", ctypes.c_int32), ("theta", ctypes.c_double),
                ("beta_last", ctypes.c_double), ("beta0", ctypes.c_double)]


_LIB = None


def lib():
    """The loaded libcb (ctypes.CDLL): the bounds-checked libcb_debug.so when
    the environment sets CB_DEBUG=1, else libcb.so."""
    global _LIB
    if _LIB is None:
        path = cb_lib_path(os.environ.get("CB_DEBUG", "0") == "1")
        if not os.path.exists(path):
            raise RuntimeError(f"{os.path.basename(path)} not built ({path}); "
                               "run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        pp = ctypes.POINTER(ctypes.c_void_p)
        L.cb_graph_upload.restype = i32
        L.cb_graph_upload.argtypes = [u32, vp, vp, pp, pp, u32, vp, ctypes.POINTER(vp)]
        L.cb_graph_free.restype = i32
        L.cb_graph_free.argtypes = [vp]
        L.cb_graph_num_instances.restype = u32
        L.cb_graph_num_instances.argtypes = [vp]
        L.cb_graph_num_nodes.restype = u32
        L.cb_graph_num_nodes.argtypes = [vp, u32]
        L.cb_graph_max_nodes.restype = u32
        L.cb_graph_max_nodes.argtypes = [vp]
        L.cb_communicability.restype = i32
        L.cb_communicability.argtypes = [vp, u32, u32, i32, vp, vp, vp, vp]
        L.cb_ensemble_scores.restype = i32
        L.cb_ensemble_scores.argtypes = [vp, u32, i32, u32, vp, vp, vp, vp]
        L.cb_ensemble_scores_restarted.restype = i32
        L.cb_ensemble_scores_restarted.argtypes = [vp, u32, u32, i32, u32, vp, vp, vp, vp]
        L.cb_topk.restype = i32
        L.cb_topk.argtypes = [vp, u32, u32, vp, vp, vp]
        L.cb_last_error.restype = ctypes.c_char_p
        L.cb_last_error.argtypes = []
        L.cb_version.restype = u32
        L.cb_version.argtypes = []
        L.cb_debug_build.restype = u32
        L.cb_debug_build.argtypes = []
        L.cb_debug_violations.restype = i32
        L.cb_debug_violations.argtypes = [ctypes.POINTER(u32), ctypes.POINTER(u64), i32]
        L.cb_scores_backward.restype = i32
        L.cb_scores_backward.argtypes = [vp, u32, i32, vp, u32, vp, vp, vp]
        L.cb_graph_generate_er.restype = i32
        L.cb_graph_generate_er.argtypes = [u32, vp, vp, u64, u32, vp, vp, ctypes.POINTER(vp)]
        L.cb_graph_generate_ws.restype = i32
        L.cb_graph_generate_ws.argtypes = [u32, vp, u32, ctypes.c_double, u64, u32, vp, vp,
                                           ctypes.POINTER(vp)]
        L.cb_graph_generate_ba.restype = i32
        L.cb_graph_generate_ba.argtypes = [u32, vp, u32, u64, u32, vp, vp, ctypes.POINTER(vp)]
        L.cb_scores_backward_budget.restype = i32
        L.cb_scores_backward_budget.argtypes = [vp, u32, i32, vp, u32, vp, vp, ctypes.c_size_t, vp]
        L.cb_graph_tune.restype = i32
        L.cb_graph_tune.argtypes = [vp, i32, ctypes.POINTER(u32), ctypes.POINTER(ctypes.c_double), vp]
        L.cb_graph_set_lanes.restype = i32
        L.cb_graph_set_lanes.argtypes = [vp, u32]
        L.cb_graph_lanes.restype = u32
        L.cb_graph_lanes.argtypes = [vp]
        L.cb_graph_set_path.restype = i32
        L.cb_graph_set_path.argtypes = [vp, i32]
        L.cb_graph_path.restype = i32
        L.cb_graph_path.argtypes = [vp]
        L.cb_subgraph_centrality.restype = i32
        L.cb_subgraph_centrality.argtypes = [vp, u32, u32, i32, u32, vp, vp, vp, vp]
        L.cb_graph_read.restype = i32
        L.cb_graph_read.argtypes = [vp, u32, vp, vp, vp]
        L.cb_graph_num_entries.restype = u64
        L.cb_graph_num_entries.argtypes = [vp, u32]
        L.cb_release_cached_memory.restype = i32
        L.cb_release_cached_memory.argtypes = []
        L.cb_set_memory_limit.restype = i32
        L.cb_set_memory_limit.argtypes = [ctypes.c_size_t]
        L.cb_memory_in_use.restype = ctypes.c_size_t
        L.cb_memory_in_use.argtypes = []
        L.cb_debug_stall_tile.restype = i32
        L.cb_debug_stall_tile.argtypes = [vp, u32]
        L.cb_topk_noalloc.restype = i32
        L.cb_topk_noalloc.argtypes = [vp, u32, u32, vp, vp, vp]
        L.cb_score_sum.restype = i32
        L.cb_score_sum.argtypes = [vp, u32, vp, u32, vp, vp]
        L.cb_grad_rescale.restype = i32
        L.cb_grad_rescale.argtypes = [vp, u64, vp, vp, vp, vp]
        L.cb_profile_enable.restype = i32
        L.cb_profile_enable.argtypes = [i32]
        L.cb_profile_read.restype = i32
        L.cb_profile_read.argtypes = [i32, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_uint64)]
        _LIB = L
    return _LIB


def declared_functions():
    """Names of the functions declared in include/*.h."""
    names = []
    for fn in sorted(os.listdir(INCLUDE)):
        if fn.endswith(".h"):
            with open(os.path.join(INCLUDE, fn)) as f:
                src = f.read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(cb_\w+)\s*\(", src, flags=re.M)
    return names


def _check(rc):
    if rc != CB_OK:
        raise CBError(rc, lib().cb_last_error().decode(errors="replace"))


def _stream_handle(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


# ---------------------------------------------------------------------------
# One-to-one wrappers of the C ABI
# ---------------------------------------------------------------------------

def cb_graph_upload(n, nnz, row_ptr_ptrs, col_ptrs, flags, stream):
    """Returns the handle (int).  Pointer lists hold integers."""
    N = len(n)
    n_arr = np.ascontiguousarray(n, dtype=np.uint32)
    nnz_arr = np.ascontiguousarray(nnz, dtype=np.uint64)
    rp = (ctypes.c_void_p * N)(*[ctypes.c_void_p(int(p)) for p in row_ptr_ptrs])
    cp = (ctypes.c_void_p * N)(*[ctypes.c_void_p(int(p)) for p in col_ptrs])
    out = ctypes.c_void_p()
    _check(lib().cb_graph_upload(N, n_arr.ctypes.data, nnz_arr.ctypes.data,
                                 ctypes.cast(rp, ctypes.POINTER(ctypes.c_void_p)),
                                 ctypes.cast(cp, ctypes.POINTER(ctypes.c_void_p)), flags,
                                 ctypes.c_void_p(stream), ctypes.byref(out)))
    return out.value


def cb_graph_free(h):
    _check(lib().cb_graph_free(ctypes.c_void_p(h)))


def cb_graph_generate_er(n, m_draws, seed, tedges, stream):
    """Returns the handle (int).  tedges: None or an (E, 2) integer array."""
    N = len(n)
    n_arr = np.ascontiguousarray(n, dtype=np.uint32)
    m_arr = np.ascontiguousarray(m_draws, dtype=np.uint64)
    te = np.zeros((0, 2), np.uint32) if tedges is None else np.ascontiguousarray(tedges, dtype=np.uint32).reshape(-1, 2)
    te_buf = te if len(te) else np.zeros((1, 2), np.uint32)
    out = ctypes.c_void_p()
    _check(lib().cb_graph_generate_er(N, n_arr.ctypes.data, m_arr.ctypes.data, seed & (2**64 - 1),
                                      len(te), te_buf.ctypes.data, ctypes.c_void_p(stream),
                                      ctypes.byref(out)))
    return out.value


def _target_buf(tedges):
    te = np.zeros((0, 2), np.uint32) if tedges is None else np.ascontiguousarray(tedges, dtype=np.uint32).reshape(-1, 2)
    return te, (te if len(te) else np.zeros((1, 2), np.uint32))


def cb_graph_generate_ws(n, k, p, seed, tedges, stream):
    """Returns the handle (int).  tedges: None or an (E, 2) integer array."""
    n_arr = np.ascontiguousarray(n, dtype=np.uint32)
    te, te_buf = _target_buf(tedges)
    out = ctypes.c_void_p()
    _check(lib().cb_graph_generate_ws(len(n_arr), n_arr.ctypes.data, int(k), float(p),
                                      seed & (2**64 - 1), len(te), te_buf.ctypes.data,
                                      ctypes.c_void_p(stream), ctypes.byref(out)))
    return out.value


def cb_graph_generate_ba(n, m, seed, tedges, stream):
    """Returns the handle (int).  tedges: None or an (E, 2) integer array."""
    n_arr = np.ascontiguousarray(n, dtype=np.uint32)
    te, te_buf = _target_buf(tedges)
    out = ctypes.c_void_p()
    _check(lib().cb_graph_generate_ba(len(n_arr), n_arr.ctypes.data, int(m), seed & (2**64 - 1),
                                      len(te), te_buf.ctypes.data, ctypes.c_void_p(stream),
                                      ctypes.byref(out)))
    return out.value


def cb_scores_backward_budget(h, m, prec, topk_idx_ptr, k, grad_ptr, log_scale_ptr, mem_budget,
                              stream):
    _check(lib().cb_scores_backward_budget(ctypes.c_void_p(h), m, prec, ctypes.c_void_p(topk_idx_ptr),
                                           k, ctypes.c_void_p(grad_ptr),
                                           ctypes.c_void_p(log_scale_ptr), mem_budget,
                                           ctypes.c_void_p(stream)))


def cb_graph_tune(h, prec, stream):
    """Returns (lanes kept, [ms per candidate: widths 1, 2, 4, 8, 16, 32 on the
    tiled-CSR path, then the format path, then the single launch of a small
    handle; -1 = not timed]).  The path kept is cb_graph_path(h)."""
    lanes = ctypes.c_uint32()
    ms = (ctypes.c_double * 8)()
    _check(lib().cb_graph_tune(ctypes.c_void_p(h), prec, ctypes.byref(lanes), ms,
                               ctypes.c_void_p(stream)))
    return int(lanes.value), list(ms)


def cb_graph_set_lanes(h, lanes):
    _check(lib().cb_graph_set_lanes(ctypes.c_void_p(h), lanes))


def cb_graph_lanes(h):
    return int(lib().cb_graph_lanes(ctypes.c_void_p(h)))


def cb_graph_set_path(h, path):
    _check(lib().cb_graph_set_path(ctypes.c_void_p(h), path))


def cb_graph_path(h):
    return int(lib().cb_graph_path(ctypes.c_void_p(h)))


def cb_subgraph_centrality(h, inst, m, prec, k, nodes_ptr, sc_ptr, log_scale_ptr, stream):
    _check(lib().cb_subgraph_centrality(ctypes.c_void_p(h), inst, m, prec, k,
                                        ctypes.c_void_p(nodes_ptr), ctypes.c_void_p(sc_ptr),
                                        ctypes.c_void_p(log_scale_ptr), ctypes.c_void_p(stream)))


def subgraph_centrality(gs, inst: int, m: int, nodes, prec: int = CB_FP32, stream=None):
    """(log_scale, sc) with SC(nodes[q]) = (e^A)_ii ~= exp(log_scale) * sc[q] (eq. 3)."""
    import torch

    nodes = torch.as_tensor(np.asarray(nodes, dtype=np.int64).astype(np.int32), device="cuda")
    sc = torch.empty(nodes.numel(), dtype=torch.float64, device="cuda")
    ls = torch.empty(1, dtype=torch.float64, device="cuda")
    cb_subgraph_centrality(gs.h, inst, m, prec, nodes.numel(), nodes.data_ptr(), sc.data_ptr(),
                           ls.data_ptr(), _stream_handle(stream))
    return ls, sc


def cb_graph_read(h, r, row_ptr_ptr, col_ptr, stream):
    _check(lib().cb_graph_read(ctypes.c_void_p(h), r, ctypes.c_void_p(row_ptr_ptr),
                               ctypes.c_void_p(col_ptr), ctypes.c_void_p(stream)))


def read_graph(gs, r, stream=None):
    """Realisation r of a handle as host numpy arrays (row_ptr, col)."""
    rp = np.empty(gs.n[r] + 1, dtype=np.uint32)
    col = np.empty(max(gs.nnz[r], 1), dtype=np.uint32)
    cb_graph_read(gs.h, r, rp.ctypes.data, col.ctypes.data, _stream_handle(stream))
    return rp, col[:gs.nnz[r]]


def cb_graph_num_entries(h, r):
    return int(lib().cb_graph_num_entries(ctypes.c_void_p(h), r))


def cb_graph_num_instances(h):
    return int(lib().cb_graph_num_instances(ctypes.c_void_p(h)))


def cb_graph_num_nodes(h, r):
    return int(lib().cb_graph_num_nodes(ctypes.c_void_p(h), r))


def cb_graph_max_nodes(h):
    return int(lib().cb_graph_max_nodes(ctypes.c_void_p(h)))


def cb_release_cached_memory():
    _check(lib().cb_release_cached_memory())


def cb_communicability(h, inst, m, prec, y_ptr, log_scale_ptr, report, stream):
    rep = ctypes.c_void_p(ctypes.addressof(report)) if report is not None else None
    _check(lib().cb_communicability(ctypes.c_void_p(h), inst, m, prec, ctypes.c_void_p(y_ptr),
                                    ctypes.c_void_p(log_scale_ptr), rep, ctypes.c_void_p(stream)))


def cb_ensemble_scores(h, m, prec, n_out, S_ptr, log_scale_ptr, report, stream):
    rep = ctypes.c_void_p(ctypes.addressof(report)) if report is not None else None
    _check(lib().cb_ensemble_scores(ctypes.c_void_p(h), m, prec, n_out, ctypes.c_void_p(S_ptr),
                                    ctypes.c_void_p(log_scale_ptr), rep, ctypes.c_void_p(stream)))


def cb_ensemble_scores_restarted(h, m, cycles, prec, n_out, S_ptr, log_scale_ptr, report, stream):
    rep = ctypes.c_void_p(ctypes.addressof(report)) if report is not None else None
    _check(lib().cb_ensemble_scores_restarted(ctypes.c_void_p(h), m, cycles, prec, n_out,
                                              ctypes.c_void_p(S_ptr), ctypes.c_void_p(log_scale_ptr),
                                              rep, ctypes.c_void_p(stream)))


def cb_topk(S_ptr, n, k, idx_ptr, val_ptr, stream):
    _check(lib().cb_topk(ctypes.c_void_p(S_ptr), n, k, ctypes.c_void_p(idx_ptr),
                         ctypes.c_void_p(val_ptr), ctypes.c_void_p(stream)))


def cb_set_memory_limit(nbytes):
    _check(lib().cb_set_memory_limit(int(nbytes)))


def cb_memory_in_use():
    return int(lib().cb_memory_in_use())


def cb_debug_stall_tile(h, btile):
    _check(lib().cb_debug_stall_tile(ctypes.c_void_p(h), btile))


def cb_topk_noalloc(S_ptr, n, k, idx_ptr, val_ptr, stream):
    _check(lib().cb_topk_noalloc(ctypes.c_void_p(S_ptr), n, k, ctypes.c_void_p(idx_ptr),
                                 ctypes.c_void_p(val_ptr), ctypes.c_void_p(stream)))


CB_K_SPMV, CB_K_FINALIZE, CB_K_TRIDIAG, CB_K_COMBINE, CB_K_TOPK, CB_K_INIT, CB_K_BACKWARD = range(7)
CB_MAX_M_ADJOINT = 64


def cb_scores_backward(h, m, prec, topk_idx_ptr, k, grad_ptr, log_scale_ptr, stream):
    _check(lib().cb_scores_backward(ctypes.c_void_p(h), m, prec, ctypes.c_void_p(topk_idx_ptr), k,
                                    ctypes.c_void_p(grad_ptr), ctypes.c_void_p(log_scale_ptr),
                                    ctypes.c_void_p(stream)))


def cb_score_sum(S_ptr, n, nodes_ptr, k, loss_ptr, stream):
    _check(lib().cb_score_sum(ctypes.c_void_p(S_ptr), n, ctypes.c_void_p(nodes_ptr), k,
                              ctypes.c_void_p(loss_ptr), ctypes.c_void_p(stream)))


def cb_grad_rescale(grad_ptr, count, ls_grad_ptr, ls_ref_ptr, grad_out_ptr, stream):
    _check(lib().cb_grad_rescale(ctypes.c_void_p(grad_ptr), count, ctypes.c_void_p(ls_grad_ptr),
                                 ctypes.c_void_p(ls_ref_ptr), ctypes.c_void_p(grad_out_ptr),
                                 ctypes.c_void_p(stream)))


def cb_profile_enable(on):
    _check(lib().cb_profile_enable(int(bool(on))))


def cb_profile_read(kernel):
    """(total_ms, launches) of one kernel family since cb_profile_enable(1)."""
    t = ctypes.c_double()
    c = ctypes.c_uint64()
    _check(lib().cb_profile_read(kernel, ctypes.byref(t), ctypes.byref(c)))
    return t.value, c.value


def cb_last_error():
    return lib().cb_last_error().decode(errors="replace")


def cb_version():
    return int(lib().cb_version())


def cb_debug_build():
    """1 if the loaded library is the bounds-checked build, else 0."""
    return int(lib().cb_debug_build())


def cb_debug_violations(reset=False):
    """(count, first) of the debug build's failed device checks since the
    last reset; ``first`` = (site << 48) | index of the first one."""
    c, f = ctypes.c_uint32(), ctypes.c_uint64()
    _check(lib().cb_debug_violations(ctypes.byref(c), ctypes.byref(f), 1 if reset else 0))
    return int(c.value), int(f.value)


# ---------------------------------------------------------------------------
# Convenience layer over torch tensors (allocation + pointers only)
# ---------------------------------------------------------------------------

def _ptr(a):
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


class GraphSet:
    """A handle holding N realisations on the current CUDA device."""

    def __init__(self, graphs, validate=False, stream=None, csr_only=False, two_phase=False,
                 path=None):
        """`graphs`: sequence of objects with .n, .row_ptr, .col (numpy uint32
        arrays, host or pinned torch tensors, or CUDA torch tensors; CUDA
        arrays hold exactly nnz columns, and the upload reads them in order on
        `stream`, so they may still be in the making there).
        `csr_only`: no column-blocked or two-phase format (CB_CSR_ONLY).
        `two_phase`: the two-phase format for every realisation (CB_TWO_PHASE).
        `path`: FP32 SpMV path (CB_PATH_*; default CB_PATH_AUTO)."""
        import torch

        graphs = list(graphs)
        dev = [hasattr(g.col, "is_cuda") and g.col.is_cuda for g in graphs]
        if any(dev) and not all(dev):
            raise ValueError("all realisations must be on the host or all on the device")
        flags = ((CB_VALIDATE if validate else 0) | (CB_DEVICE_PTRS if all(dev) else 0)
                 | (CB_CSR_ONLY if csr_only else 0) | (CB_TWO_PHASE if two_phase else 0))
        keep = []
        rps, cols = [], []
        for g in graphs:
            rp, c = g.row_ptr, g.col
            if not hasattr(rp, "data_ptr"):
                rp = np.ascontiguousarray(rp, dtype=np.uint32)
                c = np.ascontiguousarray(c, dtype=np.uint32)
                if c.size == 0:
                    c = np.zeros(1, np.uint32)
            keep += [rp, c]
            rps.append(_ptr(rp))
            cols.append(_ptr(c))
        n = [int(g.n) for g in graphs]
        # no read of a device row_ptr here: it would wait for `stream`'s work
        nnz = [int(g.col.numel()) if d else int(g.row_ptr[-1]) for g, d in zip(graphs, dev)]
        self.n = n
        self.nnz = nnz
        self.n_max = max(n)
        self.device = torch.cuda.current_device()
        self.h = cb_graph_upload(n, nnz, rps, cols, flags, _stream_handle(stream))
        if path is not None:
            cb_graph_set_path(self.h, path)

    @classmethod
    def generate_er(cls, n, dbar, seed, target_edges=None, stream=None):
        """N Erdos-Renyi backgrounds generated on the device (cb_graph_generate_er).
        `n`: nodes per realisation; `dbar`: mean degree (scalar or per
        realisation), m_draws = floor(dbar * n / 2 + 1/2)."""
        import torch

        n = [int(x) for x in n]
        dbar = list(dbar) if hasattr(dbar, "__len__") else [dbar] * len(n)
        m = [int(np.floor(float(d) * float(x) * 0.5 + 0.5)) for d, x in zip(dbar, n)]
        self = cls.__new__(cls)
        self.device = torch.cuda.current_device()
        self.h = cb_graph_generate_er(n, m, seed, target_edges, _stream_handle(stream))
        self.n = n
        self.nnz = [cb_graph_num_entries(self.h, r) for r in range(len(n))]
        self.n_max = max(n)
        return self

    @classmethod
    def _from_handle(cls, h, n):
        import torch

        self = cls.__new__(cls)
        self.device = torch.cuda.current_device()
        self.h = h
        self.n = [int(x) for x in n]
        self.nnz = [cb_graph_num_entries(self.h, r) for r in range(len(self.n))]
        self.n_max = max(self.n)
        return self

    @classmethod
    def generate_ws(cls, n, k, p, seed, target_edges=None, stream=None):
        """N Watts-Strogatz backgrounds generated on the device (cb_graph_generate_ws)."""
        n = [int(x) for x in n]
        return cls._from_handle(cb_graph_generate_ws(n, k, p, seed, target_edges,
                                                     _stream_handle(stream)), n)

    @classmethod
    def generate_ba(cls, n, m, seed, target_edges=None, stream=None):
        """N Barabasi-Albert backgrounds generated on the device (cb_graph_generate_ba)."""
        n = [int(x) for x in n]
        return cls._from_handle(cb_graph_generate_ba(n, m, seed, target_edges,
                                                     _stream_handle(stream)), n)

    def close(self):
        h = getattr(self, "h", None)
        if h:
            self.h = None  # the handle is gone even if the free reports an error
            cb_graph_free(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def communicability(gs: GraphSet, inst: int, m: int, prec: int = CB_FP32, stream=None,
                    report: bool = False):
    """(log_scale, y) with e^A 1 ~= exp(log_scale) * y for realisation inst."""
    import torch

    y = torch.empty(gs.n[inst], dtype=torch.float64, device="cuda")
    ls = torch.empty(1, dtype=torch.float64, device="cuda")
    rep = InstReport() if report else None
    cb_communicability(gs.h, inst, m, prec, y.data_ptr(), ls.data_ptr(), rep,
                       _stream_handle(stream))
    return (ls, y, rep) if report else (ls, y)


def ensemble_scores(gs: GraphSet, m: int, prec: int = CB_FP32, n_out=None, out=None,
                    stream=None, report: bool = False):
    """(log_scale, S) with sum_r e^{A_r} 1 ~= exp(log_scale) * S (eq. 5)."""
    import torch

    n_out = gs.n_max if n_out is None else n_out
    if out is None:
        S = torch.empty(n_out, dtype=torch.float64, device="cuda")
        ls = torch.empty(1, dtype=torch.float64, device="cuda")
    else:
        S, ls = out
    rep = (InstReport * len(gs.n))() if report else None
    cb_ensemble_scores(gs.h, m, prec, n_out, S.data_ptr(), ls.data_ptr(), rep,
                       _stream_handle(stream))
    return (ls, S, list(rep)) if report else (ls, S)


def ensemble_scores_restarted(gs: GraphSet, m: int, cycles: int, prec: int = CB_FP32, n_out=None,
                              out=None, stream=None, report: bool = False):
    """(log_scale, S) as ensemble_scores, each e^{A_r} 1 by `cycles` restarted
    Lanczos cycles of m steps (block bidiagonal form of the restarted method)."""
    import torch

    n_out = gs.n_max if n_out is None else n_out
    if out is None:
        S = torch.empty(n_out, dtype=torch.float64, device="cuda")
        ls = torch.empty(1, dtype=torch.float64, device="cuda")
    else:
        S, ls = out
    rep = (InstReport * len(gs.n))() if report else None
    cb_ensemble_scores_restarted(gs.h, m, cycles, prec, n_out, S.data_ptr(), ls.data_ptr(), rep,
                                 _stream_handle(stream))
    return (ls, S, list(rep)) if report else (ls, S)


def topk(S, k: int, out=None, stream=None):
    """(idx uint32 as int32 tensor, val float64) of the k largest entries."""
    import torch

    if out is None:
        idx = torch.empty(k, dtype=torch.int32, device=S.device)
        val = torch.empty(k, dtype=torch.float64, device=S.device)
    else:
        idx, val = out
    cb_topk(S.data_ptr(), S.numel(), k, idx.data_ptr(), val.data_ptr(), _stream_handle(stream))
    return idx, val


def scores_backward(gs: GraphSet, m: int, nodes, prec: int = CB_FP32, stream=None):
    """(log_scale, grad) with d/da_e sum_r sum_{i in nodes} EBTC_r(i) =
    exp(log_scale) * grad[e], grad float32 over all CSR entries of the
    handle (realisations concatenated)."""
    import torch

    nodes = torch.as_tensor(nodes, dtype=torch.int32, device="cuda").contiguous()
    grad = torch.empty(sum(gs.nnz), dtype=torch.float32, device="cuda")
    ls = torch.empty(1, dtype=torch.float64, device="cuda")
    cb_scores_backward(gs.h, m, prec, nodes.data_ptr(), nodes.numel(), grad.data_ptr(),
                       ls.data_ptr(), _stream_handle(stream))
    return ls, grad


def _summed_topk_function():
    import torch

    class SummedTopkScore(torch.autograd.Function):
        """Loss = sum_r sum_{i in nodes} EBTC_r(i), scaled by exp(-log_scale),
        as a function of the (unit) edge weights of the handle's pattern.

        forward(edge_weight, gs, m, nodes, prec) -> scaled loss (float64 0-dim),
        the summed scores of the nodes (cb_ensemble_scores + cb_score_sum).
        backward gives d loss / d edge_weight: cb_scores_backward, brought to
        the forward's units and multiplied by the upstream gradient by
        cb_grad_rescale (the edge-sensitivity map of the recovered sub-graph).
        The store is pattern-only: the scores are those of unit weights, so
        edge_weight must be all ones (anything else raises ValueError).
        """

        @staticmethod
        def forward(ctx, edge_weight, gs, m, nodes, prec=CB_FP32):
            if edge_weight.numel() != sum(gs.nnz):
                raise ValueError("edge_weight must have one entry per CSR entry of the handle")
            if not bool(torch.all(edge_weight == 1)):
                raise ValueError("edge_weight must be all ones: the adjacency store is pattern-only, "
                                 "so scores and gradients are those of unit weights")
            ls, S = ensemble_scores(gs, m, prec)
            nodes_t = torch.as_tensor(np.asarray(nodes, dtype=np.int64).astype(np.int32),
                                      device=S.device)
            loss = torch.empty((), dtype=torch.float64, device=S.device)
            cb_score_sum(S.data_ptr(), S.numel(), nodes_t.data_ptr(), nodes_t.numel(),
                         loss.data_ptr(), _stream_handle(None))
            ctx.gs, ctx.m, ctx.nodes, ctx.prec = gs, m, nodes, prec
            ctx.save_for_backward(ls)
            return loss

        @staticmethod
        def backward(ctx, grad_out):
            (ls_fwd,) = ctx.saved_tensors
            ls_bw, grad = scores_backward(ctx.gs, ctx.m, ctx.nodes, ctx.prec)
            go = grad_out.to(dtype=torch.float64, device=grad.device).contiguous()
            cb_grad_rescale(grad.data_ptr(), grad.numel(), ls_bw.data_ptr(), ls_fwd.data_ptr(),
                            go.data_ptr(), _stream_handle(None))
            return grad, None, None, None, None

    return SummedTopkScore


_FN = None


def summed_topk_score(edge_weight, gs: GraphSet, m: int, nodes, prec: int = CB_FP32):
    """Autograd entry: scaled sum of the summed scores of `nodes` (see above)."""
    global _FN
    if _FN is None:
        _FN = _summed_topk_function()
    return _FN.apply(edge_weight, gs, m, nodes, prec)
