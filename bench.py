"""Benchmark: summed Lanczos total communicability + top-k on one GB300.

One step = one pass of the hot path over one batch of synthetic input:
the Krylov (Lanczos) approximation of e^{A_r} 1 for every realisation r
(paper eq. 4 and its Krylov evaluation), the ensemble sum (eq. 5) and the
top-k selection, i.e. cb_ensemble_scores + cb_topk.

Default workload: 256 Erdos-Renyi realisations with n drawn uniformly from
[20 000, 400 000] (mean degree 20, ~1.0e9 directed CSR entries in total), a
30-node sparse target (random tree + 15 edges) OR-ed into each, Krylov depth
m = 25, FP32 Krylov vectors with FP64 scalars and sums, top-30.

Metric: edge-Lanczos-steps/s = (sum_r nnz_r * m) / time per step.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       [--workload ensemble|large|small] [--skip-extra]
With N > 1 it expects torchrun (one process per GPU); every rank runs the
same workload as an independent replica (weak scaling, no collective on the
data path) and rank 0 prints the JSON line.
"""
from __future__ import annotations

import os

# The oracle (CPU baseline / reference arm) is timed single-threaded.
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse  # noqa: E402
import json  # noqa: E402
import math  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import tempfile  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1409_5000_gb300 import synth  # noqa: E402

METRIC = "edge-Lanczos-steps/s"
UNIT = "edge*steps/s"


def workload(name):
    if name == "ensemble":
        ens = synth.er_ensemble_uneven()
        desc = dict(workload="er-ensemble-256-uneven-n20k-400k-d20-m25", n_inst=256,
                    n_range=[20_000, 400_000], dbar=20, target="tree30+15", m=25, k=30)
    elif name == "ensemble40":
        # the first 40 realisations' recipe of the default workload: the small
        # case for ncu captures (cols ~0.6 GB, still larger than L2)
        ens = synth.er_ensemble_uneven(n_inst=40)
        desc = dict(workload="er-ensemble-40-uneven-n20k-400k-d20-m25", n_inst=40,
                    n_range=[20_000, 400_000], dbar=20, target="tree30+15", m=25, k=30)
    elif name == "large":
        ens = synth.ba_clique_large()
        desc = dict(workload="ba-1e7-m8-clique20-m40", n_inst=1, n=10_000_000, ba_m=8,
                    target="clique20", m=40, k=20)
    elif name == "large2m":
        # the same recipe at n = 2e6 (3.2e7 entries, value array ~0.13 GB, larger
        # than L2): the small case for ncu captures of the two-phase kernels
        ens = synth.ba_clique_large(n=2_000_000)
        desc = dict(workload="ba-2e6-m8-clique20-m40", n_inst=1, n=2_000_000, ba_m=8,
                    target="clique20", m=40, k=20)
    elif name in ("c2er", "c2ba", "c2ws"):
        kind = name[2:]
        ens = synth.single_clique_100k(kind)
        desc = dict(workload=f"{kind}-1e5-clique12-m30", n_inst=1, n=100_000, target="clique12",
                    m=30, k=12, background={"er": "ER d=10", "ba": "BA m0=m=5",
                                            "ws": "WS k=10 p=0.1"}[kind])
    elif name == "grad":
        ens = synth.er_ensemble_grad()
        desc = dict(workload="er-ensemble-64x1e5-d16-m30-fwd+bwd", n_inst=64, n=100_000, dbar=16,
                    target="tree25+10", m=30, k=25,
                    step="ensemble scores + top-k + edge gradient of the top-k score")
    elif name == "small":
        ens = synth.er_ensemble_small()
        desc = dict(workload="er-ensemble-10x500-p0.016-m20", n_inst=10, n=500, p=0.016,
                    target="tree15+8", m=20, k=15)
    else:
        raise SystemExit(f"unknown workload {name}")
    return ens, desc


# DRAM bytes per CSR entry of the dominant SpMV kernel(s), from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum): the column-blocked
# kernel on the 40-realisation case of the default recipe, and the two
# phases of the two-phase kernel on the large graph.  Reported only while the
# source that decides the traffic (kernels, epilogue, format builder,
# constants) still hashes to the captured version.
_TRAFFIC = {
    # one launch on the 40-realisation case: 703.01 MB read + 20.04 MB written
    "blocked": {"sources_sha256_16": "4ce8ff9dadfd2966", "bytes_per_edge": (703.01e6 + 20.04e6) / 151654698,
                "kernel": "bspmv_kernel", "captured_on": "er-ensemble-40"},
    # one launch of each phase on the 10M-node graph: phase 1 492.12 MB read +
    # 661.91 MB written, phase 2 1173.79 MB read + 34.77 MB written
    "twophase": {"sources_sha256_16": "3be61c496ed83da9",
                 "bytes_per_edge": (492.12e6 + 661.91e6 + 1173.79e6 + 34.77e6) / 160000252,
                 "kernel": "pscatter_kernel + pgather_kernel", "captured_on": "ba-1e7"},
}


def _cut(text, start, end_marker):
    a = text.index(start)
    return text[a:text.index(end_marker, a)]


def _kernel_sources_hash(kind="blocked"):
    """Hash of the source that decides an SpMV path's memory traffic: its
    kernels and staging helpers, the row epilogue, its format builder and its
    constants."""
    import hashlib
    import re

    csrc = os.path.join(ROOT, "paper_1409_5000_gb300", "csrc")

    def rd(name):
        with open(os.path.join(csrc, name)) as f:
            return f.read()

    step = rd("cb_step.cuh")
    parts = [_cut(step, "__device__ __forceinline__ T row_epilogue", "\n}\n"),
             _cut(step, "// mbarrier and bulk-copy helpers", "// Two-phase SpMV step of")]
    consts = rd("cb_internal.cuh")
    if kind == "blocked":
        lz = rd("cb_lanczos.cu")
        parts.append(_cut(lz, "constexpr size_t kBSmemBytes", "// w = W_{j+1} - alpha_j"))
        bl = rd("cb_blocked.cu")  # the count and fill kernels (host code does not change the format)
        parts.append(_cut(bl, "__global__", "size_t fill_smem_bytes"))
        parts += re.findall(r"^constexpr [^\n]*\bk(?:B\w*|Threads|Group)\b[^\n]*$", consts, re.M)
    else:
        tp = rd("cb_twophase.cu")
        parts.append(_cut(tp, "__global__", "template <typename P>"))
        parts += re.findall(r"^constexpr [^\n]*\bk(?:P\w*|HeavyDeg|LongDeg|Chunk|Group)\b[^\n]*$",
                            consts, re.M)
    h = hashlib.sha256()
    for p in parts:
        h.update(p.encode())
    return h.hexdigest()[:16]


def traffic_per_launch(ens, kind):
    t = _TRAFFIC[kind]
    if t["bytes_per_edge"] is None or _kernel_sources_hash(kind) != t["sources_sha256_16"]:
        return None
    return t["bytes_per_edge"] * sum(g.nnz for g in ens.graphs)


def alg_bytes_spmv(ens, fp64=False):
    """Algorithmic bytes of one Lanczos SpMV launch over all realisations:
    4 nnz (u32 cols) + 4 (n+1) (row_ptr) + 3 n vector elements (read v_j,
    read v_{j-1}, write u), FP32 (FP64) elements."""
    esz = 8 if fp64 else 4
    return sum(4 * g.nnz + 4 * (g.n + 1) + 3 * esz * g.n for g in ens.graphs)


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_oracle_sample(ens, m, budget_s=15.0, max_inst=None, want=None):
    """Time the FP64 oracle (as it stands) on the first realisations of the
    workload until ~budget_s of CPU time; returns (value, sample, results)."""
    import oracle.communicability as oc

    t_tot, units, done, results = 0.0, 0, 0, {}
    for r, g in enumerate(ens.graphs):
        if max_inst is not None and done >= max_inst:
            break
        t0 = time.perf_counter()
        theta, y, _ = oc.krylov_expv(g.n, g.row_ptr, g.col, m)
        t_tot += time.perf_counter() - t0
        units += g.nnz * m
        done += 1
        if want is not None and r in want:
            results[r] = (theta, y)
        if t_tot >= budget_s:
            break
    return units / t_tot, done, t_tot, results


# --- the oracle on all host cores: realisations are independent terms of
# eq. 5, so a spawn pool runs them side by side (each worker single-threaded,
# the CSR shared through one shared-memory block, nothing large pickled).
_ORACLE_SHM = {}


def _oracle_attach(name, layout):
    from multiprocessing import shared_memory

    _ORACLE_SHM["shm"] = shared_memory.SharedMemory(name=name)
    _ORACLE_SHM["layout"] = layout


def _oracle_one(args):
    import oracle.communicability as oc

    r, m = args
    n, rp_off, col_off, nnz = _ORACLE_SHM["layout"][r]
    buf = _ORACLE_SHM["shm"].buf
    rp = np.frombuffer(buf, dtype=np.uint32, count=n + 1, offset=rp_off)
    col = np.frombuffer(buf, dtype=np.uint32, count=nnz, offset=col_off)
    t0 = time.perf_counter()
    oc.krylov_expv(n, rp, col, m)
    return time.perf_counter() - t0


class OraclePool:
    """Spawn pool over the first n_inst realisations of a workload."""

    def __init__(self, graphs, procs=None):
        import multiprocessing as mp
        from multiprocessing import shared_memory

        self.graphs = list(graphs)
        size = sum(4 * (g.n + 1) + 4 * g.nnz for g in self.graphs)
        self.shm = shared_memory.SharedMemory(create=True, size=max(size, 16))
        layout, o = [], 0
        for g in self.graphs:
            a = np.frombuffer(self.shm.buf, dtype=np.uint32, count=g.n + 1, offset=o)
            a[:] = g.row_ptr
            b = np.frombuffer(self.shm.buf, dtype=np.uint32, count=g.nnz, offset=o + 4 * (g.n + 1))
            b[:] = g.col
            layout.append((g.n, o, o + 4 * (g.n + 1), g.nnz))
            o += 4 * (g.n + 1) + 4 * g.nnz
            del a, b
        self.procs = procs or min(os.cpu_count() or 1, 64)
        self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_oracle_attach,
                                                 initargs=(self.shm.name, layout))

    def run(self, m, rs):
        """Wall seconds to evaluate realisations rs (and the summed busy time)."""
        t0 = time.perf_counter()
        busy = self.pool.map(_oracle_one, [(r, m) for r in rs], chunksize=1)
        return time.perf_counter() - t0, sum(busy)

    def close(self):
        self.pool.close()
        self.pool.join()
        self.shm.close()
        self.shm.unlink()


def combine_ranks(ms, units, dist=None, device="cpu"):
    """Whole-job figures over ranks: the slowest rank's ms per step, and the
    units all ranks processed per step divided by it."""
    if dist is None:
        return ms, units / (ms * 1e-3)
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    ms = float(t.item())
    return ms, float(u.item()) / (ms * 1e-3)


def run_reference(args, ens, desc, rank, world):
    if rank != 0:
        return
    m = desc["m"]
    if desc["workload"].startswith("ba-1e7"):
        raise SystemExit("reference arm on the 1e7-node graph takes minutes per step; use the default")
    # each step: the oracle on a bounded sample of the workload's realisations,
    # all host cores (one realisation per worker at a time)
    pool = OraclePool(ens.graphs[: min(len(ens.graphs), 4 * (os.cpu_count() or 1))])
    try:
        per_step = len(pool.graphs)
        rs = list(range(per_step))
        for _ in range(args.warmup):
            pool.run(m, rs[: pool.procs])
        dt = 0.0
        for _ in range(args.steps):
            dt += pool.run(m, rs)[0]
    finally:
        pool.close()
    units = args.steps * sum(g.nnz * m for g in ens.graphs[:per_step])
    value = units / dt
    sample = (f"first {per_step} of {len(ens.graphs)} realisations per step, FP64 Lanczos with full "
              f"reorthogonalisation, m={m}, {pool.procs} worker processes")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": dict(desc, sample=f"first {per_step} realisations per step"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


_FAMILIES = ["spmv", "finalize", "tridiag", "combine", "topk", "init", "backward"]


def kernel_families(B, step, steps):
    """Per-family device time (ms) and launch count over `steps` steps, from
    the library's CUDA events recorded on the launching stream."""
    import torch

    B.cb_profile_enable(1)
    for _ in range(steps):
        step()
    torch.cuda.synchronize()
    kid = {"spmv": B.CB_K_SPMV, "finalize": B.CB_K_FINALIZE, "tridiag": B.CB_K_TRIDIAG,
           "combine": B.CB_K_COMBINE, "topk": B.CB_K_TOPK, "init": B.CB_K_INIT,
           "backward": B.CB_K_BACKWARD}
    fam = {name: B.cb_profile_read(kid[name]) for name in _FAMILIES}
    B.cb_profile_enable(0)
    return fam


def spmv_path(ens, csr_only=False):
    """Which SpMV the workload runs under the automatic path: 'small' (every
    realisation at most 8192 nodes and 2^20 entries: one launch of m steps),
    'twophase' (a realisation above 2^19 nodes), 'blocked' (otherwise, when
    the handle has at least one 16384-row blocked tile per SM) or 'csr'
    (fewer tiles, or CB_CSR_ONLY)."""
    if all(g.n <= 8192 and g.nnz <= (1 << 20) for g in ens.graphs):
        return "small"
    if csr_only:
        return "csr"
    if max(g.n for g in ens.graphs) > 32 * 16384:
        return "twophase"
    import torch

    tiles = sum((g.n + 16383) // 16384 for g in ens.graphs)
    return "blocked" if tiles >= torch.cuda.get_device_properties(0).multi_processor_count else "csr"


_KERNEL_NAMES = {"small": "lanczos_small_kernel (all m Lanczos steps of a small realisation per CTA)",
                 "blocked": "bspmv_kernel (column-blocked Lanczos SpMV step)",
                 "twophase": "pscatter_kernel + pgather_kernel (two-phase Lanczos SpMV step)",
                 "csr": "spmv_kernel (tiled-CSR Lanczos SpMV step)"}


def roofline_for(ens, fam, path, m=1):
    """The roofline object of the SpMV family: algorithmic bytes of one
    launch over its average event-timed duration, against the measured HBM
    copy bandwidth.  On the 'small' path one launch runs all m steps, so its
    bytes are m SpMVs' (vector traffic beyond the SpMV's is not counted)."""
    tot = sum(t for t, _ in fam.values())
    spmv_ms, spmv_n = fam["spmv"]
    spmv_avg = spmv_ms / max(spmv_n, 1)
    peak, peak_kind = measured_peak()
    per_launch = (m if path == "small" else 1) * alg_bytes_spmv(ens)
    achieved = per_launch / (spmv_avg * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": _KERNEL_NAMES[path], "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
            "frac_of_8TBs_nominal": achieved / 8000.0,
            "traffic": traffic_per_launch(ens, path) if path in ("blocked", "twophase") else None,
            "alg_bytes_per_launch": per_launch, "avg_launch_ms": spmv_avg,
            "kernel_shares": {k: round(t / tot, 4) for k, (t, _) in fam.items()}}


def launches_for(m, path, with_grad=False, n_scores=None):
    """Kernel launches of one step: init (2) + per Lanczos step the SpMV
    (two kernels on the two-phase path), finalize and beta + tridiag +
    combine (2) + top-k (init, 12 radix passes, collect, sort; one sort of
    all scores up to 4096 of them)."""
    topk = 1 if n_scores is not None and n_scores <= 4096 else 15
    if path == "small":  # one launch for all m steps
        n = 2 + 1 + 1 + 2 + topk
        return n + (3 + 1) + 3 if with_grad else n
    per_step = (2 if path == "twophase" else 1) + 2
    n = 2 + per_step * m + 1 + 2 + topk
    if with_grad:  # the Lanczos run from the indicator (the basis from 1 is the
        # forward pass's) + 3 adjoint kernels
        n += (3 + per_step * m) + 3
    return n


def tuned_choice(B, gs, prec=0):
    """cb_graph_tune on a handle: the width and path it keeps and the ms of
    each candidate (widths 1..32 on the tiled-CSR path, then the format path)."""
    import torch

    lanes, ms = B.cb_graph_tune(gs.h, prec, torch.cuda.current_stream().cuda_stream)
    names = {B.CB_PATH_AUTO: "auto", B.CB_PATH_FORMATS: "formats", B.CB_PATH_CSR: "csr"}
    return {"lanes": lanes, "path": names.get(B.cb_graph_path(gs.h), "?"),
            "ms_per_3_step_run": {"csr_lanes_" + str(w): m for w, m in zip((1, 2, 4, 8, 16, 32), ms)} |
            {"formats": ms[6], "single_launch": ms[7]}}


def check_run(B, gs, m, prec):
    """One more call, outside the timed region, with the per-realisation
    report: a realisation that failed (a device wait that gave up, a
    non-finite recurrence scalar) makes the whole measurement invalid."""
    import torch

    ls, _, rep = B.ensemble_scores(gs, m, prec, report=True)
    torch.cuda.synchronize()
    bad = [(q, r.status) for q, r in enumerate(rep) if r.status != 0]
    if bad or not math.isfinite(float(ls.item())):
        raise RuntimeError(f"bench: realisations failed (index, status): {bad[:8]}; "
                           f"log scale {float(ls.item())}")


def budgeted_backward(B, gs, m, prec, idx, k, grad, gls, stream):
    """The adjoint of the same top-k under a budget of a quarter of its working
    set (cb_scores_backward_budget: groups of realisations, bases recomputed in
    temporary handles), timed against the unbudgeted call; both synchronous."""
    import torch

    r4 = (m + 3) // 4 * 4
    esz = 8 if prec == 1 else 4
    ws = sum(esz * n * (2 * (m + 1) + 2 * r4) for n in gs.n) + 12 * sum(gs.nnz)
    g2 = torch.empty_like(grad)
    l2 = torch.empty_like(gls)
    t = {}
    for label, budget in (("unbudgeted", 0), ("budget", ws // 4)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if budget:
            B.cb_scores_backward_budget(gs.h, m, prec, idx.data_ptr(), k, g2.data_ptr(),
                                        l2.data_ptr(), budget, stream.cuda_stream)
        else:
            B.cb_scores_backward(gs.h, m, prec, idx.data_ptr(), k, grad.data_ptr(), gls.data_ptr(),
                                 stream.cuda_stream)
        torch.cuda.synchronize()
        t[label] = 1e3 * (time.perf_counter() - t0)
    a, b = g2.double(), grad.double()
    return {"budget_bytes": ws // 4, "working_set_bytes": ws, "ms": t["budget"],
            "ms_unbudgeted": t["unbudgeted"],
            "max_abs_diff_rel": float((a - b).abs().max() / b.abs().max()),
            "api": "cb_scores_backward_budget vs cb_scores_backward, wall time of one synchronous call"}


def extra_leg(B, name, steps, warmup, dev, csr_only=False, precs=(0,), built=None, tune=False):
    """One more workload timed the way the main line is (warm-up, CUDA
    events around `steps` steps of ensemble scores + top-k (+ the edge
    gradient for 'grad'), then a profiled pass for the SpMV family).
    `built`: the (ensemble, description) pair when already generated."""
    import torch

    ens, desc = built if built is not None else workload(name)
    m, k = desc["m"], desc["k"]
    with_grad = name == "grad"
    stream = torch.cuda.current_stream()
    out = {"config": desc}
    u0 = time.perf_counter()
    gs = B.GraphSet(ens.graphs, csr_only=csr_only)
    out["upload_ms"] = 1e3 * (time.perf_counter() - u0)
    try:
        for prec in precs:
            S = torch.empty(gs.n_max, dtype=torch.float64, device=dev)
            ls = torch.empty(1, dtype=torch.float64, device=dev)
            idx = torch.empty(k, dtype=torch.int32, device=dev)
            val = torch.empty(k, dtype=torch.float64, device=dev)
            if with_grad:
                grad = torch.empty(sum(gs.nnz), dtype=torch.float32, device=dev)
                gls = torch.empty(1, dtype=torch.float64, device=dev)

            def step():
                B.ensemble_scores(gs, m, prec, out=(S, ls))
                B.topk(S, k, out=(idx, val))
                if with_grad:
                    B.cb_scores_backward(gs.h, m, prec, idx.data_ptr(), k, grad.data_ptr(),
                                         gls.data_ptr(), stream.cuda_stream)

            for _ in range(warmup):
                step()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                step()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            check_run(B, gs, m, prec)
            units = sum(g.nnz for g in ens.graphs) * m
            fam = kernel_families(B, step, steps)
            path = spmv_path(ens, csr_only)
            if path != "small" and prec == 1:
                path = "csr"
            leg = {"ms_per_step": ms, "value": units / (ms * 1e-3), "unit": UNIT,
                   "dtype": "f64" if prec == 1 else "f32", "roofline": roofline_for(ens, fam, path, m),
                   "gpu_launches_per_step": launches_for(m, path, with_grad, gs.n_max)}
            if prec == 1:  # FP64 bytes: 8-byte vector elements
                b64 = (m if path == "small" else 1) * alg_bytes_spmv(ens, fp64=True)
                leg["roofline"]["alg_bytes_per_launch"] = b64
                a = b64 / (leg["roofline"]["avg_launch_ms"] * 1e-3) / 1e9
                leg["roofline"].update(achieved=a, frac=a / leg["roofline"]["peak"],
                                       frac_of_8TBs_nominal=a / 8000.0)
            if with_grad:
                leg["backward_share"] = round(fam["backward"][0] / sum(t for t, _ in fam.values()), 4)
                leg["budgeted"] = budgeted_backward(B, gs, m, prec, idx, k, grad, gls, stream)
            leg["scores"] = (float(ls.item()), S.cpu().numpy())
            out["f64" if prec == 1 else "f32"] = leg
        if tune:
            out["tuned"] = tuned_choice(B, gs)
    finally:
        gs.close()
    if "f32" in out and "f64" in out:  # FP32 against FP64, the S10 reading (head and 2-norm)
        (la, a), (lb, b) = out["f32"]["scores"], out["f64"]["scores"]
        a = a * math.exp(la - lb)
        head = b >= 1e-3 * b.max()
        out["f32_vs_f64"] = {"head_max_rel": float(np.max(np.abs(a - b)[head] / b[head])),
                             "norm_rel": float(np.linalg.norm(a - b) / np.linalg.norm(b))}
    for p in ("f32", "f64"):
        if p in out:
            del out[p]["scores"]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ensemble", choices=["ensemble", "ensemble40", "large", "large2m", "small", "grad", "c2er", "c2ba", "c2ws"])
    ap.add_argument("--skip-extra", action="store_true",
                    help="skip the e2e, plain-FP64 and CPU-baseline legs")
    ap.add_argument("--csr-only", action="store_true",
                    help="upload without the column-blocked format (CB_CSR_ONLY): every FP32 "
                         "SpMV runs the tiled-CSR kernel")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    ens, desc = workload(args.workload)
    m, k = desc["m"], desc["k"]

    if args.impl == "reference":
        run_reference(args, ens, desc, rank, world)
        return

    import torch

    from paper_1409_5000_gb300 import binding as B

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.lib()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    units = sum(g.nnz for g in ens.graphs) * m  # edge-Lanczos-steps per step
    gs = B.GraphSet(ens.graphs, csr_only=args.csr_only)
    S = torch.empty(gs.n_max, dtype=torch.float64, device=dev)
    ls = torch.empty(1, dtype=torch.float64, device=dev)
    idx = torch.empty(k, dtype=torch.int32, device=dev)
    val = torch.empty(k, dtype=torch.float64, device=dev)

    with_grad = args.workload == "grad"
    if with_grad:
        grad = torch.empty(sum(gs.nnz), dtype=torch.float32, device=dev)
        gls = torch.empty(1, dtype=torch.float64, device=dev)

    def step():
        B.ensemble_scores(gs, m, B.CB_FP32, out=(S, ls))
        B.topk(S, k, out=(idx, val))
        if with_grad:  # the recovered top-k (still on the device) is the node set
            B.cb_scores_backward(gs.h, m, B.CB_FP32, idx.data_ptr(), k, grad.data_ptr(),
                                 gls.data_ptr(), stream.cuda_stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    check_run(B, gs, m, B.CB_FP32)
    ms, value = combine_ranks(ms, units, dist, dev)

    # per-kernel times (CUDA events around each launch, same stream), separate pass
    fam = kernel_families(B, step, args.steps)
    path_kind = spmv_path(ens, args.csr_only)
    roofline = roofline_for(ens, fam, path_kind, m)
    launches_per_step = launches_for(m, path_kind, with_grad, gs.n_max)

    extra = {}
    if with_grad:
        extra["backward_share"] = round(fam["backward"][0] / tot, 4)
    ls1 = torch.empty(1, dtype=torch.float64, device=dev)
    if rank == 0 and not args.skip_extra:
        # plain per-graph FP64 path: one cb_communicability call per realisation
        y_out = torch.empty(gs.n_max, dtype=torch.float64, device=dev)
        for r in range(min(2, len(gs.n))):
            B.cb_communicability(gs.h, r, m, B.CB_FP64, y_out.data_ptr(), ls1.data_ptr(), None,
                                 stream.cuda_stream)
        torch.cuda.synchronize()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for r in range(len(gs.n)):
            B.cb_communicability(gs.h, r, m, B.CB_FP64, y_out.data_ptr(), ls1.data_ptr(), None,
                                 stream.cuda_stream)
        p1.record(stream)
        torch.cuda.synchronize()
        plain_ms = p0.elapsed_time(p1)
        extra["plain_fp64_per_graph"] = {"ms": plain_ms, "speedup_batched_fp32": plain_ms / ms,
                                         "note": "N x cb_communicability(FP64), ensemble sum and top-k excluded"}
        # restore the FP32 workspace before the e2e leg
        step()
        torch.cuda.synchronize()

    e2e = None
    if rank == 0 and not args.skip_extra:
        pinned = [synth.Graph(g.n, torch.from_numpy(g.row_ptr.view(np.int32)).pin_memory(),
                              torch.from_numpy(g.col.view(np.int32)).pin_memory())
                  for g in ens.graphs]
        h2d = sum(4 * (g.n + 1) + 4 * g.nnz for g in ens.graphs)
        d2h = 4 * k + 8 * k + 8
        host_idx = torch.empty(k, dtype=torch.int32).pin_memory()
        host_val = torch.empty(k, dtype=torch.float64).pin_memory()
        host_ls = torch.empty(1, dtype=torch.float64).pin_memory()

        class _PG:
            def __init__(self, g, pg):
                self.n, self.row_ptr, self.col = g.n, pg.row_ptr, pg.col

        pgs = [_PG(g, pg) for g, pg in zip(ens.graphs, pinned)]
        n_e2e = max(1, min(args.steps, 3))

        up_ms = []

        def e2e_step():
            u0 = time.perf_counter()
            with B.GraphSet(pgs) as g2:
                up_ms.append(1e3 * (time.perf_counter() - u0))  # the upload synchronises
                S2 = torch.empty(g2.n_max, dtype=torch.float64, device=dev)
                l2 = torch.empty(1, dtype=torch.float64, device=dev)
                B.ensemble_scores(g2, m, B.CB_FP32, out=(S2, l2))
                i2, v2 = B.topk(S2, k)
                host_idx.copy_(i2, non_blocking=True)
                host_val.copy_(v2, non_blocking=True)
                host_ls.copy_(l2, non_blocking=True)
                torch.cuda.synchronize()

        e2e_step()
        up_ms.clear()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        serial_ms = 1e3 * (time.perf_counter() - t0) / n_e2e

        # The same steps double-buffered, as a stream of ensembles runs: step
        # q + 1's upload (its own host thread and stream) overlaps step q's
        # compute; every step still copies its whole input from pinned host
        # memory and reads its result back inside the timed region, which
        # starts before the first upload.
        from concurrent.futures import ThreadPoolExecutor

        up_stream = torch.cuda.Stream(device=dev)

        def upload():
            return B.GraphSet(pgs, stream=up_stream)

        def pipelined(n):
            with ThreadPoolExecutor(1) as ex:
                fut = ex.submit(upload)
                for q in range(n):
                    g2 = fut.result()
                    if q + 1 < n:
                        fut = ex.submit(upload)
                    S2 = torch.empty(g2.n_max, dtype=torch.float64, device=dev)
                    l2 = torch.empty(1, dtype=torch.float64, device=dev)
                    B.ensemble_scores(g2, m, B.CB_FP32, out=(S2, l2))
                    i2, v2 = B.topk(S2, k)
                    host_idx.copy_(i2, non_blocking=True)
                    host_val.copy_(v2, non_blocking=True)
                    host_ls.copy_(l2, non_blocking=True)
                    torch.cuda.current_stream().synchronize()  # this step only
                    g2.close()

        n_pipe = 8
        pipelined(2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pipelined(n_pipe)
        torch.cuda.synchronize()
        e2e_ms = 1e3 * (time.perf_counter() - t0) / n_pipe
        e2e = {"value": units / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms, "steps": n_pipe,
               "pipelined": "upload of step q+1 overlaps compute of step q (second host thread and stream)",
               "serial_ms_per_step": serial_ms, "serial_value": units / (serial_ms * 1e-3),
               "serial_steps": n_e2e, "upload_ms": sum(up_ms) / len(up_ms),
               "api": "cb_graph_upload(pinned host) + cb_ensemble_scores + cb_topk + D2H + cb_graph_free"}
        # the same shape with the backgrounds generated on the device
        # (cb_graph_generate_er: same n_r, mean degree and target; its own ER model)
        if ens.meta.get("dbar") is not None and ens.target_edges is not None:
            ns = [g.n for g in ens.graphs]
            gen_ms, gen_units = [], []

            def gen_step(q):
                u0 = time.perf_counter()
                with B.GraphSet.generate_er(ns, ens.meta["dbar"], synth.seed_for(77, q),
                                            ens.target_edges) as g3:
                    gen_ms.append(1e3 * (time.perf_counter() - u0))
                    gen_units.append(sum(g3.nnz) * m)
                    S3 = torch.empty(g3.n_max, dtype=torch.float64, device=dev)
                    l3 = torch.empty(1, dtype=torch.float64, device=dev)
                    B.ensemble_scores(g3, m, B.CB_FP32, out=(S3, l3))
                    i3, v3 = B.topk(S3, k)
                    host_idx.copy_(i3, non_blocking=True)
                    host_val.copy_(v3, non_blocking=True)
                    host_ls.copy_(l3, non_blocking=True)
                    torch.cuda.synchronize()

            gen_step(0)
            gen_ms.clear()
            gen_units.clear()
            t0 = time.perf_counter()
            for q in range(n_e2e):
                gen_step(q + 1)
            g_ms = 1e3 * (time.perf_counter() - t0) / n_e2e
            extra["e2e_generated_on_device"] = {
                "value": sum(gen_units) / len(gen_units) / (g_ms * 1e-3), "unit": UNIT,
                "ms_per_step": g_ms, "generate_ms": sum(gen_ms) / len(gen_ms), "steps": n_e2e,
                "h2d_bytes_per_step": 8 * len(ens.target_edges) + 20 * len(ns), "d2h_bytes_per_step": d2h,
                "api": "cb_graph_generate_er + cb_ensemble_scores + cb_topk + D2H + cb_graph_free"}

    if rank == 0 and not args.skip_extra:
        # sub-graph centrality (eq. 3) of the top-k nodes in the largest realisation
        r_big = max(range(len(gs.n)), key=lambda r: gs.n[r])
        B.ensemble_scores(gs, m, B.CB_FP32, out=(S, ls))
        B.topk(S, k, out=(idx, val))
        cand = idx.clone()
        sc = torch.empty(k, dtype=torch.float64, device=dev)
        B.cb_subgraph_centrality(gs.h, r_big, m, B.CB_FP32, k, cand.data_ptr(), sc.data_ptr(),
                                 ls1.data_ptr(), stream.cuda_stream)
        t0 = time.perf_counter()
        B.cb_subgraph_centrality(gs.h, r_big, m, B.CB_FP32, k, cand.data_ptr(), sc.data_ptr(),
                                 ls1.data_ptr(), stream.cuda_stream)
        sc_ms = 1e3 * (time.perf_counter() - t0)
        extra["subgraph_centrality_topk"] = {
            "ms": sc_ms, "nodes": k, "m": m, "realisation_n": gs.n[r_big],
            "realisation_nnz": gs.nnz[r_big],
            "api": "cb_subgraph_centrality (k copies of the realisation, k Lanczos runs, Gauss rule)"}

    if rank == 0 and not args.skip_extra:
        # restarted Lanczos: the same total depth m as cycles of m/5 steps, so
        # the basis held on the device is (m/5 + 1) vectors instead of m + 1
        mr, cyc = max(1, m // 5), 5
        Sr = torch.empty_like(S)
        lr = torch.empty_like(ls)
        B.ensemble_scores_restarted(gs, mr, cyc, B.CB_FP32, out=(Sr, lr))
        B.ensemble_scores(gs, m, B.CB_FP32, out=(S, ls))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.ensemble_scores_restarted(gs, mr, cyc, B.CB_FP32, out=(Sr, lr))  # synchronous
        r_ms = 1e3 * (time.perf_counter() - t0)
        a = Sr.cpu().numpy() * math.exp(float(lr.item()) - float(ls.item()))
        b = S.cpu().numpy()
        head = b >= 1e-3 * b.max()
        nodes = sum(gs.n)
        extra["restarted"] = {
            "m": mr, "cycles": cyc, "ms": r_ms, "unit": UNIT,
            "value": sum(g.nnz for g in ens.graphs) * mr * cyc / (r_ms * 1e-3),
            "basis_bytes": 4 * (mr + 1) * nodes, "plain_basis_bytes": 4 * (m + 1) * nodes,
            "head_max_rel_vs_plain": float(np.max(np.abs(a - b)[head] / b[head])),
            "api": "cb_ensemble_scores_restarted (FP32), wall time of one synchronous call"}

    if rank == 0 and not args.skip_extra:
        # full reorthogonalisation (CB_REORTH), the oracle's scheme, on the
        # device: its cost on the same workload (third call: a graph replay)
        B.ensemble_scores(gs, m, B.CB_FP32, out=(S, ls))
        b = S.cpu().numpy()
        ls_plain = float(ls.item())
        Sr2 = torch.empty_like(S)
        lr2 = torch.empty_like(ls)
        for _ in range(2):
            B.ensemble_scores(gs, m, B.CB_FP32 | B.CB_REORTH, out=(Sr2, lr2))
        torch.cuda.synchronize()
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        B.ensemble_scores(gs, m, B.CB_FP32 | B.CB_REORTH, out=(Sr2, lr2))
        q1.record(stream)
        torch.cuda.synchronize()
        a = Sr2.cpu().numpy() * math.exp(float(lr2.item()) - ls_plain)
        head = b >= 1e-3 * b.max()
        extra["reorth"] = {"ms": q0.elapsed_time(q1),
                           "head_max_rel_vs_plain": float(np.max(np.abs(a - b)[head] / b[head])),
                           "api": "cb_ensemble_scores(CB_FP32 | CB_REORTH), graph replay"}

    if rank == 0 and not args.skip_extra and args.workload == "ensemble":
        # the other configurations, each timed the same way: the 10M-node BA
        # graph (two-phase SpMV; the tiled-CSR kernel beside it), the three
        # 1e5-node single backgrounds in FP32 and FP64, and forward + adjoint
        legs = {}
        big = workload("large")
        legs["large"] = extra_leg(B, "large", 5, 3, dev, built=big, tune=True)
        csr = extra_leg(B, "large", 3, 2, dev, csr_only=True, built=big)
        legs["large"]["csr_only"] = {"ms_per_step": csr["f32"]["ms_per_step"],
                                     "spmv_avg_ms": csr["f32"]["roofline"]["avg_launch_ms"],
                                     "frac": csr["f32"]["roofline"]["frac"]}
        del big
        legs["single_1e5"] = {kind: extra_leg(B, "c2" + kind, 10, 3, dev, precs=(0, 1))
                              for kind in ("er", "ba", "ws")}
        legs["grad"] = extra_leg(B, "grad", 5, 3, dev)
        # the measured choice of SpMV width and path on the default workload
        # (after its timing; the autotuner's cache stores the same)
        legs["ensemble_tuned"] = tuned_choice(B, gs)
        B.cb_graph_set_path(gs.h, B.CB_PATH_AUTO)
        extra["configs"] = legs

    cpu = None
    if rank == 0 and not args.skip_extra and world == 1:
        v, done, t, res = cpu_oracle_sample(ens, m, budget_s=15.0, want={0, 1})
        extra["cpu_baseline_1core"] = {
            "value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {done} of {len(ens.graphs)} realisations, FP64 Lanczos with full "
                      f"reorthogonalisation, m={m}, {t:.1f} s"}
        # all host cores: a bounded sample of about 4 realisations per worker
        pool = OraclePool(ens.graphs[: min(len(ens.graphs), 4 * (os.cpu_count() or 1))])
        try:
            pool.run(m, list(range(min(pool.procs, len(pool.graphs)))))  # worker start-up
            wall, busy = pool.run(m, list(range(len(pool.graphs))))
        finally:
            pool.close()
        cpu = {"value": sum(g.nnz * m for g in pool.graphs) / wall, "unit": UNIT, "cores": pool.procs,
               "kind": "oracle",
               "sample": f"first {len(pool.graphs)} of {len(ens.graphs)} realisations, FP64 Lanczos with "
                         f"full reorthogonalisation, m={m}, {pool.procs} worker processes "
                         f"(one single-threaded oracle each), {wall:.1f} s wall, {busy:.1f} s busy"}
        # parity on the sampled realisations (CUDA FP32 per-graph call vs oracle)
        worst = 0.0
        for r, (th_o, y_o) in res.items():
            y_g = torch.empty(ens.graphs[r].n, dtype=torch.float64, device=dev)
            B.cb_communicability(gs.h, r, m, B.CB_FP32, y_g.data_ptr(), ls1.data_ptr(), None,
                                 stream.cuda_stream)
            torch.cuda.synchronize()
            th_g = float(ls1.item())
            a = y_g.cpu().numpy() * math.exp(th_g - th_o)
            head = y_o >= 1e-3 * y_o.max()
            worst = max(worst, float(np.max(np.abs(a - y_o)[head] / y_o[head])))
        extra["parity_sample"] = {"realisations": sorted(res), "fp32_head_max_rel": worst, "tol": 1e-4}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(desc, l2="inputs larger than L2 (cols %.1f GB)" % (
                    4 * sum(g.nnz for g in ens.graphs) / 1e9), parallelism=f"replicas{world}",
                    precision="FP32 Krylov vectors, FP64 scalars / tridiagonal / ensemble sum"),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
                "clocks": clk}
        line.update(extra)
        print(json.dumps(line), flush=True)
    gs.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
