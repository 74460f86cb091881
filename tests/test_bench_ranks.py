"""The bench's multi-rank path on CPU (gloo, world size 2): whole-job timing
over ranks, and the reference arm launched under torch.distributed.run."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2)
    ms, value = bench.combine_ranks([10.0, 20.0][rank], [100, 300][rank], dist, "cpu")
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_combine_ranks_gloo():
    ctx = torch.multiprocessing.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, port, out)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    # slowest rank's time, all ranks' units
    assert out[0] == out[1] == (20.0, 400 / 0.020)


def test_combine_ranks_single():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.combine_ranks(8.0, 400) == (8.0, 50_000.0)


def test_reference_arm_under_torchrun():
    """Rank 0 alone runs the oracle and prints one JSON line; rank 1 exits 0."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--workload", "small", "--steps", "1", "--warmup", "0", "--gpus", "2"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, res.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_traffic_guard_hashes_the_kernel_sources():
    """roofline.traffic is reported only while the SpMV kernel, its epilogue,
    the format builder and the blocked constants hash to the captured version;
    the anchors that cut those regions out of the sources must still exist."""
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    for kind in ("blocked", "twophase"):
        h = bench._kernel_sources_hash(kind)
        assert len(h) == 16 and int(h, 16) >= 0
        t = bench._TRAFFIC[kind]
        if t["bytes_per_edge"] is not None:  # at least the 3 B of a blocked element
            assert t["bytes_per_edge"] > 3.0


def test_launch_and_path_accounting():
    """The launch counts the bench claims follow the library's paths: one launch
    of all m steps for realisations of at most 8192 nodes, three per Lanczos
    step otherwise (four on the two-phase path), and one top-k launch for at
    most 4096 scores (15 otherwise)."""
    sys.path.insert(0, ROOT)
    import bench

    class G:
        def __init__(self, n, nnz):
            self.n, self.nnz = n, nnz

    class E:
        def __init__(self, graphs):
            self.graphs = graphs

    assert bench.spmv_path(E([G(500, 4000)] * 10)) == "small"
    assert bench.spmv_path(E([G(8192, 1 << 20)])) == "small"
    assert bench.spmv_path(E([G(8193, 80_000)]), csr_only=True) == "csr"
    assert bench.spmv_path(E([G(10_000_000, 160_000_000)])) == "twophase"
    assert bench.launches_for(20, "small", n_scores=500) == 2 + 1 + 1 + 2 + 1
    assert bench.launches_for(25, "blocked", n_scores=400_000) == 2 + 3 * 25 + 1 + 2 + 15
    assert bench.launches_for(40, "twophase", n_scores=10_000_000) == 2 + 4 * 40 + 1 + 2 + 15
    assert bench.launches_for(30, "small", with_grad=True, n_scores=1000) == 7 + 4 + 3
