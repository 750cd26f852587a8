"""The multi-rank path of bench.py on the CPU (gloo, world size 2): the job
time is the slowest rank's, the job rate counts the units of every rank,
and under torchrun only rank 0 prints the reference arm's line."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.0 + rank, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, t, bench.job_rate(world, 1000, 8, t)))


def test_max_over_ranks_and_job_rate_with_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [t for _, t, _ in res] == [2.0, 2.0]          # the slower rank's time on both
    assert all(v == 2 * 1000 * 8 / 2.0 for _, _, v in res)


@pytest.mark.slow
def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def test_traffic_is_scaled_by_points_and_kept_to_the_captured_kernel(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = {"kernel_hash": bench.kernel_hash(),
           "fp64": {"points": 1000, "dram_bytes_read": 3.0e6, "dram_bytes_write": 1.0e6},
           "mixed": {"points": 2000, "dram_bytes_read": 1.0e6, "dram_bytes_write": 1.0e6}}
    (prof / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # kernel_hash reads the kernel sources under ROOT: keep the real ones
    monkeypatch.setattr(bench, "kernel_hash", lambda h=rec["kernel_hash"]: h)
    assert bench.load_traffic(5000) == 2.0e7                 # 4 kB per point x 5000
    assert bench.load_traffic(5000, "mixed") == 5.0e6        # its own record: 1 kB per point
    assert bench.load_traffic(5000, "other") is None         # a kernel instance without a record
    assert bench.load_traffic(5000, mesh=True) is None
    rec["kernel_hash"] = "0" * 16                            # sources changed since the capture
    (prof / "traffic.json").write_text(json.dumps(rec))
    assert bench.load_traffic(5000) is None
