"""Host logic of bench.py without a GPU: the max-over-ranks aggregation of independent replicas on a
2-rank gloo process group, the algorithmic byte model, and the reference arm's JSON line."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank                     # rank 1 is the slowest
    m = bench.reduce_max(ms, dist)
    q.put((rank, m, bench.job_rate(world, 1000 * 20, m * 1e-3)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [m for _, m, _ in res] == [15.0, 15.0]
    assert res[0][2] == pytest.approx(2 * 1000 * 20 / 0.015)


def test_reduce_max_without_group_and_byte_model():
    assert bench.reduce_max(3.5, None) == 3.5
    b = bench.algorithmic_bytes_per_particle_step(3, 4, 1)
    assert b["total"] == pytest.approx(sum(v for k, v in b.items() if k != "total"))
    assert "swap" in b and "swap" not in bench.algorithmic_bytes_per_particle_step(3, 1, 1)


@pytest.mark.slow
def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == "particle-steps/sec"
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_profile_traffic_follows_the_code_not_the_comments(tmp_path, monkeypatch):
    import bench
    src = tmp_path / "k.cu"
    src.write_text("// header\\n__global__ void k() { int a = 1; /* note */ }\\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = bench.code_sha256(str(src))[:16]
    (prof / "p.md").write_text(f"code_sha256: {h}\\ndram_bytes_per_launch.k: 1234\\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic_from_profile(str(src), "p.md", "k") == 1234.0
    src.write_text("// another header\\n__global__ void k() {  int a = 1;  }\\n")      # comments only
    assert bench._traffic_from_profile(str(src), "p.md", "k") == 1234.0
    src.write_text("__global__ void k() { int a = 2; }\\n")                              # code changed
    assert bench._traffic_from_profile(str(src), "p.md", "k") is None


def test_flops_per_pair_is_the_oracles_count():
    # the roofline's FLOP unit equals the operations of one ordered pair in the oracle's pair function
    # (flux and one end's accumulation), counted on a counting scalar type
    from oracle import orc
    assert bench.FLOPS_PER_PAIR == orc.flops_per_pair()
