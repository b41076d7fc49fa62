"""The benchmark's multi-process host logic on CPU, world size 2 (the single problem runs as
replicas, one per GPU, with no data-path collective): the job's time is the largest over the
ranks (gloo all-reduce), and under torchrun the oracle arm prints exactly one JSON line, from
rank 0, while the other rank exits 0 without work."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _torchrun(args, tmp_cwd, timeout=600):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port())] + args
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    return subprocess.run(cmd, cwd=tmp_cwd, capture_output=True, text=True, timeout=timeout, env=env)


WORKER = """
import json, os, sys
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank = dist.get_rank()
v = bench.max_over_ranks(1.5 + rank, dist, "cpu")
alone = bench.max_over_ranks(7.0, None, "cpu")
line = json.dumps({"rank": rank, "world": dist.get_world_size(), "max": v, "alone": alone})
# each rank writes its own file: the ranks share one stdout pipe, where two lines can interleave
with open(os.path.join(sys.argv[1], f"rank{rank}.json"), "w") as fh:
    fh.write(line)
dist.destroy_process_group()
"""


def test_max_over_ranks_gloo_world_size_2(tmp_path):
    script = tmp_path / "worker.py"
    script.write_text(WORKER)
    out = _torchrun([str(script), str(tmp_path)], str(tmp_path))
    assert out.returncode == 0, out.stderr[-2000:]
    rows = sorted((json.loads((tmp_path / f"rank{r}.json").read_text()) for r in (0, 1)), key=lambda r: r["rank"])
    assert [r["rank"] for r in rows] == [0, 1]
    assert all(r["world"] == 2 and r["max"] == 2.5 and r["alone"] == 7.0 for r in rows)


def test_reference_arm_under_torchrun_prints_once_from_rank_0():
    out = _torchrun([os.path.join(ROOT, "bench.py"), "--impl", "reference", "--size", "small", "--gpus", "2",
                     "--steps", "1", "--warmup", "0"], ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0
