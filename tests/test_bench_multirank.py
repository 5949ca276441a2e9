"""The benchmark's multi-rank host logic on CPU, two gloo ranks launched the way a
multi-GPU run is (torch.distributed.run, rendezvous on 127.0.0.1): rank setup, the
max-over-ranks timing and the sum over ranks that the whole-job value uses, the
barrier, and the reference arm, which only rank 0 runs and prints while the other
rank exits 0 without work.  No CUDA device is touched."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytest.importorskip("torch")


def free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def torchrun(args, timeout=600):
    env = dict(os.environ)
    env["CUDA_VISIBLE_DEVICES"] = ""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port())] + args
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)


def json_lines(text):
    return [json.loads(line) for line in text.splitlines() if line.startswith("{")]


def test_reductions_and_barrier_over_two_gloo_ranks(tmp_path):
    script = tmp_path / "ranks.py"
    script.write_text(
        "import json, sys\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "import bench\n"
        "ws, rank, local = bench.dist_setup()\n"
        "import torch.distributed as dist\n"
        "assert dist.get_backend() == 'gloo'\n"
        "m = bench.max_over_ranks(1.5 + rank, ws)\n"
        "s = bench.sum_over_ranks(1.0 + 2.0 * rank, ws)\n"
        "bench.barrier(ws)\n"
        f"out = open({str(tmp_path)!r} + '/rank%d.json' % rank, 'w')\n"
        "out.write(json.dumps({'ws': ws, 'rank': rank, 'local': local, 'max': m, 'sum': s}))\n"
        "out.close()\n"
        "dist.destroy_process_group()\n")
    r = torchrun([str(script)], timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    # one file per rank: the two ranks' stdout lines may interleave
    lines = [json.loads((tmp_path / f"rank{q}.json").read_text()) for q in range(2)]
    assert [d["rank"] for d in lines] == [0, 1]
    for d in lines:
        assert d["ws"] == 2 and d["local"] == d["rank"]
        assert d["max"] == 2.5  # the slower rank's time
        assert d["sum"] == 4.0  # both ranks' units


def test_reference_arm_prints_once_from_rank_zero():
    """One timed step of the bounded oracle sample (524,288 cells) on rank 0."""
    r = torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                  "--warmup", "0"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 1
    assert d["value"] > 0 and d["unit"] == "cell-updates/s"
    assert d["e2e"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
