"""Multi-rank host logic of bench.py on the CPU (gloo, world size 2): the
job time is the slowest rank's, and under torchrun only rank 0 prints the
result line (the GPU arm runs one independent replica per rank: no data-path
collective)."""
import json
import os
import re
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


def _torchrun(args, timeout=240):
    env = dict(os.environ, OMP_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port())] + args
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)


def test_max_over_ranks_is_the_slowest_rank(tmp_path):
    script = tmp_path / "ranks.py"
    script.write_text(
        "import json, sys\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "import torch.distributed as dist\n"
        "dist.init_process_group('gloo')\n"
        "import bench\n"
        "r = dist.get_rank()\n"
        "print(json.dumps({'rank': r, 'max': bench.max_over_ranks(1.5 + 2.0 * r),"
        "}), flush=True)\n"
        "dist.destroy_process_group()\n")
    p = _torchrun([str(script)])
    assert p.returncode == 0, p.stderr[-2000:]
    # the two ranks print concurrently: their lines may share one line of output
    lines = [json.loads(m) for m in re.findall(r"\{[^{}]*\}", p.stdout)]
    assert sorted(d["rank"] for d in lines) == [0, 1]
    assert all(d["max"] == 3.5 for d in lines)


def test_max_over_ranks_without_a_group_is_the_value():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.25) == 2.25


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    p = _torchrun(["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                   "--cpu-sample-n", "1024"])
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [json.loads(l) for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["config"]["workload"].startswith("three-layer-1048576")
