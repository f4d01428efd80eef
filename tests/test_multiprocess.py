"""Multi-process paths on the CPU (gloo, world size 2).

The library solves one independent problem per GPU ("replicas": no collective on the data
path); bench.py under torchrun only synchronises the ranks and takes the slowest rank's time,
and its reference arm (the CPU oracle) runs on rank 0 alone. Both pieces of host logic are
exercised here with gloo processes on 127.0.0.1.
"""
import json
import os
import socket
import subprocess
import sys

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, values, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out[rank] = bench.max_over_ranks(values[rank], world, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = free_port()
        values = [3.25, 7.5]
        ps = [ctx.Process(target=_rank_main, args=(r, 2, port, values, out)) for r in range(2)]
        for p in ps:
            p.start()
        for p in ps:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == out[1] == 7.5


def test_reference_arm_under_torchrun_two_ranks():
    # bench.py --impl reference under torch.distributed.run: rank 0 times the oracle and prints
    # one JSON line; rank 1 exits 0 without work.
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "1", "--rows", "2048", "--cols", "256"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["higher_is_better"] is False
    assert d["cpu_baseline"]["kind"] == "oracle" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0
    # full solves of the requested problem, no scaling: the steps timed are the steps asked for
    assert d["steps"] == 2 and len(d["steps_ms"]) == 2
    assert d["config"]["m"] == 2048 and d["config"]["n"] == 256
    assert "scaled" not in json.dumps(d)
