"""The multi-GPU benchmark path without GPUs: two gloo ranks on the CPU.

bench.py --gpus N runs N independent replicas (the method does not shard);
the whole-job figures are the slowest rank's time and the sum of the ranks'
work, and only rank 0 runs and prints the reference arm."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seconds = [1.5, 2.5][rank]
    units = [1000, 3000][rank]
    t, n = bench.reduce_over_ranks(seconds, units, "cpu")
    # the reference arm: rank 0 alone prints one line, the other ranks exit quietly
    buf = io.StringIO()

    class Args:
        gpus, steps, warmup = world, 0, 0
    if rank != 0:
        with redirect_stdout(buf):
            bench.run_reference(Args)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, n, buf.getvalue()))


def test_two_gloo_ranks_take_max_time_and_sum_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, n, printed in out:
        assert t == 2.5 and n == 4000
        if rank != 0:
            assert printed == ""


def test_reference_arm_line_on_the_cpu():
    # the reference arm needs no GPU: one JSON line with the contract's keys,
    # the oracle timed on its bounded sample
    import json
    import subprocess
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "triangles/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    assert d["config"]["workload"].startswith("noise512")
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "triangles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
