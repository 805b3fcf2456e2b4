"""Host logic of bench.py's multi-rank path (replicas, one rank per GPU),
exercised with world size 2 on the gloo backend (CPU): shots are sharded
without overlap, the time is the maximum over ranks and the work the sum."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    shots = bench.shard_shots(8, world, rank, 6)
    t, u = bench.aggregate(100.0 + 50.0 * rank, 1e9 * (rank + 1), world, torch.device("cpu"))
    q.put((rank, shots, t, u))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_and_aggregate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, t0, u0), (r1, s1, t1, u1) = out
    assert set(s0).isdisjoint(s1) and set(s0) | set(s1) <= set(range(8))
    assert s0 == [0, 2, 4, 6, 0, 2] and s1 == [1, 3, 5, 7, 1, 3]
    assert t0 == t1 == 150.0
    assert u0 == u1 == 3e9


def test_single_rank_owns_every_shot():
    import bench
    assert bench.shard_shots(8, 1, 0, 10) == [0, 1, 2, 3, 4, 5, 6, 7, 0, 1]


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference times the FP64 oracle on the host cores (no
    GPU) and prints one JSON line with the bench's metric, a cpu_baseline
    describing the run and an e2e object without host-device copies."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "Gpt-updates/s" and d["higher_is_better"] is True
    assert d["metric"].startswith("3D RTM grid-point updates/s") and d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
