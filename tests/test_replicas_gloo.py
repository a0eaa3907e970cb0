"""The N>1 path of the benchmark on CPU: world_size-2 gloo process groups.

The workload shards into independent replicas (one lattice per rank, no data-path
collective).  The only cross-rank operations are the barrier and the max-over-ranks of the
timing; these run here with the gloo backend."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.rank_info()
    t = 1.0 + 0.5 * rank  # rank 1 is slower
    dist.barrier()
    q.put((r, w, local, bench.max_over_ranks(t, dist, "cpu"), bench.replica_seed(r)))
    dist.destroy_process_group()


def test_max_over_ranks_and_replica_seeds_gloo():
    world, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[3] == 1.5 for o in out)  # every rank sees the slowest rank's time
    assert out[0][4] != out[1][4]         # replicas evolve different lattices


def test_aggregate_throughput_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_gsu(1000, 4, 10, 2.0) == pytest.approx(4 * 1000 * 10 / 2.0 / 1e9)


def test_reference_arm_under_torchrun_prints_once():
    """`bench.py --impl reference` under torchrun with 2 ranks: rank 0 times the CPU oracle and
    prints one JSON line; rank 1 exits without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), "bench.py", "--impl", "reference",
           "--steps", "3", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0 and line["e2e"]["h2d_bytes_per_step"] == 0
