"""The N-rank paths of bench.py on CPU, with two gloo ranks.  The solve of one
graph does not shard: each rank runs its own replica and the job time is the
slowest rank's.  The batched workloads shard their independent problems
(right-hand sides, graphs) over the ranks and add up the units."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.slowest_rank_ms(10.0 * (rank + 1), dist, "cpu")   # rank r took 10 (r+1) ms
    dist.barrier()
    out.put((rank, ms, bench.job_value(world, 1000.0, ms)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
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
    assert [r[1] for r in res] == [20.0, 20.0]
    # 2 ranks x 1000 units in 20 ms
    assert res[0][2] == pytest.approx(2 * 1000.0 / 0.020)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--workload", "grid64"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env = dict(os.environ, RANK="0", WORLD_SIZE="2", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--workload", "grid64"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0
    import json
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def _shard_worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = W.er_batch_sizes(40, 50, 400, seed=3).tolist()
    mine = bench.shard_lpt(sizes, world)[rank]
    g, gptr = W.er_batch(40, 50, 400, seed=3, only=mine)
    units = bench.total_units(float(g.m), dist, "cpu")          # one "cycle" per graph
    ms = bench.slowest_rank_ms(5.0 + rank, dist, "cpu")
    dist.barrier()
    out.put((rank, mine, int(g.m), units, ms))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_the_graphs():
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import workloads as W
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every graph on exactly one rank; the ranks' unions together are the whole batch
    assert sorted(res[0][1] + res[1][1]) == list(range(40))
    whole, _ = W.er_batch(40, 50, 400, seed=3)
    assert res[0][2] + res[1][2] == whole.m
    assert res[0][3] == res[1][3] == float(whole.m)       # units summed over ranks
    assert res[0][4] == res[1][4] == 6.0                  # the slowest rank's time


def test_shard_helpers():
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    for count in (64, 7, 1):
        for world in range(1, 10):
            blocks = [bench.shard_block(count, world, r) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == count
            assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
            sizes = [c1 - c0 for c0, c1 in blocks]
            assert max(sizes) - min(sizes) <= 1
    loads = W.er_batch_sizes(500, 1000, 200_000, seed=7).tolist()
    assert bench.shard_lpt(loads, 1) == [list(range(500))]    # one rank: the unsharded batch, in order
    for world in (2, 4, 8):
        share = bench.shard_lpt(loads, world)
        assert sorted(k for s in share for k in s) == list(range(500))
        tot = [sum(loads[k] for k in s) for s in share]
        # largest-first list scheduling: no rank exceeds the mean by more than one item
        assert max(tot) <= sum(loads) / world + max(loads)
        assert max(tot) - min(tot) <= max(loads)
