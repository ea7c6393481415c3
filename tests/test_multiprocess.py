"""The multi-process path of bench.py on the CPU: two ranks over gloo on 127.0.0.1. The
path has no data-path collective (each rank validates or plans its own seeded inputs); the
ranks meet only in the barrier around the timed region and in the reductions of its
results (the slowest rank's time, the units of all ranks)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, queue):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank), CPRRTC_BENCH_GLOO="1")
    import torch.distributed as dist
    import bench
    w, r, _ = bench.init_dist()
    res = {"world": w, "rank": r, "backend": dist.get_backend(),
           "max": bench.max_over_ranks(1.5 + r, w), "sum": bench.sum_over_ranks(10 * (r + 1), w)}
    bench.barrier(w)
    # weak scaling: each rank's problems come from its own seed
    scenes = bench.planner_scenes(2, 2 + 1000 * r)
    res["first_obstacle"] = [float(x) for x in scenes[0].sph[0]]
    res["reference_line"] = bench.reference_arm_plan(None, w, r) if r != 0 else "rank 0"
    dist.destroy_process_group()
    queue.put(res)


def test_two_ranks_over_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    results = [queue.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    res = sorted(results, key=lambda d: d["rank"])
    assert [d["rank"] for d in res] == [0, 1]
    assert all(d["world"] == 2 and d["backend"] == "gloo" for d in res)
    assert all(d["max"] == 2.5 for d in res)        # the slowest rank's time
    assert all(d["sum"] == 30.0 for d in res)       # units of both ranks
    assert res[0]["first_obstacle"] != res[1]["first_obstacle"]
    assert res[1]["reference_line"] is None         # only rank 0 runs the CPU arm


def test_single_rank_reductions_are_identity():
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.sum_over_ranks(7, 1) == 7
    assert bench.init_dist()[0] == int(os.environ.get("WORLD_SIZE", "1"))
