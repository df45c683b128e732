"""The bench's multi-rank path on CPU: two gloo ranks split the views into
disjoint sets of the same size that cover the whole set, and the whole-job
figures take the slowest rank's time and everyone's units."""
import importlib.util
import json
import os
import socket

import numpy as np
import torch
import torch.distributed as tdist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        cams = b.rank_cameras(6, world, rank, 8)
        times, units = b.reduce_over_ranks([10.0 + 5 * rank, 3.0 - rank], 100 + 7 * rank, torch.device("cpu"))
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"eyes": [list(map(float, c.eye)) for c in cams], "times": times, "units": units}, f)
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks_split_views_and_reduce_timing(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    r = [json.load(open(tmp_path / f"r{i}.json")) for i in range(world)]
    # disjoint, same size, together the full Fibonacci set
    full = _bench().rank_cameras(6 * world, 1, 0, 8)
    eyes = [tuple(e) for x in r for e in x["eyes"]]
    assert len(r[0]["eyes"]) == len(r[1]["eyes"]) == 6
    assert len(set(eyes)) == 12
    assert sorted(eyes) == sorted(tuple(map(float, c.eye)) for c in full)
    # max of each time, sum of the units, the same on every rank
    for x in r:
        assert x["times"] == [15.0, 3.0]
        assert x["units"] == 207.0


def test_single_process_reduction_is_the_identity():
    b = _bench()
    assert b.reduce_over_ranks([4.0, 2.0], 9, torch.device("cpu")) == ([4.0, 2.0], 9.0)
    cams = b.rank_cameras(5, 1, 0, 4)
    assert len(cams) == 5 and np.allclose(np.linalg.norm(cams[0].eye), 3.0)
