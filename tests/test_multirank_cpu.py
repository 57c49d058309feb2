"""The N > 1 path of bench.py on CPU: two gloo ranks shard the plate
workload without overlap and combine their timings into the whole-job
numbers (slowest rank's time, summed solves)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
import workloads as W  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        P, probs = bench.workload(3, 4, rank, world)
        ms = [1500.0, 2500.0][rank]
        acc, tot = [3, 4][rank], 4
        res = bench.combine_ranks(ms, acc, tot, dist, device="cpu")
        out[rank] = (P.tolist(), [p.L for p in probs], res)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_combine():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        got = dict(out)
    full = W.plate_params(2, 4 * world)
    shards = [np.asarray(got[r][0]) for r in range(world)]
    # every problem solved by exactly one rank
    np.testing.assert_array_equal(np.concatenate(shards), np.concatenate([full[0::2], full[1::2]]))
    assert all(len(sh) == 4 for sh in shards)
    assert all(L == 3 for r in range(world) for L in got[r][1])
    for r in range(world):
        ms, acc, tot, value = got[r][2]
        assert ms == 2500.0 and acc == 7 and tot == 8
        assert value == pytest.approx(7 / 2.5)


def test_single_rank_combine_is_identity():
    ms, acc, tot, value = bench.combine_ranks(2000.0, 2, 2)
    assert (ms, acc, tot) == (2000.0, 2.0, 2.0)
    assert value == pytest.approx(1.0)
