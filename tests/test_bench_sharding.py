"""Host-side logic of the multi-GPU report, on two gloo ranks (CPU): disjoint account
shards, max-over-ranks timing and summed certified counts."""
import os
import socket

import pytest
import torch.multiprocessing as tmp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 25.0 * rank                      # rank 1 is the slower one
        certified = 490 + rank
        out[rank] = (bench.shard_first_account(rank),
                     bench.reduce_over_ranks(dist, ms, "max", "cpu"),
                     bench.reduce_over_ranks(dist, certified, "sum", "cpu"))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = tmp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    firsts = sorted(out[r][0] for r in range(2))
    assert firsts == [0, bench.M_ACCOUNTS]             # disjoint blocks of accounts
    for r in range(2):
        assert out[r][1] == pytest.approx(125.0)        # timing: max over ranks
        assert out[r][2] == pytest.approx(981.0)        # certified: sum over ranks


def test_single_rank_is_identity():
    assert bench.reduce_over_ranks(None, 3.5, "max", "cpu") == 3.5
    assert bench.shard_first_account(0) == 0


def test_iteration_histogram_bins():
    import numpy as np
    iters = np.asarray([3, 9, 10, 38, 45, 45, 53])
    h = bench.iter_histogram(iters)
    assert h == {"0-9": 2, "10-19": 1, "30-39": 1, "40-49": 2, "50-59": 1}
    assert sum(h.values()) == iters.size
    assert bench.iter_histogram(np.asarray([], dtype=int)) == {}


def test_cpu_model_is_a_nonempty_string():
    m = bench._cpu_model()
    assert isinstance(m, str) and m.strip()
