"""The N > 1 path on CPU with gloo, world size 2 (no GPU).

The MCQSG chains are independent, so ranks shard the work with no data-path
collective: each rank simulates its own samples, and only the timing is
reduced (max over ranks).  These tests run the benchmark's multi-rank host
logic and check that sharded oracle runs reproduce the single-process run.
"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import oracle
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # sharded oracle run: rank r simulates samples [2r, 2r+2) of one instance
        k, kt = oracle.ladder_linear(0.25, 0.45, 4, 1.0)
        st = oracle.new_state(4, 8, k, kt, 3, seed=5, a_lo=2 * rank, n_a=2)
        oracle.run(st, 6, measure_every=3)
        A = torch.from_numpy(st.A.copy())
        S = torch.from_numpy(st.S.copy())
        As = [torch.zeros_like(A) for _ in range(world)]
        Ss = [torch.zeros_like(S) for _ in range(world)]
        dist.all_gather(As, A)          # result gather only, after the run
        dist.all_gather(Ss, S)
        # benchmark timing: max over ranks
        t = torch.tensor([10.0 + rank], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        seed = bench.rank_seed(1, rank)
        seeds = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(seeds, torch.tensor([seed]))
        if rank == 0:
            out.put({"A": torch.cat(As).numpy(), "S": torch.cat(Ss).numpy(), "tmax": float(t.item()),
                     "seeds": [int(x.item()) for x in seeds],
                     "value": bench.job_value(float(t.item()), 1000, world)})
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_without_collectives():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle
    k, kt = oracle.ladder_linear(0.25, 0.45, 4, 1.0)
    whole = oracle.new_state(4, 8, k, kt, 3, seed=5, a_lo=0, n_a=4)
    oracle.run(whole, 6, measure_every=3)
    assert np.array_equal(res["A"], whole.A)
    assert np.array_equal(res["S"], whole.S)
    assert res["tmax"] == 11.0
    assert len(set(res["seeds"])) == 2
    assert res["value"] == pytest.approx(11.0 * 1e9 / 2000)
