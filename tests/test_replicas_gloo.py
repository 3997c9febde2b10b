"""The several-GPU path on the CPU: two gloo ranks, the timing / count
reductions and the balanced partition of a fixed case list."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    from paper_2603_21869_gb300 import replicas, cases
    r, w, local, on = replicas.setup(backend="gloo")
    assert on and r == rank and w == world
    t_max = replicas.max_over_ranks(1.5 + rank)            # 1.5 and 2.5 -> 2.5
    n_sum = replicas.sum_over_ranks(10 * (rank + 1))        # 10 + 20
    specs = cases.batched_channels(9, seed=4)
    weights = [s.cells for s in specs]
    mine = replicas.partition(weights, world)[rank]
    cells_sum = replicas.sum_over_ranks(sum(weights[i] for i in mine))
    dist.barrier()
    out.put((rank, t_max, n_sum, mine, cells_sum, sum(weights)))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_partition():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, s0, m0, c0, tot), (r1, t1, s1, m1, c1, _) = res
    assert t0 == t1 == 2.5 and s0 == s1 == 30.0
    assert sorted(m0 + m1) == list(range(9)) and not set(m0) & set(m1)   # every case once
    assert c0 == c1 == float(tot)


def test_partition_balances_and_is_deterministic():
    from paper_2603_21869_gb300 import replicas
    w = [5, 1, 4, 2, 3, 3, 8]
    parts = replicas.partition(w, 3)
    assert parts == replicas.partition(w, 3)
    loads = [sum(w[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(w)
    assert sorted(i for p in parts for i in p) == list(range(len(w)))
    assert replicas.partition(w, 1) == [list(range(len(w)))]
