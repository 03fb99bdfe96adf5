"""Multi-rank host logic on CPU (gloo, world size 2): windows are independent,
so ranks share only the timing reduction and the solved-window count."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2105_06975_gb300 import ranks  # noqa: E402


def test_partition_by_cost_is_complete_disjoint_and_balanced():
    costs = [5.0, 1.0, 7.0, 3.0, 3.0, 2.0, 9.0, 4.0]
    for world in (1, 2, 3, 8, 11):
        parts = ranks.partition_by_cost(costs, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT: no rank exceeds the mean by more than the largest single window
        assert max(loads) <= sum(costs) / world + max(costs)
    assert ranks.partition_by_cost(costs, 2) == ranks.partition_by_cost(list(costs), 2)  # deterministic
    with pytest.raises(ValueError):
        ranks.partition_by_cost(costs, 0)


def test_window_seeds_are_distinct_per_rank():
    seeds = [ranks.window_seed(2, r) for r in range(8)]
    assert len(set(seeds)) == 8 and seeds[0] == 2000


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = ranks.dist_info()
        costs = [float(c) for c in range(1, 11)]
        mine = ranks.partition_by_cost(costs, w)[r]
        ms = 10.0 + 5.0 * r               # rank 1 is the slow one
        thr, ms_max = ranks.job_throughput(len(mine), ms)
        out.put((r, sorted(mine), ms_max, thr, ranks.max_over_ranks(float(r))))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_only_timing_and_counts():
    mp = pytest.importorskip("torch.multiprocessing")
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
    (r0, w0, ms0, t0, m0), (r1, w1, ms1, t1, m1) = res
    assert sorted(w0 + w1) == list(range(10)) and not set(w0) & set(w1)
    assert ms0 == ms1 == 15.0                      # max over ranks
    assert t0 == t1 == pytest.approx(10 * 1e3 / 15.0)  # all windows / slowest rank
    assert m0 == m1 == 1.0
